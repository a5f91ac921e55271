"""Pins of the lumped-mass / general-EOS oracle (oracle/lumped.py) against
what the mathematics fixes, independently of the oracle's own formulas:

* for alpha = 1 the lumped weights m_i are the row sums of the consistent
  mass matrix assembled by the C oracle (an independent implementation), and
  1^T M_L x = 1^T M x = int x_h for every x;
* closed form int phi_i = h^d at interior nodes of the regular meshes, and
  sum_i m_i = |Omega|;
* the lumped system converges at second order in L2 on a manufactured
  solution (a wrong lumping weight would stall it at first order or worse);
* with b = 0 (ideal gas) one Newton step is the linear lumped solve and the
  next check sees F = 0;
* Newton recovers a manufactured root, and its residuals fall quadratically;
* the EOS enthalpy reduces to gamma/(gamma-1) Pbar/rho for b = 0;
* the operator on two right triangles equals the hand-derived rows of
  tests/golden/lumped_two_triangles.txt.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import lumped as L
from oracle import projection as PJ
from paper_2301_08357_gb300 import synthetic as S
from tests._quad import element_points


def _mesh(dim, n, jitter=0.0, seed=0):
    coords, conn = S.square_mesh(n) if dim == 2 else S.kuhn_cube_mesh(n)
    if jitter:
        coords = S.jitter_nodes(coords, n, jitter, np.random.default_rng(seed))
    return coords, conn


@pytest.mark.parametrize("dim,n", [(2, 5), (3, 3)])
def test_lumped_weights_are_consistent_mass_row_sums(dim, n):
    coords, conn = _mesh(dim, n, jitter=0.2, seed=1)
    N, E = coords.shape[0], conn.shape[0]
    M = oracle.PressureMatrix(dim, coords, conn, np.zeros(N, np.uint8), np.ones(N), np.ones(E), 1.0, part=1)
    Md = M.dense()
    m = L.lumped_weights(dim, coords, conn)
    assert np.allclose(Md.sum(axis=1), m[M.node_of_free], rtol=1e-13, atol=0)
    x = np.random.default_rng(2).standard_normal(N)
    LM = L.LumpedMatrix(dim, coords, conn, np.zeros(N, np.uint8), np.ones(N), np.ones(E), 0.0)
    assert abs(LM.apply(x).sum() - M.apply(x).sum()) <= 1e-13 * np.abs(x).sum()


@pytest.mark.parametrize("dim,n", [(2, 6), (3, 4)])
def test_lumped_weights_closed_form(dim, n):
    coords, conn = _mesh(dim, n)
    m = L.lumped_weights(dim, coords, conn)
    inner = np.all((coords > 1e-12) & (coords < 1 - 1e-12), axis=1)
    assert np.allclose(m[inner], (1.0 / n) ** dim, rtol=1e-13)
    assert abs(m.sum() - 1.0) < 1e-13


def test_lumped_matrix_structure():
    case = S.make_c2(4)
    A = L.LumpedMatrix(3, case.coords, case.conn, case.dirichlet, case.alpha, case.beta, case.dt2)
    K = oracle.PressureMatrix.from_case(case, part=2).scipy()
    D = (A.A - case.dt2 * K).toarray()
    assert np.allclose(D - np.diag(np.diag(D)), 0.0, atol=1e-15)
    m = L.lumped_weights(3, case.coords, case.conn)
    assert np.allclose(np.diag(D), (case.alpha * m)[A.free_nodes], rtol=1e-13)
    Ad = A.A.toarray()
    assert np.allclose(Ad, Ad.T, atol=1e-15)
    assert np.linalg.eigvalsh(Ad).min() > 0


def _mms_errors(ns, dt2=0.05):
    """alpha p - dt2 div(beta grad p) = f on the unit square, p = 0 on x = 0
    (Dirichlet), natural condition elsewhere; p = sin(pi x / 2) cos(pi y)."""
    def p_exact(x):
        return np.sin(0.5 * np.pi * x[..., 0]) * np.cos(np.pi * x[..., 1])

    def alpha_f(x):
        return 1.0 + 0.5 * x[..., 0] * x[..., 1]

    def f(x):
        lap = -(0.25 * np.pi ** 2 + np.pi ** 2) * p_exact(x)
        return alpha_f(x) * p_exact(x) - dt2 * lap

    errs = []
    for n in ns:
        coords, conn = S.square_mesh(n)
        coords = S.jitter_nodes(coords, n, 0.1, np.random.default_rng(n))
        N, E = coords.shape[0], conn.shape[0]
        dm = (coords[:, 0] == 0).astype(np.uint8)
        A = L.LumpedMatrix(2, coords, conn, dm, alpha_f(coords), np.ones(E), dt2)
        pts, w, bary = element_points(coords, conn, 2, 5)
        load = np.einsum("eq,eq,qa->ea", w, f(pts), bary)
        b = np.zeros(N)
        np.add.at(b, conn.ravel(), load.ravel())
        b[dm == 1] = 0.0
        x = A.solve(b)
        ph = np.einsum("qa,ea->eq", bary, x[conn])
        errs.append(math.sqrt(np.sum(w * (ph - p_exact(pts)) ** 2)))
    return np.array(errs)


def test_lumped_manufactured_solution_second_order():
    e = _mms_errors([8, 16, 32, 64])
    slopes = np.log(e[:-1] / e[1:]) / np.log(2.0)
    assert slopes[-1] >= 1.9, (e, slopes)
    assert slopes.min() >= 1.8, (e, slopes)


def _eos_inputs(case, b):
    e = case.extra
    H = L.enthalpy(case.conn, e["pn"], e["rho"], e["eos_a"], b)
    c = PJ.rhs(case.dim, case.coords, case.conn, case.dirichlet, np.zeros(case.n_nodes), H,
               PJ.kinetic(e["wu"], e["rho"], case.dim), e["wu"], e["we"], e["pn"], e["dt"])
    return H, c


def test_ideal_gas_newton_is_one_linear_solve():
    case = S.make_eos_case(3, 4, eos_b=0.0)
    e = case.extra
    a = e["eos_a"]
    H, c = _eos_inputs(case, 0.0)
    dp, hist, steps = L.newton(3, case.coords, case.conn, case.dirichlet, e["rho"], H, c, e["pn"], None, a, 0.0,
                               e["dt"], max_newton=3, tol=1e-12)
    assert steps == 1 and hist[1] <= 1e-13
    A = L.LumpedMatrix(3, case.coords, case.conn, case.dirichlet, np.full(case.n_nodes, a), H, e["dt"] ** 2)
    m = L.lumped_weights(3, case.coords, case.conn)
    x = A.solve(c - a * m * e["pn"])
    assert np.linalg.norm(dp - x) <= 1e-12 * np.linalg.norm(x)


def test_newton_recovers_manufactured_root_quadratically():
    case = S.make_eos_case(2, 12, eos_b=2.0)
    e = case.extra
    a, b, dt = e["eos_a"], e["eos_b"], e["dt"]
    rng = np.random.default_rng(5)
    H = 1.0 + rng.random(case.n_elems)
    root = 0.3 * rng.standard_normal(case.n_nodes)
    root[case.dirichlet.astype(bool)] = 0.0
    # c = Q(root) + dt^2 K root with Q in closed form P (a m + b s P)
    m, s = L.lumped_weights(2, case.coords, case.conn, e["rho"])
    P = e["pn"] + root
    K = oracle.PressureMatrix(2, case.coords, case.conn, case.dirichlet, case.alpha, H, 1.0, part=2)
    c = P * (a * m + b * s * P) + dt * dt * K.apply(root)
    c[case.dirichlet.astype(bool)] = 0.0
    dp, hist, steps = L.newton(2, case.coords, case.conn, case.dirichlet, e["rho"], H, c, e["pn"], None, a, b, dt,
                               max_newton=12, tol=1e-14)
    assert np.linalg.norm(dp - root) <= 1e-12 * np.linalg.norm(root)
    h = np.array(hist)
    assert h[0] > 1e-3 and steps <= 8
    # quadratic: the order estimate log(e2/e1)/log(e1/e0) of the residuals
    # above the rounding floor is about 2
    ok = h[h > 1e-11]
    assert ok.size >= 4
    orders = np.log(ok[2:] / ok[1:-1]) / np.log(ok[1:-1] / ok[:-2])
    assert orders.max() >= 1.8, h


def test_eos_enthalpy_reduces_to_the_ideal_gas():
    case = S.make_eos_case(3, 3, eos_b=0.0)
    e = case.extra
    gamma = 1.0 + 1.0 / e["eos_a"]
    assert np.allclose(L.enthalpy(case.conn, e["pn"], e["rho"], e["eos_a"], 0.0),
                       PJ.enthalpy(case.conn, e["pn"], e["rho"], gamma), rtol=1e-14)


def test_eos_projection_step_b0_is_the_lumped_picard_loop():
    """b = 0: every Picard iteration is one lumped linear solve with the
    ideal-gas enthalpy (checked against a loop written from LumpedMatrix)."""
    case = S.make_eos_case(2, 10, eos_b=0.0)
    e = case.extra
    a, dt = e["eos_a"], e["dt"]
    out = L.projection_step_eos(2, case.coords, case.conn, case.dirichlet, e["rho"], e["wu"], e["we"], e["pn"],
                                a, 0.0, dt, n_picard=2, max_newton=4, tol=1e-12)
    gamma = 1.0 + 1.0 / a
    m = L.lumped_weights(2, case.coords, case.conn)
    H = PJ.enthalpy(case.conn, e["pn"], e["rho"], gamma)
    rhok = PJ.kinetic(e["wu"], e["rho"], 2)
    for _ in range(2):
        c = PJ.rhs(2, case.coords, case.conn, case.dirichlet, np.zeros(case.n_nodes), H, rhok, e["wu"], e["we"],
                   e["pn"], dt)
        A = L.LumpedMatrix(2, case.coords, case.conn, case.dirichlet, np.full(case.n_nodes, a), H, dt * dt)
        b_lin = c - a * m * e["pn"]
        b_lin[case.dirichlet.astype(bool)] = 0.0
        dp = A.solve(b_lin)
        _, _, H, rhok = PJ.post(2, case.coords, case.conn, e["pn"], dp, e["wu"], e["rho"], gamma, dt)
    assert out["steps"] == [1, 1]
    assert np.linalg.norm(out["dp"] - dp) <= 1e-11 * np.linalg.norm(dp)
    assert np.allclose(out["H"], H, rtol=1e-12)


def test_lumped_operator_on_two_triangles_golden():
    """The lumped operator on the unit square cut into two right triangles
    against the hand-derived rows of tests/golden/lumped_two_triangles.txt."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "lumped_two_triangles.txt")
    rows = [list(map(float, ln.split()[1:])) for ln in open(path) if ln.startswith("row")]
    want = np.array(rows)
    coords, conn = S.square_mesh(1)
    assert np.array_equal(conn, [[0, 1, 3], [0, 3, 2]])
    A = L.LumpedMatrix(2, coords, conn, np.zeros(4, np.uint8), np.array([1.0, 2.0, 3.0, 4.0]), np.ones(2), 0.5)
    assert np.allclose(A.A.toarray(), want, rtol=0, atol=1e-15)
