"""Pins of the projection-stage oracle (oracle/projection.py) against what the
mathematics fixes, independently of the oracle's own formulas:

* int phi_i on regular meshes (closed form h^d) and the partition of unity;
* the mass term against the C oracle's assembled M_alpha (an independent
  implementation: element matrices by Gauss-Jordan inverse and monomial
  integrals);
* the discrete divergence theorem: for the P0 projection of a linear field u,
  int u.grad phi_i = -int div(u) phi_i exactly at interior nodes, and the
  gradient terms sum to zero over all nodes for any element-constant u;
* post-projection: the gradient of a linear pressure correction is exact;
* one Picard iteration equals a dense direct solve of the same system.
"""
import numpy as np
import pytest

import oracle
from oracle import projection as PJ
from paper_2301_08357_gb300 import synthetic as S


def _mesh(dim, n, jitter=0.0, seed=0):
    if dim == 2:
        coords, conn = S.square_mesh(n)
    else:
        coords, conn = S.kuhn_cube_mesh(n)
    if jitter:
        coords = S.jitter_nodes(coords, n, jitter, np.random.default_rng(seed))
    return coords, conn


def _interior(coords, tol=1e-12):
    return np.all((coords > tol) & (coords < 1 - tol), axis=1)


@pytest.mark.parametrize("dim,n", [(2, 6), (3, 4)])
def test_source_term_closed_form(dim, n):
    coords, conn = _mesh(dim, n)
    N, E = coords.shape[0], conn.shape[0]
    c = 1.7
    z = np.zeros(N)
    b = PJ.rhs(dim, coords, conn, np.zeros(N, np.uint8), np.ones(N), np.ones(E), np.zeros(E),
               np.zeros((E, dim)), np.full(E, c), z, dt=0.3)
    h = 1.0 / n
    inner = _interior(coords)
    # int phi_i = h^d at interior nodes of the regular meshes (6 triangles of
    # h^2/2 with 1/3 each; 24 Kuhn tets of h^3/6 with 1/4 each)
    assert np.allclose(b[inner], c * h ** dim, rtol=1e-13)
    assert abs(b.sum() - c) < 1e-12                     # partition of unity, |Omega| = 1


@pytest.mark.parametrize("dim,n", [(2, 5), (3, 3)])
def test_mass_term_matches_assembled_matrix(dim, n):
    coords, conn = _mesh(dim, n, jitter=0.2, seed=3)
    rng = np.random.default_rng(4)
    N, E = coords.shape[0], conn.shape[0]
    alpha = 0.5 + rng.random(N)
    p = rng.standard_normal(N)
    y = PJ.mass_alpha_full(dim, coords, conn, alpha, p)
    # without Dirichlet nodes the assembled mass-only matrix covers every column
    M = oracle.PressureMatrix(dim, coords, conn, np.zeros(N, np.uint8), alpha, np.ones(E), 1.0, part=1)
    assert np.allclose(y, M.apply(p), rtol=1e-12, atol=1e-14)
    # and the right-hand side carries it with a minus sign
    b = PJ.rhs(dim, coords, conn, np.zeros(N, np.uint8), alpha, np.ones(E), np.zeros(E),
               np.zeros((E, dim)), np.zeros(E), p, dt=0.1)
    assert np.allclose(b, -y, rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("dim,n", [(2, 6), (3, 4)])
def test_divergence_term_is_exact_for_linear_fields(dim, n):
    coords, conn = _mesh(dim, n, jitter=0.2, seed=5)
    N, E = coords.shape[0], conn.shape[0]
    rng = np.random.default_rng(6)
    A = rng.standard_normal((dim, dim))
    c0 = rng.standard_normal(dim)
    # P0 projection of the linear field u(x) = A x + c0: its value at the centroid
    cen = coords[conn].mean(axis=1)
    wu = cen @ A.T + c0
    dt = 0.37
    vol, _ = PJ.element_geometry(dim, coords, conn)
    b = PJ.rhs(dim, coords, conn, np.zeros(N, np.uint8), np.ones(N), np.ones(E), np.zeros(E), wu,
               np.zeros(E), np.zeros(N), dt)
    int_phi = np.zeros(N)
    np.add.at(int_phi, conn, np.repeat(vol[:, None] / (dim + 1), dim + 1, axis=1))
    inner = _interior(coords)
    # dt int u.grad phi_i = -dt div(u) int phi_i, div u = trace(A)
    assert np.allclose(b[inner], -dt * np.trace(A) * int_phi[inner], rtol=1e-11, atol=1e-14)
    # for an element-constant u the gradient terms sum to zero (sum_i grad phi_i = 0)
    b2 = PJ.rhs(dim, coords, conn, np.zeros(N, np.uint8), np.ones(N), rng.random(E) + 0.5, np.zeros(E),
                rng.standard_normal((E, dim)), np.zeros(E), np.zeros(N), dt)
    assert abs(b2.sum()) < 1e-12 * np.abs(b2).sum()


def test_dirichlet_rows_are_zero():
    case = S.make_c1(8)
    E = case.n_elems
    b = PJ.rhs(2, case.coords, case.conn, case.dirichlet, case.alpha, case.beta, np.zeros(E),
               np.ones((E, 2)), np.ones(E), np.ones(case.n_nodes), 0.1)
    assert np.all(b[case.dirichlet.astype(bool)] == 0.0)
    assert np.all(b[~case.dirichlet.astype(bool)] != 0.0)


@pytest.mark.parametrize("dim,n", [(2, 5), (3, 3)])
def test_post_projection_gradient_is_exact(dim, n):
    coords, conn = _mesh(dim, n, jitter=0.2, seed=8)
    N, E = coords.shape[0], conn.shape[0]
    rng = np.random.default_rng(9)
    g = rng.standard_normal(dim)
    dp = 0.3 + coords @ g
    p_n = np.full(N, 2.0)
    rho = 0.5 + rng.random(E)
    wu_tt = rng.standard_normal((E, dim))
    gamma, dt = 1.4, 0.05
    p, wu, H, rhok = PJ.post(dim, coords, conn, p_n, dp, wu_tt, rho, gamma, dt)
    assert np.allclose(p, p_n + dp, rtol=0, atol=0)
    assert np.allclose(wu, wu_tt - dt * g, rtol=1e-12, atol=1e-13)
    pbar = (p_n + dp)[conn].mean(axis=1)
    assert np.allclose(H, 3.5 * pbar / rho, rtol=1e-14)
    assert np.allclose(rhok, 0.5 * (wu ** 2).sum(axis=1) / rho, rtol=1e-14)


def test_one_picard_iteration_is_a_direct_solve():
    case = S.make_c2(4)
    dim, N, E = 3, case.n_nodes, case.n_elems
    rng = np.random.default_rng(11)
    rho = 1.0 + 0.2 * rng.random(E)
    wu_tt = 0.3 * rng.standard_normal((E, dim))
    p_n = 1.0 + 0.1 * rng.standard_normal(N)
    we = 2.5 * p_n[case.conn].mean(axis=1) + 0.1 * rng.standard_normal(E)
    alpha = np.full(N, 2.5)
    gamma, dt = 1.4, 0.05
    out = PJ.projection_step(dim, case.coords, case.conn, case.dirichlet, alpha, rho, wu_tt, we, p_n,
                             gamma, dt, n_picard=1)
    H1 = PJ.enthalpy(case.conn, p_n, rho, gamma)
    b = PJ.rhs(dim, case.coords, case.conn, case.dirichlet, alpha, H1, PJ.kinetic(wu_tt, rho, dim), wu_tt,
               we, p_n, dt)
    A = oracle.PressureMatrix(dim, case.coords, case.conn, case.dirichlet, alpha, H1, dt * dt)
    x = A.cholesky_solve(b)
    assert np.linalg.norm(out["dp"] - x) <= 1e-11 * np.linalg.norm(x)
    # a second iteration uses the updated enthalpy and kinetic energy
    out2 = PJ.projection_step(dim, case.coords, case.conn, case.dirichlet, alpha, rho, wu_tt, we, p_n,
                              gamma, dt, n_picard=2)
    assert np.allclose(out2["solves"][1]["H"], out["H"], rtol=1e-12)
    assert not np.allclose(out2["dp"], out["dp"], rtol=1e-6)


def test_element_values_golden():
    """Kinetic energy density and enthalpy of single elements against values
    derived by hand (tests/golden/projection_element_values.txt): a dropped
    1/2, a sum instead of a mean, or gamma/(gamma-1) inverted fails them."""
    from conftest import golden
    from oracle import lumped as LO
    seen = set()
    for row in golden("projection_element_values.txt"):
        kind, vals = row[0], [float(v) for v in row[1:]]
        expected = vals[-1]
        if kind == "kinetic":
            dim, rho, wu = int(vals[0]), vals[1], np.array(vals[2:-1])
            assert wu.size == dim
            got = PJ.kinetic(wu.reshape(1, dim), np.array([rho]), dim)[0]
        elif kind == "enthalpy":
            gamma, rho, p = vals[0], vals[1], np.array(vals[2:-1])
            got = PJ.enthalpy(np.arange(p.size).reshape(1, -1), p, np.array([rho]), gamma)[0]
        else:
            assert kind == "enthalpy_eos"
            a, b, rho, p = vals[0], vals[1], vals[2], np.array(vals[3:-1])
            got = LO.enthalpy(np.arange(p.size).reshape(1, -1), p, np.array([rho]), a, b)[0]
        assert abs(got - expected) <= 1e-14 * abs(expected), (row, got)
        seen.add(kind)
    assert seen == {"kinetic", "enthalpy", "enthalpy_eos"}
