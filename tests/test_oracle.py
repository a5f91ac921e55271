"""Pins of the FP64 CPU oracle against what the paper and mathematics fix.

Each test checks the oracle against something other than itself: closed-form
stencils, the textbook consistent mass matrix, brute-force quadrature with an
independent basis construction, exact invariants (symmetry, zero row sums of
the stiffness part, the patch test), positive definiteness (Section 3.4 states
the system is SPD), direct solves by a library routine, the CG error bound, and
second-order L2 convergence on a manufactured pressure field (the paper's P1
pressure reaches order 2, Section 5.1, Table TGV_errors).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2301_08357_gb300 import synthetic as S
from tests._quad import element_points
from tests.conftest import golden


def _random_simplex(rng, dim):
    while True:
        v = rng.uniform(-1.0, 1.0, size=(dim + 1, dim))
        if abs(np.linalg.det(v[1:] - v[0])) > 0.1:
            return v


def _independent_grads(v):
    """Gradients of the P1 basis from phi_i(x) = a_i + b_i.x, found by
    inverting the vertex matrix [1 v_k^T] (no Jacobian map)."""
    nv = v.shape[0]
    P = np.concatenate([np.ones((nv, 1)), v], axis=1)
    Cm = np.linalg.inv(P)
    vol = abs(np.linalg.det(P)) / math.factorial(nv - 1)
    return Cm[1:, :].T, vol                      # [nv, d], |T|


def _mesh(dim, n, jitter=0.0, seed=0):
    rng = np.random.default_rng(seed)
    if dim == 2:
        coords, conn = S.square_mesh(n)
    else:
        coords, conn = S.kuhn_cube_mesh(n)
    if jitter:
        coords = S.jitter_nodes(coords, n, jitter, rng)
    return coords, conn


# ---------------------------------------------------------------- mesh sizes
def test_generator_matches_tgv_mesh_table():
    for name, n, ne, nv in golden("tgv_mesh_sizes.txt"):
        coords, conn = S.square_mesh(int(n))
        assert conn.shape[0] == int(ne), name
        assert coords.shape[0] == int(nv), name


def test_generated_meshes_positive_and_jitter_bounded():
    for dim, n, j in ((2, 64, 0.2), (3, 12, 0.15)):
        rng = np.random.default_rng(0)
        coords0, conn = (S.square_mesh if dim == 2 else S.kuhn_cube_mesh)(n)
        coords = S.jitter_nodes(coords0, n, j, rng)
        V = coords[conn]
        det = np.linalg.det(V[:, 1:] - V[:, :1])
        nominal = (1.0 / n) ** dim
        assert det.min() > 0.2 * nominal
        assert np.abs(coords - coords0).max() <= j / n + 1e-15
        # boundary untouched: x = 0 plane is exact
        on0 = coords0[:, 0] == 0.0
        assert np.all(coords[on0, 0] == 0.0)


# ----------------------------------------------------------- element matrices
@pytest.mark.parametrize("dim", [2, 3])
def test_element_mass_alpha_one_is_textbook(dim):
    rng = np.random.default_rng(1)
    for _ in range(20):
        v = _random_simplex(rng, dim)
        _, Me, _, vol, _ = oracle.element_matrices(dim, v, np.ones(dim + 1), 1.0, 0.0)
        ref = vol * (1.0 + np.eye(dim + 1)) / ((dim + 1) * (dim + 2))
        np.testing.assert_allclose(Me, ref, rtol=1e-13, atol=1e-16)


@pytest.mark.parametrize("dim", [2, 3])
def test_element_matrices_match_quadrature(dim):
    """M^e_ij = int alpha_h phi_i phi_j and K^e_ij = beta |T| grad phi_i . grad phi_j
    against Gauss quadrature on the forward map with independently built
    gradients."""
    rng = np.random.default_rng(2)
    for _ in range(20):
        v = _random_simplex(rng, dim)
        a = rng.uniform(0.1, 3.0, size=dim + 1)
        beta = rng.uniform(0.1, 5.0)
        dt2 = rng.uniform(0.01, 2.0)
        Ae, Me, Ke, vol, _ = oracle.element_matrices(dim, v, a, beta, dt2)
        pts, w, bary = element_points(v, np.arange(dim + 1)[None], dim, 4)
        w = w[0]
        alpha_q = bary @ a
        Mq = np.einsum("q,qi,qj,q->ij", w, bary, bary, alpha_q)
        G, vol_ind = _independent_grads(v)
        Kq = beta * vol_ind * G @ G.T
        np.testing.assert_allclose(vol, vol_ind, rtol=1e-13)
        np.testing.assert_allclose(Me, Mq, rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(Ke, Kq, rtol=1e-11, atol=1e-13)
        np.testing.assert_allclose(Ae, Mq + dt2 * Kq, rtol=1e-11, atol=1e-13)
        # vertex order does not matter (a permuted element gives the permuted matrix)
        perm = rng.permutation(dim + 1)
        Ae2, _, _, _, _ = oracle.element_matrices(dim, v[perm], a[perm], beta, dt2)
        np.testing.assert_allclose(Ae2, Ae[np.ix_(perm, perm)], rtol=1e-12, atol=1e-14)


# ------------------------------------------------------- closed-form stencils
def _closed():
    return {r[0]: float(r[1]) for r in golden("p1_closed_forms.txt")}


def _row(A, node):
    r = A.free_of_node[node]
    cols = A.col[A.rowptr[r]:A.rowptr[r + 1]]
    vals = A.val[A.rowptr[r]:A.rowptr[r + 1]]
    return {int(A.node_of_free[c]): v for c, v in zip(cols, vals)}


def test_stiffness_2d_is_five_point_stencil():
    cf = _closed()
    n = 8
    coords, conn = _mesh(2, n)
    N = coords.shape[0]
    K = oracle.PressureMatrix(2, coords, conn, np.zeros(N, np.uint8), np.ones(N),
                              np.ones(conn.shape[0]), 1.0, part=2)
    i, j = 3, 4
    c = i + (n + 1) * j
    row = _row(K, c)
    assert row[c] == pytest.approx(cf["k2d_center"], abs=1e-13)
    for nb in (c + 1, c - 1, c + n + 1, c - n - 1):
        assert row[nb] == pytest.approx(cf["k2d_axis_neighbour"], abs=1e-13)
    for nb in (c + n + 2, c - n - 2):
        assert row[nb] == pytest.approx(cf["k2d_diag_neighbour"], abs=1e-13)
    assert len(row) == 7


def test_stiffness_3d_kuhn_is_scaled_seven_point_stencil():
    cf = _closed()
    n = 5
    h = 1.0 / n
    coords, conn = _mesh(3, n)
    N = coords.shape[0]
    K = oracle.PressureMatrix(3, coords, conn, np.zeros(N, np.uint8), np.ones(N),
                              np.ones(conn.shape[0]), 1.0, part=2)
    m = n + 1
    c = 2 + m * (2 + m * 2)
    row = _row(K, c)
    assert len(row) == 15
    assert row[c] == pytest.approx(cf["k3d_center"] * h, abs=1e-13)
    axis = {c + 1, c - 1, c + m, c - m, c + m * m, c - m * m}
    for nb, v in row.items():
        if nb == c:
            continue
        want = cf["k3d_axis_neighbour"] if nb in axis else cf["k3d_diag_neighbour"]
        assert v == pytest.approx(want * h, abs=1e-13)


def test_consistent_mass_rows_closed_form():
    cf = _closed()
    n = 8
    h = 1.0 / n
    coords, conn = _mesh(2, n)
    N = coords.shape[0]
    M = oracle.PressureMatrix(2, coords, conn, np.zeros(N, np.uint8), np.ones(N),
                              np.ones(conn.shape[0]), 0.0, part=1)
    c = 3 + (n + 1) * 4
    row = _row(M, c)
    assert row[c] == pytest.approx(cf["m2d_center"] * h * h, rel=1e-13)
    for nb, v in row.items():
        if nb != c:
            assert v == pytest.approx(cf["m2d_neighbour"] * h * h, rel=1e-13)
    assert sum(row.values()) == pytest.approx(cf["m2d_row_sum"] * h * h, rel=1e-13)
    n = 4
    h = 1.0 / n
    coords, conn = _mesh(3, n)
    N = coords.shape[0]
    M = oracle.PressureMatrix(3, coords, conn, np.zeros(N, np.uint8), np.ones(N),
                              np.ones(conn.shape[0]), 0.0, part=1)
    m = n + 1
    c = 2 + m * (2 + m * 2)
    row = _row(M, c)
    assert row[c] == pytest.approx(cf["m3d_center"] * h ** 3, rel=1e-13)
    assert sum(row.values()) == pytest.approx(cf["m3d_row_sum"] * h ** 3, rel=1e-13)


# -------------------------------------------------------------- invariants
@pytest.mark.parametrize("dim,n", [(2, 12), (3, 5)])
def test_invariants_symmetry_rowsums_patch(dim, n):
    rng = np.random.default_rng(3)
    coords, conn = _mesh(dim, n, jitter=0.2 if dim == 2 else 0.15, seed=4)
    N, E = coords.shape[0], conn.shape[0]
    alpha = rng.uniform(0.5, 2.0, N)
    beta = np.exp(0.5 * rng.standard_normal(E))
    nod = np.zeros(N, np.uint8)
    K = oracle.PressureMatrix(dim, coords, conn, nod, alpha, beta, 1.0, part=2)
    M = oracle.PressureMatrix(dim, coords, conn, nod, alpha, beta, 1.0, part=1)
    A = oracle.PressureMatrix(dim, coords, conn, nod, alpha, beta, 0.37, part=0)
    Kd, Md, Ad = K.dense(), M.dense(), A.dense()
    for X in (Kd, Md, Ad):
        np.testing.assert_allclose(X, X.T, rtol=0, atol=1e-14 * np.abs(X).max())
    # A = M + dt^2 K entry by entry
    np.testing.assert_allclose(Ad, Md + 0.37 * Kd, rtol=1e-13, atol=1e-16)
    # zero row sums of the stiffness part (constants are in its kernel)
    assert np.abs(Kd.sum(1)).max() < 1e-13 * np.abs(Kd).max()
    # patch test: with constant beta a linear field has zero stiffness action
    # at interior nodes (the integral of grad phi_i over its support vanishes)
    cvec = rng.standard_normal(dim)
    u = coords @ cvec
    K1 = oracle.PressureMatrix(dim, coords, conn, nod, alpha, np.full(E, 1.7), 1.0, part=2).dense()
    interior = np.all((coords > 1e-9) & (coords < 1 - 1e-9), axis=1)
    assert np.abs((K1 @ u)[interior]).max() < 1e-12 * np.abs(K1).max()
    Ku = Kd @ u
    # energy of a linear field: sum_e beta_e |T_e| |c|^2
    V = coords[conn]
    vol = np.abs(np.linalg.det(V[:, 1:] - V[:, :1])) / math.factorial(dim)
    assert u @ Ku == pytest.approx(float(np.sum(beta * vol)) * float(cvec @ cvec), rel=1e-11)
    # total mass: 1^T M 1 = sum_e |T_e| mean(alpha over the vertices)
    assert Md.sum() == pytest.approx(float(np.sum(vol * alpha[conn].mean(1))), rel=1e-12)
    # alpha == 1 on the unit square / cube: total mass is the domain measure 1
    M1 = oracle.PressureMatrix(dim, coords, conn, nod, np.ones(N), beta, 1.0, part=1)
    assert M1.dense().sum() == pytest.approx(1.0, rel=1e-12)


def test_dirichlet_elimination_is_the_restriction():
    coords, conn = _mesh(2, 6, jitter=0.2, seed=5)
    N, E = coords.shape[0], conn.shape[0]
    rng = np.random.default_rng(5)
    alpha, beta = rng.uniform(0.5, 2, N), rng.uniform(0.5, 2, E)
    full = oracle.PressureMatrix(2, coords, conn, np.zeros(N, np.uint8), alpha, beta, 0.3)
    dmask = (coords[:, 0] == 0).astype(np.uint8)
    red = oracle.PressureMatrix(2, coords, conn, dmask, alpha, beta, 0.3)
    free = np.flatnonzero(dmask == 0)
    np.testing.assert_allclose(red.dense(), full.dense()[np.ix_(free, free)], rtol=1e-14)
    x = rng.standard_normal(N)
    y = red.apply(x)
    assert np.all(y[dmask == 1] == 0.0)
    np.testing.assert_allclose(y[free], full.dense()[np.ix_(free, free)] @ x[free], rtol=1e-12)


def test_poisson_limit_is_scaled_stiffness():
    """alpha -> 0 leaves dt^2 K (the pressure Poisson limit of Section 3)."""
    coords, conn = _mesh(3, 3, jitter=0.15, seed=6)
    N, E = coords.shape[0], conn.shape[0]
    beta = np.ones(E)
    dm = (coords[:, 0] == 0).astype(np.uint8)
    A = oracle.PressureMatrix(3, coords, conn, dm, np.zeros(N), beta, 0.5)
    K = oracle.PressureMatrix(3, coords, conn, dm, np.ones(N), beta, 1.0, part=2)
    np.testing.assert_allclose(A.dense(), 0.5 * K.dense(), rtol=1e-14, atol=1e-18)


# -------------------------------------------------------------- SPD + solves
@pytest.mark.parametrize("dim,n", [(2, 2), (2, 5), (2, 8), (3, 2), (3, 3), (3, 4)])
def test_spd_cholesky_and_cg_agree_with_library_solve(dim, n):
    case = (S.make_c1 if dim == 2 else S.make_c2)(n=n, seed=n)
    A = oracle.PressureMatrix.from_case(case)
    D = A.dense()
    ev = np.linalg.eigvalsh(D)
    assert ev[0] > 0.0
    xd = np.linalg.solve(D, A.restrict(case.b))
    xc = A.restrict(A.cholesky_solve(case.b))
    np.testing.assert_allclose(xc, xd, rtol=1e-11, atol=1e-12 * np.abs(xd).max())
    for pre in (0, 1):
        xg, st, it, rr = A.cg(case.b, precond=pre, tol=1e-13)
        assert st == 0 and rr <= 1e-13
        np.testing.assert_allclose(A.restrict(xg), xd, rtol=0, atol=1e-10 * np.abs(xd).max())


def test_cholesky_rejects_indefinite():
    """A negative dt^2 makes the stiffness part negative: no longer SPD."""
    case = S.make_c1(n=4)
    A = oracle.PressureMatrix(2, case.coords, case.conn, case.dirichlet, case.alpha,
                              case.beta, -10.0)
    with pytest.raises(np.linalg.LinAlgError):
        A.cholesky_solve(case.b)


def test_cg_error_bound():
    """A-norm error after k plain-CG steps is below 2 ((sqrt k - 1)/(sqrt k + 1))^k."""
    case = S.make_c1(n=10, seed=3)
    A = oracle.PressureMatrix.from_case(case)
    D = A.dense()
    ev = np.linalg.eigvalsh(D)
    kap = ev[-1] / ev[0]
    xs = np.linalg.solve(D, A.restrict(case.b))
    e0 = math.sqrt(xs @ D @ xs)
    rho = (math.sqrt(kap) - 1) / (math.sqrt(kap) + 1)
    for k in (5, 10, 20, 40):
        xk, _, it, _ = A.cg(case.b, precond=0, tol=1e-30, max_it=k, max_restarts=0)
        assert it == k
        e = A.restrict(xk) - xs
        assert math.sqrt(e @ D @ e) <= 2 * rho ** k * e0 * (1 + 1e-9)


def test_cg_warm_start_converges_from_guess():
    case = S.make_c3(n=6)
    A = oracle.PressureMatrix.from_case(case)
    xs = case.extra["xstar"]
    b = A.apply(xs)
    x, st, it, rr = A.cg(b, x0_full=case.x0, precond=1, tol=1e-13)
    assert st == 0
    assert np.linalg.norm(x - xs) <= 1e-9 * np.linalg.norm(xs)
    _, _, it_cold, _ = A.cg(b, precond=1, tol=1e-13)
    assert it <= it_cold


# ------------------------------------------------ manufactured solution O(h^2)
def _mms_errors(dim, ns, dt2=0.1):
    def p_exact(x):
        v = np.sin(0.5 * np.pi * x[..., 0]) * np.cos(np.pi * x[..., 1])
        return v * np.cos(np.pi * x[..., 2]) if dim == 3 else v

    def alpha_f(x):
        return 1.0 + 0.5 * np.sin(2 * np.pi * x[..., 0]) * np.cos(2 * np.pi * x[..., 1])

    def beta_f(x):
        return 1.0 + 0.5 * x[..., 0] * x[..., 1]

    def grad_beta(x):
        g = np.zeros(x.shape)
        g[..., 0] = 0.5 * x[..., 1]
        g[..., 1] = 0.5 * x[..., 0]
        return g

    def grad_p(x):
        sx, cx = np.sin(0.5 * np.pi * x[..., 0]), np.cos(0.5 * np.pi * x[..., 0])
        sy, cy = np.sin(np.pi * x[..., 1]), np.cos(np.pi * x[..., 1])
        g = np.zeros(x.shape)
        if dim == 2:
            g[..., 0] = 0.5 * np.pi * cx * cy
            g[..., 1] = -np.pi * sx * sy
        else:
            cz, sz = np.cos(np.pi * x[..., 2]), np.sin(np.pi * x[..., 2])
            g[..., 0] = 0.5 * np.pi * cx * cy * cz
            g[..., 1] = -np.pi * sx * sy * cz
            g[..., 2] = -np.pi * sx * cy * sz
        return g

    lap_fac = -(0.25 * np.pi ** 2 + np.pi ** 2 + (np.pi ** 2 if dim == 3 else 0.0))

    def f(x):
        p = p_exact(x)
        div = np.sum(grad_beta(x) * grad_p(x), axis=-1) + beta_f(x) * lap_fac * p
        return alpha_f(x) * p - dt2 * div

    errs = []
    for n in ns:
        coords, conn = _mesh(dim, n, jitter=0.1, seed=n)
        N = coords.shape[0]
        cen = coords[conn].mean(1)
        dm = (coords[:, 0] == 0).astype(np.uint8)
        A = oracle.PressureMatrix(dim, coords, conn, dm, alpha_f(coords), beta_f(cen), dt2)
        pts, w, bary = element_points(coords, conn, dim, 5)
        fq = f(pts)                                         # [E, Q]
        load = np.einsum("eq,eq,qa->ea", w, fq, bary)       # int f phi_a
        b = np.zeros(N)
        np.add.at(b, conn.ravel(), load.ravel())
        b[dm == 1] = 0.0
        x, st, it, rr = A.cg(b, precond=1, tol=1e-12)
        assert st == 0
        ph = np.einsum("qa,ea->eq", bary, x[conn])
        err = math.sqrt(np.sum(w * (ph - p_exact(pts)) ** 2))
        errs.append(err)
    return np.array(errs)


def test_manufactured_solution_second_order_2d():
    ns = [8, 16, 32, 64]
    e = _mms_errors(2, ns)
    slopes = np.log(e[:-1] / e[1:]) / np.log(2.0)
    assert slopes[-1] >= 1.9, (e, slopes)
    assert slopes.min() >= 1.8, (e, slopes)


def test_manufactured_solution_second_order_3d():
    ns = [4, 8, 16]
    e = _mms_errors(3, ns)
    slopes = np.log(e[:-1] / e[1:]) / np.log(2.0)
    assert slopes[-1] >= 1.9, (e, slopes)
