"""Pins of the periodic-boundary oracle (oracle/periodic.py, Section 3.6 vertex
merging) against what the mathematics fixes:

* the merged matrix is symmetric, the stiffness part has zero row sums (the
  constant is in its kernel on a fully periodic / Neumann domain);
* on a regular mesh with beta = 1 every row away from x = 0 and x = 1 is the
  5-point stencil [4, -1, -1, -1, -1] -- the rows on the periodic seam too;
* merging only identity pairs gives back the unmerged matrix;
* a y-periodic manufactured pressure converges at second order in L2.
"""
import math

import numpy as np

import oracle
from oracle.periodic import PeriodicMatrix
from paper_2301_08357_gb300 import synthetic as S
from tests._quad import element_points


def test_symmetric_and_zero_row_sums():
    case = S.make_periodic_case(3, 4)
    N = case.n_nodes
    K = PeriodicMatrix(3, case.coords, case.conn, np.zeros(N, np.uint8), case.extra["master"], case.alpha,
                       case.beta, case.dt2, part=2)
    A = K.A.toarray()
    assert np.allclose(A, A.T, atol=1e-14)
    assert np.max(np.abs(A.sum(axis=1))) <= 1e-12 * np.abs(A).max()
    assert K.n_dofs == 5 * 4 * 4          # x: 0..4 (5 planes), y and z: 4 distinct planes each


def test_five_point_stencil_across_the_seam():
    n = 6
    coords, conn = S.square_mesh(n)
    master = S.periodic_master(coords, (1,))
    N, E = coords.shape[0], conn.shape[0]
    K = PeriodicMatrix(2, coords, conn, np.zeros(N, np.uint8), master, np.ones(N), np.ones(E), 1.0, part=2)
    Ad = K.A_dofs.toarray()
    dof_x = coords[K.dofs, 0]
    checked = 0
    for r in range(K.n_dofs):
        if dof_x[r] in (0.0, 1.0):
            continue
        row = Ad[r]
        nz = np.sort(row[np.abs(row) > 1e-14])
        assert np.allclose(nz, [-1, -1, -1, -1, 4]), (r, nz)
        checked += 1
    assert checked == (n - 1) * n          # includes the n - 1 rows on the seam y = 0


def test_identity_merge_is_the_plain_matrix():
    case = S.make_c1(6)
    ident = np.arange(case.n_nodes, dtype=np.int32)
    Pm = PeriodicMatrix(2, case.coords, case.conn, case.dirichlet, ident, case.alpha, case.beta, case.dt2)
    A = oracle.PressureMatrix.from_case(case)
    x = np.random.default_rng(1).standard_normal(case.n_nodes)
    assert np.allclose(Pm.apply(x), A.apply(x), rtol=1e-13, atol=1e-15)


def _periodic_mms_errors(ns, dt2=0.1):
    """p = sin(pi x / 2) cos(2 pi y): p = 0 on x = 0, dp/dx = 0 on x = 1,
    periodic in y; alpha and beta periodic in y."""
    def p_exact(x):
        return np.sin(0.5 * np.pi * x[..., 0]) * np.cos(2 * np.pi * x[..., 1])

    def grad_p(x):
        g = np.zeros(x.shape)
        g[..., 0] = 0.5 * np.pi * np.cos(0.5 * np.pi * x[..., 0]) * np.cos(2 * np.pi * x[..., 1])
        g[..., 1] = -2 * np.pi * np.sin(0.5 * np.pi * x[..., 0]) * np.sin(2 * np.pi * x[..., 1])
        return g

    def alpha_f(x):
        return 1.0 + 0.5 * np.sin(2 * np.pi * x[..., 0]) * np.cos(2 * np.pi * x[..., 1])

    def beta_f(x):
        return 1.0 + 0.5 * x[..., 0] ** 2

    def f(x):
        lap = -(0.25 * np.pi ** 2 + 4 * np.pi ** 2) * p_exact(x)
        div = x[..., 0] * grad_p(x)[..., 0] + beta_f(x) * lap
        return alpha_f(x) * p_exact(x) - dt2 * div

    errs = []
    for n in ns:
        coords, conn = S.square_mesh(n)
        coords = S.jitter_nodes(coords, n, 0.1, np.random.default_rng(n))
        master = S.periodic_master(coords, (1,))
        N = coords.shape[0]
        cen = coords[conn].mean(1)
        dm = (coords[:, 0] == 0).astype(np.uint8)
        A = PeriodicMatrix(2, coords, conn, dm, master, alpha_f(coords[master]), beta_f(cen), dt2)
        pts, w, bary = element_points(coords, conn, 2, 5)
        load = np.einsum("eq,eq,qa->ea", w, f(pts), bary)
        b = np.zeros(N)
        np.add.at(b, conn.ravel(), load.ravel())
        b[dm == 1] = 0.0
        x = A.solve(b)
        ph = np.einsum("qa,ea->eq", bary, x[conn])
        errs.append(math.sqrt(np.sum(w * (ph - p_exact(pts)) ** 2)))
    return np.array(errs)


def test_periodic_manufactured_solution_second_order():
    e = _periodic_mms_errors([8, 16, 32, 64])
    slopes = np.log(e[:-1] / e[1:]) / np.log(2.0)
    assert slopes[-1] >= 1.9, (e, slopes)
    assert slopes.min() >= 1.8, (e, slopes)
