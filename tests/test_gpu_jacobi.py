"""Parity of the Jacobi preconditioner's diagonal with the oracle's matrix.

The preconditioner applies D^-1 with D_ii = sum_e (M^e_ii + dt^2 K^e_ii), the
diagonal of the weak problem's matrix (Section 3.4).  A solve converges to the
same answer whatever D^-1 is, so the solve tests cannot see a wrong diagonal;
this test reads the device copies through ps_mesh_get_jacobi (caller
numbering) and compares them entry by entry with the diagonal of the
oracle's assembled matrix:

  FP64 copy:  |dinv64 * A_ii - 1| <= 1e-13   (FP64 element sums and one division)
  FP32 copy:  |dinv32 * A_ii - 1| <= 1.2e-7  (the FP64 value rounded to float)
  Dirichlet nodes: exactly 0 in both copies.

A diagonal without its mass term, without dt^2 or with a wrong mass weight
misses the first bar by orders of magnitude on every case below.
"""
import numpy as np
import pytest

import oracle
from oracle import lumped as L
from oracle.periodic import PeriodicMatrix
from paper_2301_08357_gb300 import synthetic as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_2301_08357_gb300 import build
    build.build()
    from paper_2301_08357_gb300 import pressure as P
    assert torch.cuda.is_available()
    ctx = P.ps_ctx_create(0)
    yield P, torch, ctx
    P.ps_ctx_destroy(ctx)


def _check(P, m, diag_user, dirichlet_user):
    d64 = P.ps_mesh_get_jacobi(m, P.PS_F64)
    d32 = P.ps_mesh_get_jacobi(m, P.PS_F32).astype(np.float64)
    dirm = np.asarray(dirichlet_user, dtype=bool)
    assert np.all(d64[dirm] == 0.0) and np.all(d32[dirm] == 0.0)
    free = ~dirm
    assert np.all(diag_user[free] > 0.0)
    e64 = np.max(np.abs(d64[free] * diag_user[free] - 1.0))
    e32 = np.max(np.abs(d32[free] * diag_user[free] - 1.0))
    assert e64 <= 1e-13, e64
    assert e32 <= 1.2e-7, e32
    return e64, e32


def _csr_diag(A):
    """Diagonal of the oracle's reduced CSR matrix, in the caller's numbering."""
    return A.extend(A.scipy().diagonal())


CASES = [
    ("c1_24", lambda: S.make_c1(24), 0),
    ("c1_24_shuffled_chunk37", lambda: S.shuffle_case(S.make_c1(24)), 37),
    ("c2_8", lambda: S.make_c2(8), 0),
    ("c2_9_small_chunks", lambda: S.make_c2(9), 60),
    ("c2_8_shuffled", lambda: S.shuffle_case(S.make_c2(8), seed=3), 0),
    ("c3_n12_stiff", lambda: S.make_c3(12), 0),
    ("batch_mesh_3", lambda: S.make_batch_case(3, lo=2e3, hi=5e3), 0),
]


@pytest.mark.parametrize("name,make,chunk", CASES, ids=[c[0] for c in CASES])
def test_jacobi_diagonal_matches_oracle(env, name, make, chunk):
    P, torch, ctx = env
    case = make()
    m = P.ps_mesh_upload(ctx, case.dim, case.coords, case.conn, case.dirichlet, chunk_elems=chunk)
    try:
        P.ps_coeff_set(m, case.alpha, case.beta, case.dt2)
        A = oracle.PressureMatrix.from_case(case)
        _check(P, m, _csr_diag(A), case.dirichlet)
        # a new beta (ps_coeff_set_beta) rebuilds the diagonal
        beta2 = case.beta * np.exp(0.3 * np.random.default_rng(5).standard_normal(case.n_elems))
        P.ps_coeff_set_beta(m, beta2)
        _check(P, m, _csr_diag(oracle.PressureMatrix.from_case(case, beta=beta2)), case.dirichlet)
    finally:
        P.ps_mesh_free(m)


@pytest.mark.parametrize("name,make,chunk", CASES[:5], ids=[c[0] for c in CASES[:5]])
def test_jacobi_diagonal_lumped(env, name, make, chunk):
    """Mass-lumped form: D_ii = alpha_i m_i + dt^2 K_ii; switching back to the
    consistent form restores the consistent diagonal."""
    P, torch, ctx = env
    case = make()
    m = P.ps_mesh_upload(ctx, case.dim, case.coords, case.conn, case.dirichlet, chunk_elems=chunk)
    try:
        P.ps_coeff_set(m, case.alpha, case.beta, case.dt2)
        P.ps_mesh_set_mass(m, P.PS_MASS_LUMPED)
        AL = L.LumpedMatrix(case.dim, case.coords, case.conn, case.dirichlet, case.alpha, case.beta, case.dt2)
        _check(P, m, AL.extend(AL.A.diagonal()), case.dirichlet)
        P.ps_mesh_set_mass(m, P.PS_MASS_CONSISTENT)
        _check(P, m, _csr_diag(oracle.PressureMatrix.from_case(case)), case.dirichlet)
    finally:
        P.ps_mesh_free(m)


@pytest.mark.parametrize("dim,n,chunk", [(2, 24, 0), (3, 8, 0), (3, 9, 60)])
def test_jacobi_diagonal_periodic(env, dim, n, chunk):
    """Merged periodic vertices: D of an unknown sums the elements around all
    of its vertices (the diagonal of P^T A P); every vertex reports its
    unknown's value."""
    P, torch, ctx = env
    case = S.make_periodic_case(dim, n)
    master = case.extra["master"]
    A = PeriodicMatrix(dim, case.coords, case.conn, case.dirichlet, master, case.alpha, case.beta, case.dt2)
    m = P.ps_mesh_upload(ctx, dim, case.coords, case.conn, case.dirichlet, chunk_elems=chunk, periodic=master)
    try:
        P.ps_coeff_set(m, case.alpha, case.beta, case.dt2)
        diag = A.to_user(A.A.diagonal())
        _check(P, m, diag, case.dirichlet)
        d64 = P.ps_mesh_get_jacobi(m, P.PS_F64)
        assert np.array_equal(d64, d64[master])
    finally:
        P.ps_mesh_free(m)


def test_jacobi_rejects_bad_calls(env):
    P, torch, ctx = env
    case = S.make_c2(3)
    m = P.ps_mesh_upload(ctx, case.dim, case.coords, case.conn, case.dirichlet)
    try:
        with pytest.raises(P.PressureError) as e:
            P.ps_mesh_get_jacobi(m, P.PS_F64)       # coefficients not set
        assert e.value.status == P.PS_ESTATE
        P.ps_coeff_set(m, case.alpha, case.beta, case.dt2)
        with pytest.raises(P.PressureError) as e:
            P.ps_mesh_get_jacobi(m, 3)
        assert e.value.status == P.PS_EINVAL
    finally:
        P.ps_mesh_free(m)
