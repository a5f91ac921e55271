"""Parity of the solver's FP32 CG operator kernel with the oracle, in isolation.

The mixed-precision solve spends its time in the FP32 operator kernel of the
two-kernel CG iteration (q = A p and the chunk shares of p.Ap).  A solve test
cannot pin that kernel exactly: the outer FP64 defect correction reaches the
oracle's answer even when the inner operator is somewhat off.  Here
ps_debug_cg_apply runs one pass of the kernel with direction p = x and the
result is compared element by element with the oracle's assembled matrix:

  |y_gpu - (A x)_i| <= 2e-5 s_i,   s_i = sum_j |A_ij x_j|   (FP32 element arithmetic)
  |x^T A x (kernel) - x^T A x (oracle)| <= 2e-5 sum_i |x_i| s_i

for both kernel variants (one patch per thread; paired patches with packed
FP32x2 arithmetic), the consistent and the lumped mass, shuffled numberings,
small and large chunks and a periodic mesh.  Dirichlet rows are exactly 0.
"""
import numpy as np
import pytest

import oracle
from oracle import lumped as L
from oracle.periodic import PeriodicMatrix
from paper_2301_08357_gb300 import synthetic as S
from tests.gpu_util import row_scale_fast

pytestmark = pytest.mark.gpu

TOL = 2e-5


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


def _run(P, torch, m, x):
    xd = torch.as_tensor(x, dtype=torch.float32, device="cuda")
    yd = torch.full_like(xd, float("nan"))
    pap = P.ps_debug_cg_apply(m, xd, yd)
    return yd.cpu().double().numpy(), pap, xd.cpu().double().numpy()


def _check(y, pap, xs, ref, scale, dirm):
    assert np.all(y[dirm] == 0.0)
    free = ~dirm
    err = np.max(np.abs(y - ref)[free] / np.maximum(scale[free], 1e-300))
    assert err <= TOL, err
    want = float(xs[free] @ ref[free])
    bound = float(np.abs(xs[free]) @ scale[free])
    assert abs(pap - want) <= TOL * bound, (pap, want, bound)


CASES = [
    ("c2_8", lambda: S.make_c2(8), 0),
    ("c2_9_chunk60", lambda: S.make_c2(9), 60),
    ("c2_12_chunk4096", lambda: S.make_c2(12), 4096),
    ("c2_8_shuffled", lambda: S.shuffle_case(S.make_c2(8), seed=3), 0),
    ("c3_12_stiff", lambda: S.make_c3(12), 0),
    ("batch_mesh_3", lambda: S.make_batch_case(3, lo=2e3, hi=6e3), 0),
    ("c1_24_2d", lambda: S.make_c1(24), 0),
]


@pytest.mark.parametrize("name,make,chunk", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("variant", [1, 2], ids=["per_patch", "paired"])
def test_cg_operator_matches_oracle(env, name, make, chunk, variant):
    P, torch, ctx = env
    case = make()
    A = oracle.PressureMatrix.from_case(case)
    m = P.ps_mesh_upload(ctx, case.dim, case.coords, case.conn, case.dirichlet, chunk_elems=chunk,
                         operator_kernel=variant)
    try:
        P.ps_coeff_set(m, case.alpha, case.beta, case.dt2)
        rng = np.random.default_rng(7)
        for trial in range(2):
            x = rng.standard_normal(case.n_nodes)
            if trial == 1:       # smooth input: the stiffness part nearly cancels
                x = np.sin(3 * case.coords[:, 0]) + case.coords[:, 1] ** 2
            y, pap, xs = _run(P, torch, m, x)
            _check(y, pap, xs, A.apply(xs), row_scale_fast(A, xs), case.dirichlet.astype(bool))
    finally:
        P.ps_mesh_free(m)


@pytest.mark.parametrize("name,make,chunk", CASES[:4], ids=[c[0] for c in CASES[:4]])
@pytest.mark.parametrize("variant", [1, 2], ids=["per_patch", "paired"])
def test_cg_operator_lumped(env, name, make, chunk, variant):
    P, torch, ctx = env
    case = make()
    AL = L.LumpedMatrix(case.dim, case.coords, case.conn, case.dirichlet, case.alpha, case.beta, case.dt2)
    m = P.ps_mesh_upload(ctx, case.dim, case.coords, case.conn, case.dirichlet, chunk_elems=chunk,
                         operator_kernel=variant)
    try:
        P.ps_coeff_set(m, case.alpha, case.beta, case.dt2)
        P.ps_mesh_set_mass(m, P.PS_MASS_LUMPED)
        x = np.random.default_rng(9).standard_normal(case.n_nodes)
        y, pap, xs = _run(P, torch, m, x)
        ref = AL.apply(xs)
        scale = AL.extend(abs(AL.A) @ np.abs(AL.restrict(xs)))
        _check(y, pap, xs, ref, scale, case.dirichlet.astype(bool))
    finally:
        P.ps_mesh_free(m)


@pytest.mark.parametrize("variant", [1, 2], ids=["per_patch", "paired"])
def test_cg_operator_periodic(env, variant):
    P, torch, ctx = env
    case = S.make_periodic_case(3, 8)
    master = case.extra["master"]
    A = PeriodicMatrix(3, case.coords, case.conn, case.dirichlet, master, case.alpha, case.beta, case.dt2)
    m = P.ps_mesh_upload(ctx, 3, case.coords, case.conn, case.dirichlet, periodic=master, operator_kernel=variant)
    try:
        P.ps_coeff_set(m, case.alpha, case.beta, case.dt2)
        x = np.random.default_rng(4).standard_normal(case.n_nodes)
        y, pap, xs = _run(P, torch, m, x)
        xf = A.to_dofs(xs)[A.free]
        ref = A.to_user(A.A @ xf)
        scale = A.to_user(abs(A.A) @ np.abs(xf))
        dirm = case.dirichlet.astype(bool)
        assert np.all(y[dirm] == 0.0)
        free = scale > 0
        assert np.max(np.abs(y - ref)[free] / scale[free]) <= TOL
        assert abs(pap - float(xf @ (A.A @ xf))) <= TOL * float(np.abs(xf) @ (abs(A.A) @ np.abs(xf)))
        assert np.array_equal(y, y[master])
    finally:
        P.ps_mesh_free(m)


def test_cg_operator_full_size_c3_sampled_rows(env):
    """160^3 stiff case, paired-patch kernel: rows sampled over the whole mesh
    (every 5,000th node, computed one by one from the oracle's element
    matrices) and x^T A x against the oracle's assembled matrix."""
    from tests.gpu_util import sampled_rows
    P, torch, ctx = env
    case = S.make_c3()
    m = P.ps_mesh_upload(ctx, 3, case.coords, case.conn, case.dirichlet, operator_kernel=2)
    try:
        P.ps_coeff_set(m, case.alpha, case.beta, case.dt2)
        x = case.extra["xstar"]
        y, pap, xs = _run(P, torch, m, x)
        nodes = np.arange(0, case.n_nodes, 5000)
        ref, sc = sampled_rows(case, xs, nodes)
        dirm = case.dirichlet.astype(bool)[nodes]
        assert np.all(y[nodes][dirm] == 0.0)
        free = ~dirm
        assert np.max(np.abs(y[nodes] - ref)[free] / sc[free]) <= TOL
        A = oracle.PressureMatrix.from_case(case)
        ax = A.apply(xs)
        bound = float(np.abs(xs) @ row_scale_fast(A, xs))
        assert abs(pap - float(xs @ ax)) <= TOL * bound
    finally:
        P.ps_mesh_free(m)


SOLVES = [
    ("c2_12", lambda: S.make_c2(12), 0, False),
    ("c3_12_stiff_warm", lambda: S.make_c3(12), 0, False),
    ("c2_10_shuffled_chunk77", lambda: S.shuffle_case(S.make_c2(10), seed=5), 77, False),
    ("c2_9_lumped", lambda: S.make_c2(9), 0, True),
    ("periodic_3d_8", lambda: S.make_periodic_case(3, 8), 0, False),
]


@pytest.mark.parametrize("name,make,chunk,lumped", SOLVES, ids=[c[0] for c in SOLVES])
@pytest.mark.parametrize("threads", [128, 256])
def test_paired_kernel_solves_match_oracle(env, name, make, chunk, lumped, threads):
    """Mixed-precision two-kernel solves with the paired-patch operator kernel
    (its update kernel then keeps the shared nodes' inputs in the chunk-major
    halo): the oracle's residual gate at 1e-10, the error gate at 1e-13, and
    two runs bitwise equal."""
    P, torch, ctx = env
    case = make()
    master = case.extra.get("master")
    if master is not None:
        A = PeriodicMatrix(3, case.coords, case.conn, case.dirichlet, master, case.alpha, case.beta, case.dt2)
        resid = A.residual
        ref = A.solve(case.b)
    elif lumped:
        A = L.LumpedMatrix(case.dim, case.coords, case.conn, case.dirichlet, case.alpha, case.beta, case.dt2)
        resid = A.residual
        ref = A.solve(case.b)
    else:
        A = oracle.PressureMatrix.from_case(case)
        resid = A.residual
        ref = None
    b = A.apply(case.extra["xstar"]) if "xstar" in case.extra else case.b
    if ref is None:
        ref, _, _, _ = A.cg(b, x0_full=case.x0, precond=1, tol=1e-13)
    m = P.ps_mesh_upload(ctx, case.dim, case.coords, case.conn, case.dirichlet, chunk_elems=chunk,
                         periodic=master, operator_kernel=2, operator_threads=threads)
    try:
        assert P.ps_mesh_get_stats(m).operator_kernel == 2
        P.ps_coeff_set(m, case.alpha, case.beta, case.dt2)
        if lumped:
            P.ps_mesh_set_mass(m, P.PS_MASS_LUMPED)
        bd = torch.as_tensor(b, device="cuda")
        xs = []
        for _ in range(2):
            x = torch.as_tensor(case.x0, device="cuda").clone()
            st, info = P.ps_pressure_solve(m, bd, x, P.make_opts(mode=1, tol=1e-10, engine=P.PS_ENGINE_GRAPH))
            assert st == P.PS_OK
            xs.append(x.cpu().numpy())
        assert np.array_equal(xs[0], xs[1])
        assert resid(b, xs[0]) <= 1.05e-10
        x = torch.as_tensor(case.x0, device="cuda").clone()
        st, info = P.ps_pressure_solve(m, bd, x, P.make_opts(mode=1, tol=1e-13, max_outer=12,
                                                            engine=P.PS_ENGINE_GRAPH))
        xt = x.cpu().numpy()
        assert np.linalg.norm(xt - ref) <= 1e-9 * np.linalg.norm(ref)
    finally:
        P.ps_mesh_free(m)
