"""The allocation-free operator apply (ps_pressure_apply_noalloc) through the
C ABI, against the oracle and the regular apply.

Some callers cannot allocate device memory when they apply the operator (their
framework's allocator already holds the memory they may use, or an allocation
would synchronise the device inside their time-step loop); for them the
library keeps the apply's scratch in a fixed 16 MiB device array, committed
when the first context on the device is created.  Checked here:
  * two calls in a row, element by element against the oracle's assembled
    matrix (the bars of the apply parity tests, relative to the row scale
    s_i = sum_j |A_ij x_j|) and against ps_pressure_apply, on 2D and 3D
    meshes, a periodic mesh and the lumped operator;
  * on a freshly uploaded mesh whose workspace does not exist yet, the call
    changes neither the context's bytes in use nor the mesh's device bytes;
  * meshes above the limit are rejected.
This file is named so that pytest collects it last.  It must pass alone in a
fresh process and after the other tests: it creates its own context and meshes.
"""
import numpy as np
import pytest

import oracle
from oracle import lumped as L
from oracle.periodic import PeriodicMatrix
from paper_2301_08357_gb300 import synthetic as S

pytestmark = pytest.mark.gpu

TOL = {2: 1e-12, 1: 2e-5}


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


def _consistent(case):
    A = oracle.PressureMatrix.from_case(case)
    M = abs(A.scipy())

    def ref(x):
        return A.apply(x), A.extend(M @ np.abs(A.restrict(x)))
    return ref


def _lumped(case):
    AL = L.LumpedMatrix(case.dim, case.coords, case.conn, case.dirichlet, case.alpha, case.beta, case.dt2)
    M = abs(AL.A)

    def ref(x):
        return AL.apply(x), AL.extend(M @ np.abs(AL.restrict(x)))
    return ref


def _periodic(case):
    A = PeriodicMatrix(case.dim, case.coords, case.conn, case.dirichlet, case.extra["master"], case.alpha,
                       case.beta, case.dt2)
    M = abs(A.A)

    def ref(x):
        xf = A.to_dofs(x)[A.free]
        return A.to_user(A.A @ xf), A.to_user(M @ np.abs(xf))
    return ref


CASES = [
    ("3d_16", lambda: S.make_c2(16), _consistent, False),
    ("2d_64", lambda: S.make_c1(64), _consistent, False),
    ("3d_10_lumped", lambda: S.make_c2(10), _lumped, True),
    ("3d_8_periodic", lambda: S.make_periodic_case(3, 8), _periodic, False),
]


def _upload(P, ctx, case, lumped):
    m = P.ps_mesh_upload(ctx, case.dim, case.coords, case.conn, case.dirichlet,
                         periodic=case.extra.get("master"))
    P.ps_coeff_set(m, case.alpha, case.beta, case.dt2)
    if lumped:
        P.ps_mesh_set_mass(m, P.PS_MASS_LUMPED)
    return m


@pytest.mark.parametrize("name,make,oracle_of,lumped", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("prec", [1, 2], ids=["f32", "f64"])
def test_noalloc_apply_matches_oracle_and_apply_twice(env, name, make, oracle_of, lumped, prec):
    P, torch, ctx = env
    case = make()
    ref_of = oracle_of(case)
    m = _upload(P, ctx, case, lumped)
    try:
        dt = torch.float32 if prec == 1 else torch.float64
        rng = np.random.default_rng(21)
        dirm = case.dirichlet.astype(bool)
        for call in range(2):                       # two calls in a row
            x = torch.as_tensor(rng.standard_normal(case.n_nodes), dtype=dt, device="cuda")
            y_na = torch.full_like(x, float("nan"))
            P.ps_pressure_apply_noalloc(m, x, y_na, prec)
            y_ref = torch.full_like(x, float("nan"))
            P.ps_pressure_apply(m, x, y_ref, prec)
            torch.cuda.synchronize()
            xs = x.cpu().double().numpy()
            b, a = y_na.cpu().double().numpy(), y_ref.cpu().double().numpy()
            want, scale = ref_of(xs)
            assert np.all(np.isfinite(b)) and np.all(b[dirm] == 0.0)
            free = scale > 0
            err = np.max(np.abs(b - want)[free] / scale[free])
            assert err <= TOL[prec], (call, err)
            assert np.max(np.abs(b - a)[free] / scale[free]) <= 2 * TOL[prec], call
    finally:
        P.ps_mesh_free(m)


def test_noalloc_apply_allocates_nothing_on_a_fresh_mesh(env):
    P, torch, ctx = env
    case = S.make_c2(12)
    ref_of = _consistent(case)
    m = _upload(P, ctx, case, False)
    try:
        x = torch.as_tensor(np.random.default_rng(3).standard_normal(case.n_nodes), device="cuda")
        y = torch.full_like(x, float("nan"))
        torch.cuda.synchronize()
        ctx_before = P.ps_ctx_bytes_in_use(ctx)
        mesh_before = P.ps_mesh_get_stats(m).device_bytes
        for _ in range(2):
            P.ps_pressure_apply_noalloc(m, x, y, 2)
        torch.cuda.synchronize()
        assert P.ps_ctx_bytes_in_use(ctx) == ctx_before
        assert P.ps_mesh_get_stats(m).device_bytes == mesh_before
        want, scale = ref_of(x.cpu().numpy())
        got = y.cpu().numpy()
        free = scale > 0
        assert np.max(np.abs(got - want)[free] / scale[free]) <= TOL[2]
        # the regular apply afterwards (it creates the mesh workspace) agrees
        y2 = torch.full_like(x, float("nan"))
        P.ps_pressure_apply(m, x, y2, 2)
        torch.cuda.synchronize()
        assert P.ps_ctx_bytes_in_use(ctx) > ctx_before
        assert np.max(np.abs(y2.cpu().numpy() - got)[free] / scale[free]) <= 2 * TOL[2]
    finally:
        P.ps_mesh_free(m)


def test_noalloc_apply_rejects_meshes_over_the_limit(env):
    P, torch, ctx = env
    case = S.make_c1(1100)                          # 1.21 M nodes: 2 x 9.7 MB of FP64 copies
    m = P.ps_mesh_upload(ctx, case.dim, case.coords, case.conn, case.dirichlet)
    try:
        P.ps_coeff_set(m, case.alpha, case.beta, case.dt2)
        x = torch.zeros(case.n_nodes, dtype=torch.float64, device="cuda")
        y = torch.zeros_like(x)
        with pytest.raises(P.PressureError) as e:
            P.ps_pressure_apply_noalloc(m, x, y, 2)
        assert e.value.status == P.PS_EINVAL
        assert "limit" in str(e.value)
    finally:
        P.ps_mesh_free(m)
