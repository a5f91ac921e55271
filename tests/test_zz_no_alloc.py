"""The allocation-free operator apply (ps_pressure_apply_noalloc) against the
regular apply, through the C ABI.

Some callers cannot allocate device memory when they apply the operator (their
framework's allocator already holds the memory they may use, or an allocation
would synchronise the device inside their time-step loop); for them the
library keeps the apply's scratch in a fixed 16 MiB device array.  This file
is named so that pytest collects it last.  It must pass alone in a fresh
process and after the other tests: it creates its own context and meshes.
"""
import numpy as np
import pytest

from paper_2301_08357_gb300 import synthetic as S

pytestmark = pytest.mark.gpu

# same bars as the apply parity tests (relative to the largest |entry|)
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


@pytest.mark.parametrize("make", [lambda: S.make_c2(16), lambda: S.make_c1(64)], ids=["3d_16", "2d_64"])
@pytest.mark.parametrize("prec", [1, 2], ids=["f32", "f64"])
def test_noalloc_apply_matches_apply_twice(env, make, prec):
    P, torch, ctx = env
    case = make()
    m = P.ps_mesh_upload(ctx, case.dim, case.coords, case.conn, case.dirichlet)
    try:
        P.ps_coeff_set(m, case.alpha, case.beta, case.dt2)
        dt = torch.float32 if prec == 1 else torch.float64
        rng = np.random.default_rng(21)
        for call in range(2):                       # two calls in a row
            x = torch.as_tensor(rng.standard_normal(case.n_nodes), dtype=dt, device="cuda")
            y_ref = torch.zeros_like(x)
            y_na = torch.full_like(x, float("nan"))
            P.ps_pressure_apply(m, x, y_ref, prec)
            P.ps_pressure_apply_noalloc(m, x, y_na, prec)
            torch.cuda.synchronize()
            a, b = y_ref.cpu().double().numpy(), y_na.cpu().double().numpy()
            assert np.all(np.isfinite(b))
            scale = max(np.abs(a).max(), 1e-300)
            assert np.max(np.abs(a - b)) <= TOL[prec] * scale, (call, np.max(np.abs(a - b)) / scale)
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
