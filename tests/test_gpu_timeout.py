"""The failure path of the persistent kernels' bounded grid barrier.

Every device-side wait of the library is bounded: when a wait gives up, the
kernel records an error bit and returns, and the host reports PS_ETIMEOUT
instead of hanging.  Here the grid barrier of the batched persistent kernel
is given a limit of one poll (ps_solve_opts.grid_spin_limit), so that blocks
arriving early give up before the last block arrives.  No bulk copy is in
flight at that barrier (each block's chunk copies completed before its pass
ended), and every block leaves the kernel.  The test checks that the call
returns PS_ETIMEOUT, that the context stays usable, and that the next call
with the default limit solves the same systems to the oracle's residual gate.
(The limit of the bulk-copy mbarrier waits is not shortened: a block that
left with a copy still in flight would be unsafe.)
"""
import numpy as np
import pytest

import oracle
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


def _meshes(P, ctx, cases):
    ms = []
    for c in cases:
        m = P.ps_mesh_upload(ctx, c.dim, c.coords, c.conn, c.dirichlet, chunk_elems=96)
        P.ps_coeff_set(m, c.alpha, c.beta, c.dt2)
        ms.append(m)
    return ms


def test_grid_barrier_timeout_is_reported_and_recovered(env):
    P, torch, ctx = env
    cases = [S.make_c2(12), S.make_c1(48)]        # 108 + 48 chunks: a grid of many blocks
    ms = _meshes(P, ctx, cases)
    try:
        bs = [torch.as_tensor(c.b, device="cuda") for c in cases]
        xs = [torch.zeros(c.n_nodes, dtype=torch.float64, device="cuda") for c in cases]
        with pytest.raises(P.PressureError) as e:
            P.ps_batch_solve(ms, bs, xs, P.make_opts(tol=1e-10, grid_spin_limit=1))
        assert e.value.status == P.PS_ETIMEOUT
        # the same call again, default limit: every system meets the oracle gate
        for x in xs:
            x.zero_()
        st, infos = P.ps_batch_solve(ms, bs, xs, P.make_opts(tol=1e-10))
        assert st == P.PS_OK
        for c, x, inf in zip(cases, xs, infos):
            assert inf.status == P.PS_OK
            assert oracle.PressureMatrix.from_case(c).residual(c.b, x.cpu().numpy()) <= 1.05e-10
        # a single solve on the persistent engine takes the same path
        with pytest.raises(P.PressureError) as e:
            x = torch.zeros_like(bs[0])
            P.ps_pressure_solve(ms[0], bs[0], x, P.make_opts(tol=1e-10, engine=P.PS_ENGINE_PERSISTENT,
                                                            grid_spin_limit=1))
        assert e.value.status == P.PS_ETIMEOUT
        x = torch.zeros_like(bs[0])
        st, info = P.ps_pressure_solve(ms[0], bs[0], x, P.make_opts(tol=1e-10, engine=P.PS_ENGINE_PERSISTENT))
        assert st == P.PS_OK
        assert oracle.PressureMatrix.from_case(cases[0]).residual(cases[0].b, x.cpu().numpy()) <= 1.05e-10
    finally:
        for m in ms:
            P.ps_mesh_free(m)
