"""The autotuner picks a layout and an inner tolerance by measurement through
the C ABI; the parameters it returns give a correct solve."""
import numpy as np
import pytest

import oracle
from paper_2301_08357_gb300 import synthetic as S

pytestmark = pytest.mark.gpu


def test_autotune_returns_working_parameters():
    import torch
    from paper_2301_08357_gb300 import autotune, build
    build.build()
    from paper_2301_08357_gb300 import pressure as P
    case = S.make_c2(14)
    ctx = P.ps_ctx_create(0)
    try:
        res = autotune.tune(P, ctx, case, chunks=(256, 1024), pipelines=(0, 1), inner_tols=(1e-3, 1e-5),
                            reps=5, solve_reps=1)
        assert res["chunk_elems"] in (256, 1024) and res["pipeline"] in (0, 1)
        assert res["inner_tol"] in (1e-3, 1e-5)
        assert len(res["table"]) == 4 and all(r["op_ms"] > 0 for r in res["table"])
        assert res["engine"] in (P.PS_ENGINE_GRAPH, P.PS_ENGINE_FUSED)
        assert all(r["fused_ms"] > 0 for r in res["table"] if r["pipeline"] == 0)
        m = P.ps_mesh_upload(ctx, case.dim, case.coords, case.conn, case.dirichlet,
                             chunk_elems=res["chunk_elems"], pipeline=res["pipeline"])
        P.ps_coeff_set(m, case.alpha, case.beta, case.dt2)
        b = torch.as_tensor(case.b, device="cuda")
        x = torch.zeros_like(b)
        st, info = P.ps_pressure_solve(m, b, x, P.make_opts(inner_tol=res["inner_tol"], engine=res["engine"]))
        A = oracle.PressureMatrix.from_case(case)
        assert st == P.PS_OK and A.residual(case.b, x.cpu().numpy()) <= 1.05e-10
        P.ps_mesh_free(m)
    finally:
        P.ps_ctx_destroy(ctx)


def test_batch_autotune_picks_a_measured_chunk():
    import torch
    from paper_2301_08357_gb300 import autotune, build
    build.build()
    from paper_2301_08357_gb300 import pressure as P
    cases = [S.make_batch_case(i, lo=2e3, hi=6e3) for i in range(4)]
    ctx = P.ps_ctx_create(0)
    try:
        res = autotune.tune_batch(P, ctx, cases, chunks=(0, 768), reps=1)
        assert res["chunk_elems"] in (0, 768)
        assert {r["chunk_elems"] for r in res["table"]} == {0, 768}
        assert all(r["batch_ms"] > 0 for r in res["table"])
        # the chosen layout solves the batch to the gate
        meshes = [P.ps_mesh_upload(ctx, c.dim, c.coords, c.conn, c.dirichlet, chunk_elems=res["chunk_elems"])
                  for c in cases]
        for m, c in zip(meshes, cases):
            P.ps_coeff_set(m, c.alpha, c.beta, c.dt2)
        bs = [torch.as_tensor(c.b, device="cuda") for c in cases]
        xs = [torch.zeros(c.n_nodes, dtype=torch.float64, device="cuda") for c in cases]
        st, infos = P.ps_batch_solve(meshes, bs, xs)
        assert st == P.PS_OK
        for c, x in zip(cases, xs):
            A = oracle.PressureMatrix.from_case(c)
            assert A.residual(c.b, x.cpu().numpy()) <= 1.05e-10
        for m in meshes:
            P.ps_mesh_free(m)
    finally:
        P.ps_ctx_destroy(ctx)
