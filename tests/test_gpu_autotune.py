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
        # per chunk size: one patch per thread (plain, pipelined), paired patches (128, 256 threads)
        assert len(res["table"]) == 8 and all(r["op_ms"] > 0 for r in res["table"])
        assert {(r["operator_kernel"], r["operator_threads"]) for r in res["table"]} == {(1, 0), (2, 128), (2, 256)}
        assert all(r["halo_ms"] > 0 for r in res["table"] if r["operator_kernel"] == 2)
        assert res["engine"] in (P.PS_ENGINE_GRAPH, P.PS_ENGINE_FUSED)
        assert all(r["fused_ms"] > 0 for r in res["table"] if r["pipeline"] == 0 and r["operator_kernel"] == 1)
        m = P.ps_mesh_upload(ctx, case.dim, case.coords, case.conn, case.dirichlet,
                             chunk_elems=res["chunk_elems"], pipeline=res["pipeline"],
                             operator_kernel=res["operator_kernel"], operator_threads=res["operator_threads"])
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
        # threads per block and task order swept on the best chunk size
        assert {(r["batch_threads"], r["batch_order"]) for r in res["table"]} == {(128, 0), (128, 1), (256, 0),
                                                                                 (256, 1)}
        assert res["batch_threads"] in (128, 256) and res["batch_order"] in (0, 1)
        # the chosen layout solves the batch to the gate
        meshes = [P.ps_mesh_upload(ctx, c.dim, c.coords, c.conn, c.dirichlet, chunk_elems=res["chunk_elems"])
                  for c in cases]
        for m, c in zip(meshes, cases):
            P.ps_coeff_set(m, c.alpha, c.beta, c.dt2)
        bs = [torch.as_tensor(c.b, device="cuda") for c in cases]
        xs = [torch.zeros(c.n_nodes, dtype=torch.float64, device="cuda") for c in cases]
        st, infos = P.ps_batch_solve(meshes, bs, xs, P.make_opts(batch_threads=res["batch_threads"],
                                                                  batch_order=res["batch_order"]))
        assert st == P.PS_OK
        for c, x in zip(cases, xs):
            A = oracle.PressureMatrix.from_case(c)
            assert A.residual(c.b, x.cpu().numpy()) <= 1.05e-10
        for m in meshes:
            P.ps_mesh_free(m)
    finally:
        P.ps_ctx_destroy(ctx)


@pytest.mark.parametrize("threads", [128, 256])
def test_batch_knobs(threads):
    """The task order changes only which block evaluates which chunk: each
    mesh's arithmetic and reduction order stay the same, so the compacted
    order gives bitwise the result of the (mesh, chunk) order.  The threads per
    block change how a chunk's dot products are split over threads (another
    rounding), so there the gate is the oracle's residual."""
    import torch
    from paper_2301_08357_gb300 import build
    build.build()
    from paper_2301_08357_gb300 import pressure as P
    cases = [S.make_batch_case(i, lo=2e3, hi=2e4) for i in range(6)]
    ctx = P.ps_ctx_create(0)
    try:
        meshes = [P.ps_mesh_upload(ctx, c.dim, c.coords, c.conn, c.dirichlet, chunk_elems=192) for c in cases]
        for m, c in zip(meshes, cases):
            P.ps_coeff_set(m, c.alpha, c.beta, c.dt2)
        bs = [torch.as_tensor(c.b, device="cuda") for c in cases]
        out = []
        for o in (P.make_opts(batch_threads=threads, batch_order=0),
                  P.make_opts(batch_threads=threads, batch_order=1)):
            xs = [torch.zeros(c.n_nodes, dtype=torch.float64, device="cuda") for c in cases]
            st, infos = P.ps_batch_solve(meshes, bs, xs, o)
            assert st == P.PS_OK
            out.append([x.cpu().numpy() for x in xs])
        for c, a, b in zip(cases, out[0], out[1]):
            assert np.array_equal(a, b)
            assert oracle.PressureMatrix.from_case(c).residual(c.b, b) <= 1.05e-10
        for m in meshes:
            P.ps_mesh_free(m)
    finally:
        P.ps_ctx_destroy(ctx)
