"""Autotuner for the solver's free parameters (chunk size, operator-kernel
variant, single-solve engine, inner tolerance of the mixed solver; chunk size
of meshes solved in batches).

It measures through the C ABI only: each candidate mesh layout is uploaded,
the FP32 CG kernels are timed with ps_profile_kernel (CUDA events on the
caller's stream): the operator and update kernels of the two-kernel
iteration and the fused one-reduction pass; the cheaper iteration picks the
engine.  On the best layout whole solves are timed with ps_pressure_solve to
pick the inner tolerance.  The result is a plain
dict that the caller passes back as ps_mesh_upload / ps_solve_opts
arguments; nothing is cached behind the caller's back.
"""
from __future__ import annotations

import time

import numpy as np

CHUNKS = (768, 1536, 3072)
PIPELINES = (0, 1)
INNER_TOLS = (1e-3, 1e-4, 1e-5)


def tune(P, ctx, case, stream=None, chunks=CHUNKS, pipelines=PIPELINES, inner_tols=INNER_TOLS,
         reps=20, solve_reps=2):
    """Return {'chunk_elems', 'pipeline', 'engine', 'inner_tol', 'table': [...]} for `case`
    (a synthetic.Case or any object with dim/coords/conn/dirichlet/alpha/beta/dt2/b).

    `P` is the pressure binding, `ctx` a ps_ctx.  Requires torch for device
    buffers.  Candidates whose layout does not fit the device are skipped."""
    import torch

    table = []
    b = torch.as_tensor(case.b, device="cuda")
    x = torch.zeros_like(b)
    opts = P.make_opts(tol=1e-10)
    for ce in chunks:
        for pl in pipelines:
            try:
                m = P.ps_mesh_upload(ctx, case.dim, case.coords, case.conn, case.dirichlet, chunk_elems=ce,
                                     pipeline=pl)
            except P.PressureError:
                continue
            try:
                P.ps_coeff_set(m, case.alpha, case.beta, case.dt2)
                x.zero_()
                P.ps_pressure_solve(m, b, x, opts, stream)      # warm-up, fills the workspace
                k1 = P.ps_profile_kernel(m, P.PS_KERNEL_CG_F32, reps, stream)
                k2 = P.ps_profile_kernel(m, P.PS_KERNEL_UPDATE_F32, reps, stream)
                row = {"chunk_elems": ce, "pipeline": pl, "op_ms": k1, "update_ms": k2,
                       "iter_ms": k1 + k2, "engine": P.PS_ENGINE_GRAPH}
                if pl == 0:        # the fused pass does not use the pipelined kernel
                    kf = P.ps_profile_kernel(m, P.PS_KERNEL_CG1_F32, reps, stream)
                    row["fused_ms"] = kf
                    if kf < row["iter_ms"]:
                        row["iter_ms"], row["engine"] = kf, P.PS_ENGINE_FUSED
                table.append(row)
            finally:
                P.ps_mesh_free(m)
    if not table:
        raise RuntimeError("autotune: no candidate layout could be built")
    table.sort(key=lambda r: r["iter_ms"])
    best = table[0]
    # inner tolerance: whole solves on the best layout
    m = P.ps_mesh_upload(ctx, case.dim, case.coords, case.conn, case.dirichlet, chunk_elems=best["chunk_elems"],
                         pipeline=best["pipeline"])
    solves = []
    try:
        P.ps_coeff_set(m, case.alpha, case.beta, case.dt2)
        for it in inner_tols:
            o = P.make_opts(tol=1e-10, inner_tol=it, engine=best["engine"])
            ts = []
            for _ in range(solve_reps + 1):
                x.zero_()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                st, info = P.ps_pressure_solve(m, b, x, o, stream)
                torch.cuda.synchronize()
                ts.append(time.perf_counter() - t0)
            if st == P.PS_OK:
                solves.append({"inner_tol": it, "solve_ms": 1e3 * float(np.min(ts[1:])),
                               "iters": info.iters_inner, "outer": info.iters_outer})
    finally:
        P.ps_mesh_free(m)
    solves.sort(key=lambda r: r["solve_ms"])
    return {"chunk_elems": best["chunk_elems"], "pipeline": best["pipeline"], "engine": best["engine"],
            "inner_tol": solves[0]["inner_tol"] if solves else 1e-4, "table": table, "solves": solves}


BATCH_CHUNKS = (0, 768, 1536)


def tune_batch(P, ctx, cases, stream=None, chunks=BATCH_CHUNKS, reps=2, opts=None):
    """Chunk size for meshes that are solved together (ps_batch_solve or the
    serving loop): there the other meshes fill the GPU, so larger chunks (fewer
    shared nodes, less redundant work per pass) can beat the single-solve
    default.  `cases` is a sample of the batch (synthetic.Case objects); each
    candidate uploads the sample, warms up once and keeps the best of `reps`
    timed batch solves.  Returns {'chunk_elems', 'table'}; 0 means the library
    default.  Candidates whose layout does not fit are skipped."""
    import torch

    opts = opts if opts is not None else P.make_opts(tol=1e-10)
    table = []
    for ce in chunks:
        meshes = []
        try:
            for c in cases:
                m = P.ps_mesh_upload(ctx, c.dim, c.coords, c.conn, c.dirichlet, chunk_elems=ce)
                meshes.append(m)
                P.ps_coeff_set(m, c.alpha, c.beta, c.dt2)
        except P.PressureError:
            for m in meshes:
                P.ps_mesh_free(m)
            continue
        bs = [torch.as_tensor(c.b, device="cuda") for c in cases]
        xs = [torch.zeros(c.n_nodes, dtype=torch.float64, device="cuda") for c in cases]
        ts = []
        try:
            for r in range(reps + 1):
                for x in xs:
                    x.zero_()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                st, _ = P.ps_batch_solve(meshes, bs, xs, opts, stream)
                torch.cuda.synchronize()
                if st == P.PS_OK:
                    ts.append(time.perf_counter() - t0)
        finally:
            for m in meshes:
                P.ps_mesh_free(m)
        if len(ts) > 1:
            table.append({"chunk_elems": ce, "batch_ms": 1e3 * float(np.min(ts[1:]))})
    if not table:
        raise RuntimeError("autotune: no candidate chunk size could be measured")
    table.sort(key=lambda r: r["batch_ms"])
    return {"chunk_elems": table[0]["chunk_elems"], "table": table}
