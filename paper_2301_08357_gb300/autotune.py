"""Autotuner for the solver's free parameters: for single solves the chunk
size, the FP32 CG operator kernel (one patch per thread, its pipelined
persistent form, or paired patches with 128 or 256 threads per block), the
engine and the inner tolerance of the mixed solver; for meshes solved in
batches the chunk size, the persistent kernel's threads per block and its
task order (batch packing).

It measures through the C ABI only: each candidate mesh layout is uploaded,
the FP32 CG kernels are timed with ps_profile_kernel (CUDA events on the
caller's stream): the operator and update kernels of the two-kernel
iteration (plus the halo gather of the paired-patch kernel) and the fused
one-reduction pass; the cheaper iteration picks the engine.  On the best
layout whole solves are timed with ps_pressure_solve to pick the inner
tolerance.  Batches are timed as whole ps_batch_solve calls on a sample.
The result is a plain dict that the caller passes back as ps_mesh_upload /
ps_solve_opts arguments; nothing is cached behind the caller's back.
"""
from __future__ import annotations

import time

import numpy as np

CHUNKS = (768, 1536, 3072)
PIPELINES = (0, 1)
INNER_TOLS = (1e-3, 1e-4, 1e-5)
# FP32 CG operator kernels: (operator_kernel, operator_threads); the paired
# kernel exists for 3D meshes only
KERNELS = ((1, 0), (2, 128), (2, 256))


def _layout_kw(row):
    return {"chunk_elems": row["chunk_elems"], "pipeline": row["pipeline"],
            "operator_kernel": row["operator_kernel"], "operator_threads": row["operator_threads"]}


def tune(P, ctx, case, stream=None, chunks=CHUNKS, pipelines=PIPELINES, inner_tols=INNER_TOLS,
         kernels=KERNELS, reps=20, solve_reps=2):
    """Return {'chunk_elems', 'pipeline', 'operator_kernel', 'operator_threads', 'engine',
    'inner_tol', 'table': [...]} for `case` (a synthetic.Case or any object
    with dim/coords/conn/dirichlet/alpha/beta/dt2/b).

    `P` is the pressure binding, `ctx` a ps_ctx.  Requires torch for device
    buffers.  Candidates whose layout does not fit the device are skipped.
    The pipelined persistent form exists for the one-patch kernel only."""
    import torch

    table = []
    b = torch.as_tensor(case.b, device="cuda")
    x = torch.zeros_like(b)
    opts = P.make_opts(tol=1e-10)
    cands = []
    for ce in chunks:
        for ok, ot in kernels:
            if ok == 2 and case.dim != 3:
                continue
            for pl in (pipelines if ok == 1 else (0,)):
                cands.append({"chunk_elems": ce, "pipeline": pl, "operator_kernel": ok, "operator_threads": ot})
    for row in cands:
        try:
            m = P.ps_mesh_upload(ctx, case.dim, case.coords, case.conn, case.dirichlet, **_layout_kw(row))
        except P.PressureError:
            continue
        try:
            P.ps_coeff_set(m, case.alpha, case.beta, case.dt2)
            x.zero_()
            P.ps_pressure_solve(m, b, x, opts, stream)      # warm-up, fills the workspace
            k1 = P.ps_profile_kernel(m, P.PS_KERNEL_CG_F32, reps, stream)
            k2 = P.ps_profile_kernel(m, P.PS_KERNEL_UPDATE_F32, reps, stream)
            kh = P.ps_profile_kernel(m, P.PS_KERNEL_HALO_F32, reps, stream) if row["operator_kernel"] == 2 else 0.0
            row.update({"op_ms": k1, "update_ms": k2, "halo_ms": kh, "iter_ms": k1 + k2 + kh,
                        "engine": P.PS_ENGINE_GRAPH})
            if row["pipeline"] == 0 and row["operator_kernel"] == 1:   # the fused pass: one candidate per chunk
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
    m = P.ps_mesh_upload(ctx, case.dim, case.coords, case.conn, case.dirichlet, **_layout_kw(best))
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
    return dict(_layout_kw(best), engine=best["engine"], inner_tol=solves[0]["inner_tol"] if solves else 1e-4,
                table=table, solves=solves)


BATCH_CHUNKS = (0, 768, 1536)
BATCH_THREADS = (128, 256)
BATCH_ORDERS = (0, 1)


def _time_batch(P, ctx, cases, chunk, opts, reps, stream):
    """Best of `reps` timed ps_batch_solve calls (after one warm-up) on the
    sample uploaded with `chunk`; None if the layout does not fit or a solve
    fails."""
    import torch

    meshes = []
    try:
        for c in cases:
            m = P.ps_mesh_upload(ctx, c.dim, c.coords, c.conn, c.dirichlet, chunk_elems=chunk)
            meshes.append(m)
            P.ps_coeff_set(m, c.alpha, c.beta, c.dt2)
    except P.PressureError:
        for m in meshes:
            P.ps_mesh_free(m)
        return None
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
    except P.PressureError:
        ts = []
    finally:
        for m in meshes:
            P.ps_mesh_free(m)
    return 1e3 * float(np.min(ts[1:])) if len(ts) > 1 else None


def tune_batch(P, ctx, cases, stream=None, chunks=BATCH_CHUNKS, threads=BATCH_THREADS, orders=BATCH_ORDERS,
               reps=2, opts=None):
    """Parameters for meshes that are solved together (ps_batch_solve or the
    serving loop): the chunk size (there the other meshes fill the GPU, so
    larger chunks -- fewer shared nodes, less redundant work per pass -- can
    beat the single-solve default), then on the best chunk size the
    persistent kernel's threads per block and its task order (batch
    packing: the (mesh, chunk) list, or the running meshes' chunks compacted
    each pass so that the meshes still iterating are spread over all blocks).
    `cases` is a sample of the batch (synthetic.Case objects); each candidate
    uploads the sample, warms up once and keeps the best of `reps` timed
    batch solves.  Returns {'chunk_elems', 'batch_threads', 'batch_order',
    'table'}; chunk 0 means the library default.  Candidates whose layout does
    not fit are skipped."""
    base = opts if opts is not None else P.make_opts(tol=1e-10)

    def with_(**kw):
        o = P.ps_solve_opts.from_buffer_copy(base)
        for k, v in kw.items():
            setattr(o, k, v)
        return o

    table = []
    for ce in chunks:
        ms = _time_batch(P, ctx, cases, ce, with_(), reps, stream)
        if ms is not None:
            table.append({"chunk_elems": ce, "batch_threads": base.batch_threads or 256,
                          "batch_order": base.batch_order, "batch_ms": ms})
    if not table:
        raise RuntimeError("autotune: no candidate chunk size could be measured")
    best_chunk = min(table, key=lambda r: r["batch_ms"])["chunk_elems"]
    for nt in threads:
        for od in orders:
            if any(r["chunk_elems"] == best_chunk and r["batch_threads"] == nt and r["batch_order"] == od
                   for r in table):
                continue
            ms = _time_batch(P, ctx, cases, best_chunk, with_(batch_threads=nt, batch_order=od), reps, stream)
            if ms is not None:
                table.append({"chunk_elems": best_chunk, "batch_threads": nt, "batch_order": od, "batch_ms": ms})
    table.sort(key=lambda r: r["batch_ms"])
    best = table[0]
    return {"chunk_elems": best["chunk_elems"], "batch_threads": best["batch_threads"],
            "batch_order": best["batch_order"], "table": table}
