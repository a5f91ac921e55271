#!/usr/bin/env python
"""Benchmark of the pressure solve: DOF-iterations/s of matrix-free (P)CG on the
P1 pressure system A = M_alpha + dt^2 K_beta (Section 3.4), one GB300.

Default (no flags): the headline line on the stiff 3D case -- the unit cube
160^3 cut into 24,576,000 Kuhn tetrahedra (4,173,281 nodes), alpha from 8
seeded Fourier modes x 1e-4, beta lognormal(0, 1) with a 100x spherical
inclusion, dt^2 = 1e-2, Dirichlet x = 0, b = A x* formed by the FP64 oracle's
assembled matrix, warm start x0 = x*(1 + 0.01 xi).  One step = one solve to a
true FP64 relative residual of 1e-10 through the C ABI (FP32 Jacobi-PCG inside
FP64 defect correction).  value = free nodes x (inner + outer iterations) /
device time, inputs resident in HBM (0.64 GB per operator pass, five times
the L2) and a 256 MB write between steps.  The same line carries the error
against the oracle's solution, the time at the tightened tolerance that
meets the 1e-9 error gate, the roofline of the dominant kernels, the oracle
timed on the host cores, an end-to-end figure with host buffers, and three
sub-objects: "batched" (256 meshes in one batched solve), "served" (a
continuous-batching stream of 64 cases x 20 time steps with per-size-bucket
latency, against the same requests solved one at a time in plain FP64) and
"c2" (the 64^3 single solve).

Prints ONE JSON line (rank 0).  Under torchrun every rank solves its own
replica of the workload (independent systems, no collective on the data
path: weak scaling); value is the sum over ranks / the max time over ranks.

--impl reference times the FP64 CPU oracle (CSR assembly excluded, textbook
Jacobi-PCG with OpenMP sparse products) on the same system, same metric:
each step a bounded sample of Jacobi-PCG iterations.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "pressure CG DOF-iters/s + HBM GB/s; solves/s, p50/p99 ms at 1e-10 rel residual"
UNIT = "DOF-iter/s"

# DRAM bytes (read + write) per launch of a kernel, from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum) of the kernel source as it
# stands, keyed by (kernel, workload), with the capture it came from.  An
# entry is removed whenever the kernel changes; missing means not captured
# (the line then reports null).
TRAFFIC = {
    ("k_cg2_units<false,128,5>", "c3_3d_kuhn_160^3_stiff_warm_tets24576000_nodes4173281"): {
        "bytes": 345454336 + 28280064,
        "source": "ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum (1 pass, cold L2), third launch of "
                  "`python bench.py --workload c3 --steps 1 --warmup 2 --launch-list --no-clocks`; "
                  "profiles/k_cg2_units_kuhn128.md"},
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--n", type=int, default=0, help="cells per side of the Kuhn cube (0 = 160 for c3, 64 else)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="budget of the oracle baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-clocks", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="c4/c5: library default chunks, no batch autotuning")
    ap.add_argument("--launch-list", action="store_true",
                    help="c1/c2/c3: warm-up and timed solves alone (no e2e pass, no kernel timing, no CPU "
                         "baseline), for a profiler's launch list; the line then has no roofline or e2e")
    ap.add_argument("--chunk", type=int, default=0, help="elements per chunk (0 = library default)")
    ap.add_argument("--pipeline", type=int, default=0, help="persistent double-buffered operator kernel")
    ap.add_argument("--operator-kernel", type=int, default=0,
                    help="FP32 CG operator kernel of 3D meshes: 0 auto, 1 one patch per thread, 2 paired patches")
    ap.add_argument("--operator-threads", type=int, default=0, help="threads per block of the paired-patch kernel")
    ap.add_argument("--engine", default="auto", choices=["auto", "graph", "persistent", "fused"])
    ap.add_argument("--workload", default="headline",
                    choices=["headline", "c1", "c2", "c3", "c4", "c5", "projection", "periodic", "eos"],
                    help="headline (default) = the c3 line with batched, served and c2 sub-objects; "
                         "c1/c2/c3 single solves alone; c4 = 256-mesh batch; c5 = served stream with a "
                         "Poisson rate sweep")
    ap.add_argument("--no-sub", action="store_true", help="headline: the c3 line without sub-objects")
    ap.add_argument("--tight-tol", type=float, default=1e-13,
                    help="c3: tolerance of the solves that meet the 1e-9 error gate")
    ap.add_argument("--meshes", type=int, default=256, help="c4: meshes in the batch")
    ap.add_argument("--cases", type=int, default=64, help="c5: simulated cases")
    ap.add_argument("--case-steps", type=int, default=20, help="c5: time steps per case")
    ap.add_argument("--rates", default="0.5,1,2", help="c5: arrival rates as multiples of saturation")
    ap.add_argument("--size-scale", type=float, default=1.0, help="c4/c5: scale the mesh-size range")
    return ap.parse_args()


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def aggregate(total_ms, work, device=None):
    """Whole-job numbers over ranks (replicas): the max time and the summed
    work.  A no-op without an initialised process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(total_ms), float(work)
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    w = torch.tensor([float(work)], dtype=torch.float64, device=device)
    dist.all_reduce(w)
    return float(t.item()), float(w.item())


def parse_clocks(lines):
    """nvidia-smi --query-gpu=<Clocks.Q> --format=csv,noheader,nounits lines ->
    {sm_mhz (median), sm_max_mhz, reasons (throttle reasons seen active), samples}."""
    sm, mx, reasons = [], 0.0, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in lines:
        parts = [p.strip() for p in line.split(",")]
        if len(parts) < 9:
            continue
        try:
            sm.append(float(parts[1]))
            mx = max(mx, float(parts[2]))
        except ValueError:
            continue
        for nm, v in zip(names, parts[5:9]):
            if v.lower().startswith("active"):
                reasons.add(nm)
    if not sm:
        return None
    return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def workload_name(n):
    return "c2_3d_kuhn_%d^3_tets%d_nodes%d" % (n, 6 * n ** 3, (n + 1) ** 3)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        with open(self.path) as f:
            out = parse_clocks(f.readlines())
        os.unlink(self.path)
        return out


def cpu_baseline(case, seconds, steps=None):
    """Oracle Jacobi-PCG to 1e-10 on the full system, repeated until `seconds`."""
    import oracle
    A = oracle.PressureMatrix.from_case(case)
    done, iters, t_used, times = 0, 0, 0.0, []
    while (steps is None and (t_used < seconds or done == 0)) or (steps is not None and done < steps):
        t0 = time.perf_counter()
        x, st, it, rr = A.cg(case.b, precond=1, tol=1e-10)
        dt = time.perf_counter() - t0
        times.append(dt)
        t_used += dt
        iters += it
        done += 1
    return {"value": case.n_free * iters / t_used, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": "%d full Jacobi-PCG solve(s) of the same system to 1e-10 (%d iterations each, "
                      "CSR assembly excluded), %.1f s" % (done, iters // max(done, 1), t_used),
            "solves": done, "seconds": t_used, "times": times}


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo), for the record."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


C3_ITERS_PER_CALL = 25   # oracle Jacobi-PCG iterations per timed call (CPU samples)


def c3_name(case):
    return "c3_3d_kuhn_%d^3_stiff_warm_tets%d_nodes%d" % (case.n, case.n_elems, case.n_nodes)


def headline_config(case, ws=1):
    """The workload of the headline line, shared by both arms (same keys and values)."""
    return {"workload": c3_name(case), "n_free": int(case.n_free), "n_elems": int(case.n_elems),
            "mode": "mixed (FP32 Jacobi-PCG inside FP64 defect correction)", "precond": "jacobi", "tol": 1e-10,
            "b": "A x* formed by the FP64 oracle's assembled matrix", "x0": "x* (1 + 0.01 xi)",
            "l2": "inputs larger than L2 (0.64 GB per operator pass) and a 256 MB write between steps",
            "parallelism": "replicas" if ws > 1 else "single"}


def oracle_pcg_sample(A, b, x0, seconds=0.0, calls=None):
    """The oracle's Jacobi-PCG on a bounded sample of the workload: calls of
    C3_ITERS_PER_CALL iterations from x0 (each starting from the true
    residual), repeated until `seconds` have passed (or `calls` times)."""
    import oracle
    iters, t_used, n, times = 0, 0.0, 0, []
    while (calls is None and (n == 0 or t_used < seconds)) or (calls is not None and n < calls):
        t0 = time.perf_counter()
        _, _, it, _ = A.cg(b, x0_full=x0, precond=1, tol=1e-30, max_it=C3_ITERS_PER_CALL, max_restarts=0)
        dt = time.perf_counter() - t0
        times.append(dt)
        t_used += dt
        iters += it
        n += 1
    return {"value": A.n_free * iters / t_used, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": "%d call(s) of %d Jacobi-PCG iterations of the oracle on the full system from x0 "
                      "(CSR assembly excluded), %.1f s" % (n, C3_ITERS_PER_CALL, t_used),
            "iters": iters, "seconds": t_used, "times": times}


def run_reference(args):
    """The oracle on the headline workload, timed on the host cores: every
    step is one bounded sample (C3_ITERS_PER_CALL Jacobi-PCG iterations on
    the full system from x0).  Rank 0 only under torchrun."""
    ws, rank, local = dist_setup()
    if rank != 0:
        return
    import oracle
    from paper_2301_08357_gb300 import synthetic as S
    case = S.make_c3(args.n or 160)
    t0 = time.perf_counter()
    A = oracle.PressureMatrix.from_case(case)
    t_asm = time.perf_counter() - t0
    b = A.apply(case.extra["xstar"])
    if max(args.warmup, 0):
        oracle_pcg_sample(A, b, case.x0, calls=1)
    cb = oracle_pcg_sample(A, b, case.x0, calls=max(args.steps, 1))
    ms = 1e3 * cb["seconds"] / max(args.steps, 1)
    out = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": headline_config(case),
           "cpu_baseline": {"value": cb["value"], "unit": UNIT, "cores": cb["cores"], "kind": "oracle",
                            "sample": cb["sample"] + "; each step is one call", "assembly_s": t_asm},
           "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


# FP64 peak of the part: 152 SMs x 2 DFMA per clock x 2 flops x 2.07 GHz
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def fp64_flops(stats, lumped, cg):
    """Algorithmic FP64 flops of one FP64 operator pass with the precomputed
    element geometry (an FMA counts 2): per element the stiffness differences
    (3D 24, 2D 13) and the mass term (consistent 3D 47 / 2D 35, lumped 4(d+1)+1),
    3 accumulations; per node the incidence sums E(d+1)/N plus 3 (residual and
    its dot) or 4 (CG direction and p.Ap)."""
    E, N, d = stats.n_elems, stats.n_nodes, stats.dim
    k = 24 if d == 3 else 13
    mass = (2 * (d + 1) + 1) if lumped else (47 if d == 3 else 35)
    per_elem = k + mass + (d if d == 3 else 2)
    per_node = E * (d + 1) / N + (4 if cg else 3)
    return per_elem * E + per_node * N


def kernel_roofline(P, m, stats, mode, fused, stream, workload, lumped=False):
    """Roofline entry of the solve's dominant kernel: algorithmic bytes per
    launch over its CUDA-event time (ps_profile_kernel, back-to-back launches
    on `stream`), against the measured HBM copy bandwidth.  The FP64 passes
    are bound by the FP64 pipe instead: FP64 mode reports its operator kernel
    as "alu" (algorithmic FP64 flops against FP64_PEAK_TFLOPS, HBM fraction
    beside it), and every line carries the FP64 residual pass the same way."""
    if fused:
        which, kname = P.PS_KERNEL_CG1_F32, "k_cg1_chunks<%d>" % stats.dim
    elif mode == P.PS_MODE_MIXED and stats.operator_kernel == 2:
        which, kname = P.PS_KERNEL_CG_F32, "k_cg2_units<%s,128,5>" % ("true" if lumped else "false")
    elif mode == P.PS_MODE_MIXED:
        which, kname = P.PS_KERNEL_CG_F32, "k_cg2_chunks<%d,float>" % stats.dim
    else:
        which, kname = P.PS_KERNEL_CG_F64, "k_cg2_chunks<%d,double>" % stats.dim
    kern_ms = P.ps_profile_kernel(m, which, reps=50, stream=stream)
    kern_other = {name: P.ps_profile_kernel(m, k, reps=20, stream=stream)
                  for name, k in (("cg1_f32_fused", P.PS_KERNEL_CG1_F32), ("cg_f32_two_pass", P.PS_KERNEL_CG_F32),
                                  ("update_f32", P.PS_KERNEL_UPDATE_F32), ("apply_f32", P.PS_KERNEL_APPLY_F32),
                                  ("resid_f64", P.PS_KERNEL_RESID_F64), ("halo_f32", P.PS_KERNEL_HALO_F32))}
    E, N, d = stats.n_elems, stats.n_nodes, stats.dim
    esz = 8 if mode == P.PS_MODE_FP64 else 4
    # per element: d+1 vertex ids (i32) + beta*dt^2
    elem_b = 4 * (d + 1) + esz
    if fused:
        # per node: coordinates + alpha, r w s p x D^-1 read, r s p x w written
        node_b = esz * (d + 1) + 6 * esz + 5 * esz
    else:
        # per node: coordinates + alpha, p_old r D^-1 read, p q written
        node_b = esz * (d + 1) + 3 * esz + 2 * esz
    alg_bytes = elem_b * E + node_b * N
    peak, peak_kind = peaks()
    achieved = alg_bytes / (kern_ms / 1e3) / 1e9
    res_ms = kern_other["resid_f64"]
    res_flops = fp64_flops(stats, lumped, cg=False)
    res_bytes = (4 * (d + 1) + 8) * E + (8 * (d + 1) + 3 * 8) * N
    fp64_resid = {"kernel": "k_chunks<%d,double,kResid>" % d, "bound": "alu", "unit": "TFLOP/s",
                  "achieved": res_flops / (res_ms / 1e3) / 1e12, "peak": FP64_PEAK_TFLOPS,
                  "frac": res_flops / (res_ms / 1e3) / 1e12 / FP64_PEAK_TFLOPS,
                  "hbm_frac": res_bytes / (res_ms / 1e3) / 1e9 / peak, "flops_per_launch": res_flops,
                  "kernel_ms": res_ms}
    if mode == P.PS_MODE_FP64:
        flops = fp64_flops(stats, lumped, cg=True)
        tf = flops / (kern_ms / 1e3) / 1e12
        tr = TRAFFIC.get((kname, workload))
        return {"bound": "alu", "achieved": tf, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": tf / FP64_PEAK_TFLOPS, "traffic": tr["bytes"] if tr else None, "kernel": kname,
                "kernel_ms": kern_ms, "flops_per_launch": flops, "hbm_frac": achieved / peak,
                "alg_bytes_per_launch": alg_bytes, "peak_kind": "nominal FP64 (2 DFMA/clk/SM x 152 SMs x 2.07 GHz)",
                "other_kernels_ms": kern_other, "fp64_resid": fp64_resid, "chunks": stats.n_chunks}
    tr = TRAFFIC.get((kname, workload))
    upd_ms = kern_other["update_f32"]
    upd_bytes = 28 * N   # x, r, p, q, D^-1 read and x, r written, FP32
    update = {"kernel": "k_cg2_update<float>", "bound": "hbm", "unit": "GB/s", "kernel_ms": upd_ms,
              "alg_bytes_per_launch": upd_bytes, "achieved": upd_bytes / (upd_ms / 1e3) / 1e9,
              "peak": peak, "frac": upd_bytes / (upd_ms / 1e3) / 1e9 / peak}
    if stats.operator_kernel == 2:
        update["note"] = ("blocks store their rz, rr shares only; the halo gather (halo_f32) sums them in its "
                          "first block and ends the iteration")
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": tr["bytes"] if tr else None,
            "traffic_source": tr["source"] if tr else "not captured for the kernel as it stands",
            "kernel": kname, "update": update,
            "kernel_ms": kern_ms, "alg_bytes_per_launch": alg_bytes, "peak_kind": peak_kind,
            "other_kernels_ms": kern_other, "fp64_resid": fp64_resid, "chunks": stats.n_chunks,
            "shared_node_frac": stats.n_shared / stats.n_nodes,
            "note": "working set ~%.0f MB/launch: %s" % (
                alg_bytes / 1e6, "L2-resident between iterations" if alg_bytes < 100e6 else "exceeds L2 (129 MB)")}


def run_ours(args):
    import torch

    ws, rank, local = dist_setup()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    import contextlib
    from __graft_entry__ import build
    if rank == 0 or ws == 1:
        with contextlib.redirect_stdout(sys.stderr):   # keep stdout to the one JSON line
            build()
    if ws > 1:
        torch.distributed.barrier()
    from paper_2301_08357_gb300 import pressure as P
    from paper_2301_08357_gb300 import synthetic as S

    args.n = args.n or 64
    case = S.make_c2(args.n)
    ctx = P.ps_ctx_create(local)
    m = P.ps_mesh_upload(ctx, case.dim, case.coords, case.conn, case.dirichlet, chunk_elems=args.chunk,
                         pipeline=args.pipeline, operator_kernel=args.operator_kernel,
                         operator_threads=args.operator_threads)
    P.ps_coeff_set(m, case.alpha, case.beta, case.dt2)
    stats = P.ps_mesh_get_stats(m)
    stream = torch.cuda.current_stream()
    mode = P.PS_MODE_MIXED if args.mode == "mixed" else P.PS_MODE_FP64
    engine = {"auto": P.PS_ENGINE_AUTO, "graph": P.PS_ENGINE_GRAPH, "persistent": P.PS_ENGINE_PERSISTENT,
              "fused": P.PS_ENGINE_FUSED}[args.engine]
    opts = P.make_opts(mode=mode, tol=1e-10, engine=engine)
    b = torch.as_tensor(case.b, device="cuda")
    x = torch.zeros_like(b)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def one(timed_events=None):
        x.zero_()
        st, info = P.ps_pressure_solve(m, b, x, opts, stream)
        if st != P.PS_OK:
            raise RuntimeError("solve failed: %s" % P.ps_status_str(st))
        return info

    for _ in range(max(args.warmup, 3)):
        one()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    if not args.no_clocks:
        clocks.start()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    step_ms, iters, launches = [], 0, 0
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for k in range(args.steps):
        flush.fill_(k & 0xff)          # L2 flush between steps (not timed)
        x.zero_()
        ev[k][0].record(stream)
        st, info = P.ps_pressure_solve(m, b, x, opts, stream)
        ev[k][1].record(stream)
        if st != P.PS_OK:
            raise RuntimeError("solve failed: %s" % P.ps_status_str(st))
        iters += info.iters_inner + info.iters_outer
        launches += info.kernel_launches
    torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b_) for a, b_ in ev]
    total_ms = float(np.sum(step_ms))
    if ws > 1:
        torch.distributed.barrier()
    clk = clocks.stop() if not args.no_clocks else None
    last_info = info
    dof_iters = case.n_free * iters
    t_max, tot_dof = aggregate(total_ms, dof_iters, device="cuda")
    value = tot_dof / (t_max / 1e3)
    if args.launch_list:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                              "warmup": max(args.warmup, 3), "ms_per_step": t_max / args.steps,
                              "config": {"workload": workload_name(args.n), "engine": args.engine},
                              "gpu_launches": launches, "launch_list_run": True}))
        P.ps_mesh_free(m)
        P.ps_ctx_destroy(ctx)
        return

    # ---- end to end through the C ABI with host buffers (copies timed)
    b_h = torch.as_tensor(case.b).pin_memory()
    x0_h = torch.zeros(case.n_nodes, dtype=torch.float64).pin_memory()
    x_h = torch.empty_like(x0_h).pin_memory()
    e2e_ms = []
    for k in range(args.steps):
        flush.fill_(k & 0xff)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b.copy_(b_h, non_blocking=True)
        x.copy_(x0_h, non_blocking=True)
        st, info = P.ps_pressure_solve(m, b, x, opts, stream)
        x_h.copy_(x, non_blocking=True)
        torch.cuda.synchronize()
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
    e2e_val = case.n_free * (info.iters_inner + info.iters_outer) * len(e2e_ms) / (np.sum(e2e_ms) / 1e3)

    # ---- roofline of the dominant kernel
    fused = mode == P.PS_MODE_MIXED and (args.engine == "fused" or (args.engine == "auto" and case.n_nodes <= 200000))
    roof = kernel_roofline(P, m, stats, mode, fused, stream, workload_name(args.n))

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cb = cpu_baseline(case, args.cpu_seconds)
        cpu = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")}
        # the same oracle on one core (one solve), and the host's CPU model
        import oracle
        n_all = oracle.num_threads()
        oracle.set_threads(1)
        try:
            c1 = cpu_baseline(case, 0.0, steps=1)
        finally:
            oracle.set_threads(n_all)
        cpu["single_core"] = {"value": c1["value"], "unit": UNIT, "cores": 1, "sample": c1["sample"]}
        cpu["cpu_model"] = cpu_model()

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": max(args.warmup, 3), "ms_per_step": t_max / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": "f32+f64" if mode == P.PS_MODE_MIXED else "f64", "data": "synthetic",
           "config": {"workload": workload_name(args.n), "n_free": case.n_free, "n_elems": case.n_elems,
                      "mode": args.mode, "precond": "jacobi", "tol": 1e-10,
                      "iters_per_solve": last_info.iters_inner + last_info.iters_outer,
                      "outer_per_solve": last_info.iters_outer, "rel_res": last_info.rel_res,
                      "l2": "flushed between steps (256 MB write); the 64^3 system itself fits in L2",
                      "parallelism": "replicas" if ws > 1 else "single"},
           "solves_per_s": 1e3 * args.steps / t_max * ws,
           "p50_ms": float(np.percentile(step_ms, 50)), "p99_ms": float(np.percentile(step_ms, 99)),
           "roofline": roof, "cpu_baseline": cpu,
           "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": 16 * case.n_nodes,
                   "d2h_bytes_per_step": 8 * case.n_nodes, "ms_per_step": float(np.mean(e2e_ms))},
           "gpu_launches": launches, "clocks": clk}
    if rank == 0:
        print(json.dumps(out))
    P.ps_mesh_free(m)
    P.ps_ctx_destroy(ctx)
    if ws > 1:
        torch.distributed.destroy_process_group()


def _pctl(v, q):
    return float(np.percentile(np.asarray(v), q)) if len(v) else None


def run_single(args, which):
    """c1 (2D 64^2, FP64 plain PCG), c3 (160^3 stiff, mixed, warm start) and
    periodic (the C2 set-up on n^3, periodic in y and z by vertex merging)."""
    import contextlib
    import torch
    from __graft_entry__ import build
    with contextlib.redirect_stdout(sys.stderr):
        build()
    from paper_2301_08357_gb300 import pressure as P
    from paper_2301_08357_gb300 import synthetic as S
    case = S.make_c1() if which == "c1" else (S.make_c3(args.n or 160) if which == "c3"
                                              else S.make_periodic_case(3, args.n or 64))
    mode = P.PS_MODE_FP64 if (which == "c1" or args.mode == "fp64") else P.PS_MODE_MIXED
    ctx = P.ps_ctx_create(0)
    m = P.ps_mesh_upload(ctx, case.dim, case.coords, case.conn, case.dirichlet, chunk_elems=args.chunk,
                         periodic=case.extra.get("master"))
    P.ps_coeff_set(m, case.alpha, case.beta, case.dt2)
    stream = torch.cuda.current_stream()
    if which == "c3":
        # b = A xstar with the library's FP64 operator (an input of the timed
        # solve, not a parity value); x0 = xstar (1 + 0.01 xi)
        xs = torch.as_tensor(case.extra["xstar"], device="cuda")
        b = torch.empty_like(xs)
        P.ps_pressure_apply(m, xs, b, P.PS_F64, stream)
        x0 = torch.as_tensor(case.x0, device="cuda")
    else:
        b = torch.as_tensor(case.b, device="cuda")
        x0 = torch.zeros_like(b)
    opts = P.make_opts(mode=mode, tol=1e-10)
    x = x0.clone()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(max(args.warmup, 3)):
        x.copy_(x0)
        P.ps_pressure_solve(m, b, x, opts, stream)
    times, iters, infos = [], 0, None
    for k in range(args.steps):
        flush.fill_(k & 0xff)
        x.copy_(x0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st, info = P.ps_pressure_solve(m, b, x, opts, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
        iters += info.iters_inner + info.iters_outer
        infos = info
    # free unknowns (merged periodic vertices counted once)
    n_free = infos.n_free if infos is not None else case.n_free
    if args.launch_list:
        tot = float(np.sum(times))
        print(json.dumps({"metric": METRIC, "value": n_free * iters / (tot / 1e3), "unit": UNIT,
                          "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": tot / args.steps,
                          "config": {"workload": case.name}, "launch_list_run": True}))
        P.ps_mesh_free(m)
        P.ps_ctx_destroy(ctx)
        return
    stats = P.ps_mesh_get_stats(m)
    roof = kernel_roofline(P, m, stats, mode, False, stream, case.name)
    err = None
    if which == "c3":
        xs_h = case.extra["xstar"]
        err = float(np.linalg.norm(x.cpu().numpy() - xs_h) / np.linalg.norm(xs_h))
    tot = float(np.sum(times))
    out = {"metric": METRIC, "value": n_free * iters / (tot / 1e3), "unit": UNIT, "n_gpus": 1,
           "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": tot / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64" if mode == P.PS_MODE_FP64 else "f32+f64", "data": "synthetic",
           "config": {"workload": case.name, "n_free": n_free, "n_elems": case.n_elems,
                      "mode": "fp64" if mode == P.PS_MODE_FP64 else "mixed",
                      "iters_per_solve": infos.iters_inner + infos.iters_outer, "outer_per_solve": infos.iters_outer,
                      "rel_res": infos.rel_res, "rel_err_vs_xstar": err,
                      "l2": "flushed between steps (256 MB write)"},
           "solves_per_s": 1e3 * args.steps / tot, "p50_ms": _pctl(times, 50), "p99_ms": _pctl(times, 99),
           "roofline": roof}
    print(json.dumps(out))
    P.ps_mesh_free(m)
    P.ps_ctx_destroy(ctx)


def batch_tuning(args, autotune, P, ctx, cases):
    """Chunk size, persistent-kernel threads per block and task order for the
    batched / served workloads: --chunk if given (library defaults for the
    rest), else the batch autotuner on every 8th case (outside any timed
    region).  Returns (chunk_elems, {"batch_threads", "batch_order"}, record)."""
    if args.chunk or args.no_tune:
        return args.chunk, {"batch_threads": 0, "batch_order": 0}, None
    sample = cases[::8]
    res = autotune.tune_batch(P, ctx, sample)
    return (res["chunk_elems"], {"batch_threads": res["batch_threads"], "batch_order": res["batch_order"]},
            {"sample_meshes": len(sample), "table": res["table"]})


def bench_batch(args, P, S, autotune, torch):
    """c4: 256 independent meshes (half 2D triangle squares, half 3D Kuhn cubes,
    2k-200k nodes) in one batched solve per step.  Returns the measurement as
    a dict (solves/s, batch-time percentiles over the steps, accuracy, clocks)."""
    ctx = P.ps_ctx_create(0)
    meshes, bs, xs, n_free = [], [], [], []
    t0 = time.perf_counter()
    cases = [S.make_batch_case(i, lo=2e3 * args.size_scale, hi=2e5 * args.size_scale) for i in range(args.meshes)]
    chunk, knobs, tune = batch_tuning(args, autotune, P, ctx, cases)
    for c in cases:
        m = P.ps_mesh_upload(ctx, c.dim, c.coords, c.conn, c.dirichlet, chunk_elems=chunk)
        P.ps_coeff_set(m, c.alpha, c.beta, c.dt2)
        meshes.append(m)
        bs.append(torch.as_tensor(c.b, device="cuda"))
        xs.append(torch.zeros(c.n_nodes, dtype=torch.float64, device="cuda"))
        n_free.append(c.n_free)
    setup_s = time.perf_counter() - t0
    opts = P.make_opts(tol=1e-10, **knobs)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(max(args.warmup, 3)):
        for x in xs:
            x.zero_()
        P.ps_batch_solve(meshes, bs, xs, opts, stream)
    torch.cuda.synchronize()
    clocks = Clocks(0)
    if not args.no_clocks:
        clocks.start()
    times, dof_iters, launches, alg_bytes = [], 0, 0, 0.0
    for k in range(args.steps):
        flush.fill_(k & 0xff)
        for x in xs:
            x.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st, infos = P.ps_batch_solve(meshes, bs, xs, opts, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
        if st != P.PS_OK:
            raise RuntimeError("batched solve failed: %s" % P.ps_status_str(st))
        dof_iters += sum(nf * (inf.iters_inner + inf.iters_outer) for nf, inf in zip(n_free, infos))
        launches += max(inf.kernel_launches for inf in infos)
        # algorithmic bytes of the inner iterations (the fused one-reduction
        # pass of the persistent kernel: per element d + 1 vertex ids and
        # beta dt^2, per node coordinates + alpha and the x r s p w reads and
        # writes, FP32); the outer FP64 passes are not counted
        alg_bytes += sum(inf.iters_inner * ((4 * (c.dim + 1) + 4) * c.n_elems + (4 * (c.dim + 1) + 44) * c.n_nodes)
                         for c, inf in zip(cases, infos))
    clk = clocks.stop() if not args.no_clocks else None
    tot = float(np.sum(times))
    peak, peak_kind = peaks()
    ach = alg_bytes / (tot / 1e3) / 1e9
    roof = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
            "peak_kind": peak_kind, "alg_bytes_per_batch": alg_bytes / args.steps,
            "basis": "whole batch solve time (every kernel of the solve, FP64 passes and launch gaps "
                     "included): a lower bound on the persistent inner kernel's own fraction"}
    # the oracle's residual of every 32nd mesh's solution (assembled on the host)
    check = None
    if not args.no_cpu_baseline:
        import oracle
        worst = 0.0
        for i in range(0, len(cases), 32):
            A = oracle.PressureMatrix.from_case(cases[i])
            worst = max(worst, A.residual(cases[i].b, xs[i].cpu().numpy()))
        check = {"meshes": len(range(0, len(cases), 32)), "max_rel_res_oracle": worst,
                 "note": "every 32nd mesh: the FP64 oracle's relative residual of the GPU solution"}
    out = {"workload": "c4_batch_%d_meshes" % args.meshes, "value": dof_iters / (tot / 1e3), "unit": UNIT,
           "steps": args.steps, "ms_per_batch": tot / args.steps, "p50_ms": _pctl(times, 50),
           "p99_ms": _pctl(times, 99), "solves_per_s": 1e3 * args.meshes * args.steps / tot,
           "n_free_total": int(sum(n_free)), "max_rel_res": max(inf.rel_res for inf in infos),
           "oracle_check": check,
           "iters_inner_mean": float(np.mean([inf.iters_inner for inf in infos])),
           "iters_inner_max": int(max(inf.iters_inner for inf in infos)),
           "chunk_elems": chunk, **knobs, "tuning": tune, "setup_s": setup_s, "gpu_launches": launches,
           "roofline": roof, "l2": "flushed between steps (256 MB write)", "clocks": clk}
    for m in meshes:
        P.ps_mesh_free(m)
    P.ps_ctx_destroy(ctx)
    return out


def run_batch(args):
    """c4 alone: one JSON line."""
    import contextlib
    import torch
    from __graft_entry__ import build
    with contextlib.redirect_stdout(sys.stderr):
        build()
    from paper_2301_08357_gb300 import pressure as P
    from paper_2301_08357_gb300 import synthetic as S
    from paper_2301_08357_gb300 import autotune
    r = bench_batch(args, P, S, autotune, torch)
    out = {"metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
           "warmup": max(args.warmup, 3), "ms_per_step": r["ms_per_batch"], "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
           "config": {"workload": r["workload"], "l2": r["l2"]}, "batched": r,
           "solves_per_s": r["solves_per_s"], "clocks": r["clocks"]}
    print(json.dumps(out))


SIZE_BUCKETS = ((0, 5e4, "< 50k nodes"), (5e4, 5e5, "50k-500k nodes"), (5e5, 1e12, ">= 500k nodes"))


def _buckets(lat_s, sizes):
    """p50/p99 latency (ms) per case-size bucket."""
    out = []
    lat_s, sizes = np.asarray(lat_s), np.asarray(sizes)
    for lo, hi, name in SIZE_BUCKETS:
        sel = (sizes >= lo) & (sizes < hi)
        if sel.any():
            out.append({"bucket": name, "requests": int(sel.sum()), "p50_ms": 1e3 * _pctl(lat_s[sel], 50),
                        "p99_ms": 1e3 * _pctl(lat_s[sel], 99)})
    return out


class _DriftAhead:
    """Each case's next time-step inputs (synthetic.served_step_drift from
    the case's current state), computed in a thread pool while the case's
    current request is in flight, so that generating the synthetic request
    stream (numpy over every element of every case) does not stall the
    requests.  One computation per case is outstanding at a time, so every
    case draws its seeded random stream in the same order as a sequential
    loop."""

    def __init__(self, S, cases, workers=8):
        import concurrent.futures as cf
        self.ex = cf.ThreadPoolExecutor(max_workers=workers)
        self.S, self.cases, self.fut = S, cases, {}

    def prime(self, ci, state):
        self.fut[ci] = self.ex.submit(self.S.served_step_drift, self.cases[ci], *state)

    def take(self, ci):
        return self.fut.pop(ci).result()

    def close(self):
        self.ex.shutdown(wait=True)


def bench_served(args, P, S, autotune, torch, rates=None, single_steps=None, budget_steps=None):
    """c5: time-step solves from simulated cases through the serving loop
    (continuous batching), closed loop with every case in flight; optionally
    Poisson arrivals at multiples of the closed-loop rate; the closed loop
    under an HBM budget that admits about a quarter of the workspaces; and the
    same requests solved one at a time (plain FP64 PCG and the mixed
    single-solve engine).  Returns a dict."""
    ctx = P.ps_ctx_create(0)
    meshes = []
    cases = [S.make_served_case(c, lo=5e3 * args.size_scale, hi=2e6 * args.size_scale, median=1e5 * args.size_scale)
             for c in range(args.cases)]
    chunk, knobs, tune = batch_tuning(args, autotune, P, ctx, cases)
    for cs in cases:
        m = P.ps_mesh_upload(ctx, cs.dim, cs.coords, cs.conn, cs.dirichlet, chunk_elems=chunk)
        P.ps_coeff_set(m, cs.alpha, cs.beta, cs.dt2)
        meshes.append(m)
    nodes_total = sum(c.n_nodes for c in cases)
    sizes = [c.n_nodes for c in cases]
    n_check = 4 if not args.no_cpu_baseline else 0
    check_cases = sorted(range(len(cases)), key=lambda c: sizes[c])[:n_check]   # the smallest cases

    def one_run(rate, budget=0, steps=None, single_nodes=0):
        """rate None = closed loop (each case submits its next step when the last completes);
        budget: the server's HBM cap on in-flight solver workspaces (0 = the context's);
        single_nodes: cases with at least this many nodes are served by the single-solve
        engine, one request at a time between epochs (0 = every request batched)."""
        steps = steps or args.case_steps
        srv = P.ps_server_create(ctx, max_slots=64, epoch_iters=32, hbm_budget_bytes=budget,
                                 opts=P.make_opts(tol=1e-10, **knobs), single_nodes=single_nodes)
        ids = [P.ps_server_add_case(srv, m) for m in meshes]
        state = [(c.beta.copy(), c.b.copy()) for c in cases]
        lat, qwait, req_size, done_iters, worst = [], [], [], 0, 0.0
        last_x = {}
        rng = np.random.default_rng(7)
        clocks = Clocks(0)
        if not args.no_clocks:
            clocks.start()
        ahead = _DriftAhead(S, cases)
        t_start = time.perf_counter()
        order = [(k, ci) for k in range(steps) for ci in range(len(cases))]
        pending = {}

        def finish(t, ci, k, polled=None):
            want_x = ci in check_cases and k + 1 == steps
            xo = np.empty(cases[ci].n_nodes) if want_x else None
            if polled is None:
                st, info = P.ps_solve_wait(srv, t, 600.0, x_out=xo)
            else:
                st, info = polled
                if want_x:
                    P.ps_solve_poll(srv, t, x_out=xo)
            P.ps_server_release(srv, t)
            if st != P.PS_OK:
                raise RuntimeError("served solve failed: %s" % P.ps_status_str(st))
            lat.append(info.seconds)
            qwait.append(info.queue_seconds)
            req_size.append(sizes[ci])
            if want_x:
                last_x[ci] = (xo, state[ci][0].copy(), state[ci][1].copy())
            return info

        if rate is None:
            # every case resubmits as soon as its request completes: all
            # pending tickets are polled, none is waited on in order
            for ci in range(len(cases)):
                pending[P.ps_solve_submit(srv, ids[ci], state[ci][1])] = (ci, 0)
                if steps > 1:
                    ahead.prime(ci, state[ci])
            while pending:
                progressed = False
                for t in list(pending):
                    polled = P.ps_solve_poll(srv, t)
                    if polled[0] == P.PS_PENDING:
                        continue
                    ci, k = pending.pop(t)
                    info = finish(t, ci, k, polled)
                    progressed = True
                    worst = max(worst, info.rel_res)
                    done_iters += cases[ci].n_free * (info.iters_inner + info.iters_outer)
                    if k + 1 < steps:
                        beta, b = ahead.take(ci)
                        state[ci] = (beta, b)
                        pending[P.ps_solve_submit(srv, ids[ci], b, beta)] = (ci, k + 1)
                        if k + 2 < steps:
                            ahead.prime(ci, state[ci])
                if not progressed:
                    time.sleep(0.0002)
        else:
            next_t = time.perf_counter()
            for ci in range(len(cases)):
                if steps > 1:
                    ahead.prime(ci, state[ci])
            for k, ci in order:
                next_t += rng.exponential(1.0 / rate)
                while time.perf_counter() < next_t:
                    time.sleep(min(0.001, max(0.0, next_t - time.perf_counter())))
                if k > 0:
                    state[ci] = ahead.take(ci)
                    if k + 1 < steps:
                        ahead.prime(ci, state[ci])
                beta = state[ci][0] if k > 0 else None
                pending[P.ps_solve_submit(srv, ids[ci], state[ci][1], beta)] = (ci, k)
            for t, (ci, k) in list(pending.items()):
                info = finish(t, ci, k)
                worst = max(worst, info.rel_res)
                done_iters += cases[ci].n_free * (info.iters_inner + info.iters_outer)
        wall = time.perf_counter() - t_start
        ahead.close()
        clk = clocks.stop() if not args.no_clocks else None
        stats = P.ps_server_get_stats(srv).as_dict()
        P.ps_server_destroy(srv)
        # the oracle's residual of the last step of the smallest cases, with that step's beta and b
        ocheck = None
        if last_x:
            import oracle
            ow = 0.0
            for ci, (xo, beta, b) in last_x.items():
                A = oracle.PressureMatrix.from_case(cases[ci], beta=beta)
                ow = max(ow, A.residual(b, xo))
            ocheck = {"cases": len(last_x), "max_rel_res_oracle": ow,
                      "note": "last step of the %d smallest cases, recomputed by the FP64 oracle" % len(last_x)}
        n = len(lat)
        return {"rate": rate, "single_nodes": single_nodes, "single_solves": stats["single_solves"],
                "solves": n, "steps_per_case": steps, "wall_s": wall, "solves_per_s": n / wall,
                "dof_iters_per_s": done_iters / wall, "p50_ms": 1e3 * _pctl(lat, 50), "p99_ms": 1e3 * _pctl(lat, 99),
                "per_bucket": _buckets(lat, req_size), "queue_p50_ms": 1e3 * _pctl(qwait, 50),
                "peak_in_flight": stats["peak_in_flight"], "epochs": stats["epochs"], "max_rel_res": worst,
                "oracle_check": ocheck, "clocks": clk}

    def single_run(mode, steps):
        """The same kind of requests (every case, `steps` steps, its drift
        continuing the case's seeded stream) solved one at a time through
        ps_pressure_solve (plain FP64 PCG or the mixed single-solve engine),
        each case warm-starting from its previous pressure."""
        opts = P.make_opts(mode=mode, tol=1e-10)
        lat, req_size, done_iters, worst = [], [], 0, 0.0
        xs = [torch.zeros(c.n_nodes, dtype=torch.float64, device="cuda") for c in cases]
        state = [(c.beta.copy(), c.b.copy()) for c in cases]
        clocks = Clocks(0)
        if not args.no_clocks:
            clocks.start()
        ahead = _DriftAhead(S, cases)
        t_start = time.perf_counter()
        for ci in range(len(cases)):
            if steps > 1:
                ahead.prime(ci, state[ci])
        for k in range(steps):
            for ci, c in enumerate(cases):
                if k > 0:
                    state[ci] = ahead.take(ci)
                    if k + 1 < steps:
                        ahead.prime(ci, state[ci])
                    P.ps_coeff_set_beta(meshes[ci], state[ci][0])
                t0 = time.perf_counter()
                b = torch.as_tensor(state[ci][1], device="cuda")
                st, info = P.ps_pressure_solve(meshes[ci], b, xs[ci], opts)
                torch.cuda.synchronize()
                lat.append(time.perf_counter() - t0)
                req_size.append(sizes[ci])
                worst = max(worst, info.rel_res)
                done_iters += c.n_free * (info.iters_inner + info.iters_outer)
        wall = time.perf_counter() - t_start
        ahead.close()
        clk = clocks.stop() if not args.no_clocks else None
        for ci, c in enumerate(cases):          # restore the case coefficients
            P.ps_coeff_set_beta(meshes[ci], c.beta)
        return {"mode": "fp64" if mode == P.PS_MODE_FP64 else "mixed", "solves": len(lat), "steps_per_case": steps,
                "wall_s": wall, "solves_per_s": len(lat) / wall, "dof_iters_per_s": done_iters / wall,
                "p50_ms": 1e3 * _pctl(lat, 50), "p99_ms": 1e3 * _pctl(lat, 99),
                "per_bucket": _buckets(lat, req_size), "max_rel_res": worst, "clocks": clk}

    # closed loop: every request batched, then the larger cases routed to the
    # single-solve engine (500k and 100k nodes and up); the configuration with
    # the highest throughput is the line's served figure and runs the rest
    closed = [one_run(None, single_nodes=t) for t in (0, 500000, 100000)]
    sat = max(closed, key=lambda r: r["solves_per_s"])
    route = sat["single_nodes"]
    runs = list(closed)
    for f in (rates or []):
        runs.append(dict(one_run(f * sat["solves_per_s"], single_nodes=route), rate_x_sat=f))
    # closed loop under an HBM budget that admits about a quarter of the cases'
    # workspaces at once (never less than the largest): admission queues requests
    ws_bytes = [P.ps_mesh_get_stats(m).solve_bytes for m in meshes]
    budget = int(max(max(ws_bytes), sum(ws_bytes) // 4))
    runs.append(dict(one_run(None, budget, steps=budget_steps, single_nodes=route), hbm_budget_bytes=budget,
                     workspace_bytes_total=int(sum(ws_bytes))))
    s_steps = single_steps or args.case_steps
    singles = [single_run(P.PS_MODE_FP64, s_steps), single_run(P.PS_MODE_MIXED, s_steps)]
    out = {"workload": "c5_served_%d_cases_x_%d_steps" % (args.cases, args.case_steps),
           "value": sat["dof_iters_per_s"], "unit": UNIT, "nodes_total": nodes_total,
           "case_nodes_min_max": [int(min(sizes)), int(max(sizes))],
           "solves_per_s": sat["solves_per_s"], "p50_ms": sat["p50_ms"], "p99_ms": sat["p99_ms"],
           "per_bucket": sat["per_bucket"], "max_rel_res": sat["max_rel_res"], "oracle_check": sat["oracle_check"],
           "served_vs_fp64_single_solves_per_s": sat["solves_per_s"] / singles[0]["solves_per_s"],
           "served_vs_mixed_single_solves_per_s": sat["solves_per_s"] / singles[1]["solves_per_s"],
           "single_nodes": route, "chunk_elems": chunk, **knobs, "tuning": tune, "runs": runs,
           "single_solves": singles,
           "clocks": sat["clocks"]}
    for m in meshes:
        P.ps_mesh_free(m)
    P.ps_ctx_destroy(ctx)
    return out


def run_served(args):
    """c5 alone (with the Poisson rate sweep): one JSON line."""
    import contextlib
    import torch
    from __graft_entry__ import build
    with contextlib.redirect_stdout(sys.stderr):
        build()
    from paper_2301_08357_gb300 import pressure as P
    from paper_2301_08357_gb300 import synthetic as S
    from paper_2301_08357_gb300 import autotune
    rates = [float(v) for v in args.rates.split(",") if v]
    r = bench_served(args, P, S, autotune, torch, rates=rates)
    out = {"metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": 1, "steps": args.case_steps,
           "warmup": 0, "ms_per_step": 1e3 / r["solves_per_s"], "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic", "config": {"workload": r["workload"]},
           "served": r, "solves_per_s": r["solves_per_s"], "p50_ms": r["p50_ms"], "p99_ms": r["p99_ms"],
           "clocks": r["clocks"]}
    print(json.dumps(out))


def bench_c2_sub(args, P, S, torch, steps):
    """The 64^3 single solve (mixed, x0 = 0), as a sub-object of the headline."""
    case = S.make_c2(64)
    ctx = P.ps_ctx_create(0)
    m = P.ps_mesh_upload(ctx, 3, case.coords, case.conn, case.dirichlet)
    P.ps_coeff_set(m, case.alpha, case.beta, case.dt2)
    stream = torch.cuda.current_stream()
    opts = P.make_opts(mode=P.PS_MODE_MIXED, tol=1e-10)
    b = torch.as_tensor(case.b, device="cuda")
    x = torch.zeros_like(b)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(3):
        x.zero_()
        P.ps_pressure_solve(m, b, x, opts, stream)
    times, iters = [], 0
    for k in range(steps):
        flush.fill_(k & 0xff)
        x.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st, info = P.ps_pressure_solve(m, b, x, opts, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
        iters += info.iters_inner + info.iters_outer
    stats = P.ps_mesh_get_stats(m)
    k1 = P.ps_profile_kernel(m, P.PS_KERNEL_CG1_F32 if case.n_nodes <= 200000 else P.PS_KERNEL_CG_F32, reps=50,
                             stream=stream)
    tot = float(np.sum(times))
    out = {"workload": workload_name(64), "value": case.n_free * iters / (tot / 1e3), "unit": UNIT,
           "ms_per_solve": tot / steps, "p50_ms": _pctl(times, 50), "iters_per_solve": iters // steps,
           "rel_res": info.rel_res, "operator_pass_ms": k1, "chunks": stats.n_chunks,
           "note": "the 64^3 system (41 MB per operator pass) is L2-resident between iterations"}
    P.ps_mesh_free(m)
    P.ps_ctx_destroy(ctx)
    return out


def run_headline(args):
    """The default line: the stiff 160^3 solve (mixed precision, warm start,
    b = A x* from the oracle), with the batched, served and c2 sub-objects."""
    import contextlib
    import torch

    ws, rank, local = dist_setup()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from __graft_entry__ import build
    if rank == 0 or ws == 1:
        with contextlib.redirect_stdout(sys.stderr):   # keep stdout to the one JSON line
            build()
    if ws > 1:
        torch.distributed.barrier()
    from paper_2301_08357_gb300 import pressure as P
    from paper_2301_08357_gb300 import synthetic as S
    from paper_2301_08357_gb300 import autotune

    case = S.make_c3(args.n or 160)
    ctx = P.ps_ctx_create(local)
    m = P.ps_mesh_upload(ctx, 3, case.coords, case.conn, case.dirichlet, chunk_elems=args.chunk,
                         pipeline=args.pipeline, operator_kernel=args.operator_kernel,
                         operator_threads=args.operator_threads)
    P.ps_coeff_set(m, case.alpha, case.beta, case.dt2)
    stats = P.ps_mesh_get_stats(m)
    stream = torch.cuda.current_stream()
    xs_h = case.extra["xstar"]
    use_oracle = ws == 1 and not args.no_cpu_baseline
    A, t_asm = None, None
    if use_oracle:
        # the oracle's b = A x* (so that x* is the solution of the oracle's system)
        import oracle
        t0 = time.perf_counter()
        A = oracle.PressureMatrix.from_case(case)
        t_asm = time.perf_counter() - t0
        b_h = A.apply(xs_h)
        b = torch.as_tensor(b_h, device="cuda")
    else:
        # replicas under torchrun: b from the library's FP64 operator on every rank
        xs_d = torch.as_tensor(xs_h, device="cuda")
        b = torch.empty_like(xs_d)
        P.ps_pressure_apply(m, xs_d, b, P.PS_F64, stream)
        torch.cuda.synchronize()
        b_h = b.cpu().numpy()
        del xs_d
    engine = {"auto": P.PS_ENGINE_AUTO, "graph": P.PS_ENGINE_GRAPH, "persistent": P.PS_ENGINE_PERSISTENT,
              "fused": P.PS_ENGINE_FUSED}[args.engine]
    opts = P.make_opts(mode=P.PS_MODE_MIXED, tol=1e-10, engine=engine)
    x0 = torch.as_tensor(case.x0, device="cuda")
    x = x0.clone()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def solve(o):
        x.copy_(x0)
        st, info = P.ps_pressure_solve(m, b, x, o, stream)
        if st != P.PS_OK:
            raise RuntimeError("solve failed: %s" % P.ps_status_str(st))
        return info

    for _ in range(max(args.warmup, 3)):
        solve(opts)
    torch.cuda.synchronize()
    clocks = Clocks(local)
    if not args.no_clocks:
        clocks.start()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    iters, launches = 0, 0
    for k in range(args.steps):
        flush.fill_(k & 0xff)          # L2 flush between steps (not timed)
        x.copy_(x0)
        ev[k][0].record(stream)
        st, info = P.ps_pressure_solve(m, b, x, opts, stream)
        ev[k][1].record(stream)
        if st != P.PS_OK:
            raise RuntimeError("solve failed: %s" % P.ps_status_str(st))
        iters += info.iters_inner + info.iters_outer
        launches += info.kernel_launches
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clk = clocks.stop() if not args.no_clocks else None
    step_ms = [a.elapsed_time(b_) for a, b_ in ev]
    total_ms = float(np.sum(step_ms))
    last = info
    x_h = x.cpu().numpy()
    t_max, tot_dof = aggregate(total_ms, case.n_free * iters, device="cuda")
    value = tot_dof / (t_max / 1e3)
    nx = np.linalg.norm(xs_h)
    accuracy = {"rel_res_gpu": last.rel_res,
                "rel_res_oracle": A.residual(b_h, x_h) if A is not None else None,
                "rel_err_vs_oracle": float(np.linalg.norm(x_h - xs_h) / nx) if A is not None else None,
                "rel_err_vs_xstar": float(np.linalg.norm(x_h - xs_h) / nx),
                "gates": "residual <= 1e-10 is the stop test; the error <= 1e-9 gate needs the tightened "
                         "tolerance on this stiff system (error <= kappa x residual), see 'tight'"}
    # the tolerance that meets both gates
    tight_opts = P.make_opts(mode=P.PS_MODE_MIXED, tol=args.tight_tol, max_outer=16, engine=engine)
    t_ms, t_it = [], 0
    for k in range(3):
        flush.fill_(k & 0xff)
        x.copy_(x0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st, ti = P.ps_pressure_solve(m, b, x, tight_opts, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        t_ms.append(e0.elapsed_time(e1))
        t_it += ti.iters_inner + ti.iters_outer
    xt = x.cpu().numpy()
    tight = {"tol": args.tight_tol, "ms_per_solve": float(np.mean(t_ms)), "iters_per_solve": t_it // 3,
             "status": P.ps_status_str(st), "rel_res_gpu": ti.rel_res,
             "rel_res_oracle": A.residual(b_h, xt) if A is not None else None,
             "rel_err_vs_oracle": float(np.linalg.norm(xt - xs_h) / nx) if A is not None else None,
             "solves_per_s": 1e3 / float(np.mean(t_ms))}

    # ---- end to end through the C ABI with host buffers (copies timed)
    b_pin = torch.as_tensor(b_h).pin_memory()
    x0_pin = torch.as_tensor(case.x0).pin_memory()
    x_pin = torch.empty_like(x0_pin).pin_memory()
    e2e_ms, e2e_it = [], 0
    for k in range(args.steps):
        flush.fill_(k & 0xff)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b.copy_(b_pin, non_blocking=True)
        x.copy_(x0_pin, non_blocking=True)
        st, ei = P.ps_pressure_solve(m, b, x, opts, stream)
        x_pin.copy_(x, non_blocking=True)
        torch.cuda.synchronize()
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
        e2e_it += ei.iters_inner + ei.iters_outer
    e2e_val = case.n_free * e2e_it / (np.sum(e2e_ms) / 1e3)

    # ---- roofline of the dominant kernels
    roof = kernel_roofline(P, m, stats, P.PS_MODE_MIXED, False, stream, c3_name(case))
    ipi = (last.iters_inner + last.iters_outer)
    roof["in_solve_check"] = {
        "solve_ms_per_iteration": total_ms / args.steps / max(ipi, 1),
        "isolated_iteration_kernels_ms": roof["kernel_ms"] + roof["update"]["kernel_ms"] +
                                          (roof["other_kernels_ms"]["halo_f32"] if stats.operator_kernel == 2 else 0.0),
        "note": "kernel_ms is the mean of back-to-back launches of the kernel alone; the solve's time per "
                "iteration also holds the outer FP64 passes and graph launch gaps"}
    P.ps_mesh_free(m)
    P.ps_ctx_destroy(ctx)
    del x, x0, b, flush
    torch.cuda.empty_cache()

    cpu = None
    if rank == 0 and use_oracle:
        import oracle
        cb = oracle_pcg_sample(A, b_h, case.x0, args.cpu_seconds)
        cpu = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")}
        n_all = oracle.num_threads()
        oracle.set_threads(1)
        try:
            c1 = oracle_pcg_sample(A, b_h, case.x0, calls=1)
        finally:
            oracle.set_threads(n_all)
        cpu["single_core"] = {"value": c1["value"], "unit": UNIT, "cores": 1, "sample": c1["sample"]}
        cpu["cpu_model"] = cpu_model()
        cpu["assembly_s"] = t_asm
    del A

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": max(args.warmup, 3), "ms_per_step": t_max / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
           "config": headline_config(case, ws),
           "solves_per_s": 1e3 * args.steps / t_max * ws,
           "p50_ms": _pctl(step_ms, 50), "p99_ms": _pctl(step_ms, 99),
           "solve": {"iters_per_solve": ipi, "outer_per_solve": last.iters_outer, "chunks": stats.n_chunks},
           "accuracy": accuracy, "tight": tight,
           "roofline": roof, "cpu_baseline": cpu,
           "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": 16 * case.n_nodes,
                   "d2h_bytes_per_step": 8 * case.n_nodes, "ms_per_step": float(np.mean(e2e_ms))},
           "gpu_launches": launches, "clocks": clk}
    if ws == 1 and not args.no_sub:
        out["c2"] = bench_c2_sub(args, P, S, torch, args.steps)
        out["batched"] = bench_batch(args, P, S, autotune, torch)
        out["served"] = bench_served(args, P, S, autotune, torch)
    if rank == 0:
        print(json.dumps(out))
    if ws > 1:
        torch.distributed.destroy_process_group()


def run_projection(args, eos=False):
    """One time step's projection stage (ps_projection_step) on the 3D Kuhn cube
    n^3 with seeded flow fields: first guesses, 2 Picard iterations of [operator
    update, right-hand side, mixed-precision solve to 1e-10, post-projection].
    Every step starts from dP = 0 (the same work each step).
    eos: the general-EOS step instead (ps_projection_step_eos, rho e =
    2.5 P + 0.5 P^2 / rho, lumped mass, Newton to ||F|| <= 1e-8 ||c|| with
    mixed-precision solves to 1e-10 inside each Picard iteration)."""
    import contextlib
    import torch
    from __graft_entry__ import build
    with contextlib.redirect_stdout(sys.stderr):
        build()
    from paper_2301_08357_gb300 import pressure as P
    from paper_2301_08357_gb300 import synthetic as S
    n_pic = 2
    args.n = args.n or 64
    case = S.make_eos_case(3, args.n) if eos else S.make_projection_case(3, args.n)
    e = case.extra
    ctx = P.ps_ctx_create(0)
    m = P.ps_mesh_upload(ctx, 3, case.coords, case.conn, case.dirichlet, chunk_elems=args.chunk)
    P.ps_coeff_set(m, case.alpha, case.beta, case.dt2)
    if eos:
        P.ps_mesh_set_mass(m, P.PS_MASS_LUMPED)
    n_checks = [0]
    stream = torch.cuda.current_stream()
    N, E = case.n_nodes, case.n_elems
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")
    ins = [dev(e["rho"]), dev(e["wu"]), dev(e["we"]), dev(e["pn"])]
    dp = torch.zeros(N, dtype=torch.float64, device="cuda")
    outs = [torch.empty(N, dtype=torch.float64, device="cuda"), torch.empty(E * 3, dtype=torch.float64, device="cuda"),
            torch.empty(E, dtype=torch.float64, device="cuda"), torch.empty(E, dtype=torch.float64, device="cuda")]
    opts = P.make_opts(tol=1e-10)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def step():
        dp.zero_()
        if eos:
            st, info, res = P.ps_projection_step_eos(m, *ins, dp, *outs, eos_a=e["eos_a"], eos_b=e["eos_b"],
                                                     dt=e["dt"], n_picard=n_pic, max_newton=8, newton_tol=1e-8,
                                                     solve_opts=opts, stream=stream)
            n_checks[0] = int((res >= 0).sum())
            return st, info
        return P.ps_projection_step(m, *ins, dp, *outs, gamma=e["gamma"], dt=e["dt"], n_picard=n_pic,
                                    solve_opts=opts, stream=stream)

    for _ in range(max(args.warmup, 3)):
        step()
    clocks = Clocks(0)
    if not args.no_clocks:
        clocks.start()
    times, iters, launches = [], 0, 0
    for k in range(args.steps):
        flush.fill_(k & 0xff)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st, info = step()
        e1.record(stream)
        torch.cuda.synchronize()
        if st != P.PS_OK:
            raise RuntimeError("projection step failed: %s" % P.ps_status_str(st))
        times.append(e0.elapsed_time(e1))
        iters += info.iters_inner + info.iters_outer
        if eos:
            # solve launches + first guess, weights (3), final alpha + diagonal (3) + per Picard
            # iteration: check, beta, right-hand side (2), post (2), diagonal (2) + per Newton check:
            # linearise, alpha, FP64 apply (4), norms
            launches += info.kernel_launches + 7 + 8 * n_pic + 7 * n_checks[0]
        else:
            # solve launches + per Picard iteration: check, beta, diagonal (2), right-hand side (2),
            # post (2); + first guess
            launches += info.kernel_launches + 7 * n_pic + 1
    clk = clocks.stop() if not args.no_clocks else None
    tot = float(np.sum(times))
    wname = ("eos_3d_kuhn_%d" if eos else "projection_3d_kuhn_%d") % args.n
    if args.launch_list:
        # warm-up and timed steps only (identical work), for a launch-list capture
        print(json.dumps({"metric": METRIC, "value": case.n_free * iters / (tot / 1e3), "unit": UNIT,
                          "ms_per_step": tot / args.steps, "config": {"workload": wname},
                          "gpu_launches": launches, "launch_list_run": True}))
        P.ps_mesh_free(m)
        P.ps_ctx_destroy(ctx)
        return
    # end to end: host inputs copied in, outputs copied back, inside the timed region
    h_in = [torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64)).pin_memory()
            for a in (e["rho"], e["wu"], e["we"], e["pn"])]
    h_out = [torch.empty(o.numel(), dtype=torch.float64).pin_memory() for o in [dp] + outs]
    e2e = []
    for k in range(args.steps):
        flush.fill_(k & 0xff)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for d_, h_ in zip(ins, h_in):
            d_.copy_(h_, non_blocking=True)
        step()
        for h_, d_ in zip(h_out, [dp] + outs):
            h_.copy_(d_, non_blocking=True)
        torch.cuda.synchronize()
        e2e.append(1e3 * (time.perf_counter() - t0))
    stats = P.ps_mesh_get_stats(m)
    roof = kernel_roofline(P, m, stats, P.PS_MODE_MIXED, case.n_nodes <= 200000, stream, wname, lumped=eos)
    cpu = None
    if not args.no_cpu_baseline and eos:
        from oracle import lumped as LO
        import oracle
        n_s = min(args.n, 24)
        cs = S.make_eos_case(3, n_s)
        es = cs.extra
        t0 = time.perf_counter()
        LO.projection_step_eos(3, cs.coords, cs.conn, cs.dirichlet, es["rho"], es["wu"], es["we"], es["pn"],
                               es["eos_a"], es["eos_b"], es["dt"], n_pic, 8, tol=1e-8)
        t_cpu = time.perf_counter() - t0
        cpu = {"value": 1.0 / t_cpu, "unit": "steps/s (%d^3 sample)" % n_s, "cores": oracle.num_threads(),
               "kind": "oracle",
               "sample": "one general-EOS projection step on the %d^3 Kuhn cube (%d free nodes; 2 Picard "
                         "iterations, Newton with SciPy direct sparse solves), %.2f s; not in DOF-it/s: the "
                         "oracle solves directly" % (n_s, cs.n_free, t_cpu)}
    elif not args.no_cpu_baseline:
        from oracle import projection as PJ
        t0 = time.perf_counter()
        ref = PJ.projection_step(3, case.coords, case.conn, case.dirichlet, case.alpha, e["rho"], e["wu"], e["we"],
                                 e["pn"], e["gamma"], e["dt"], n_pic, tol=1e-10)
        t_cpu = time.perf_counter() - t0
        it_cpu = sum(s_["iters"] for s_ in ref["solves"])
        import oracle
        cpu = {"value": case.n_free * it_cpu / t_cpu, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
               "sample": "one full projection step (2 Picard iterations, NumPy right-hand side and updates, "
                         "C Jacobi-PCG to 1e-10), %.1f s" % t_cpu}
    bytes_in = 8 * (E * 5 + N)
    bytes_out = 8 * (2 * N + 5 * E)
    out = {"metric": METRIC, "value": case.n_free * iters / (tot / 1e3), "unit": UNIT, "n_gpus": 1,
           "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": tot / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
           "data": "synthetic",
           "config": {"workload": "%s^3_picard%d" % (wname, n_pic), "n_free": case.n_free,
                      "n_elems": E, "iters_per_step": iters // max(args.steps, 1), "dt": e["dt"],
                      "l2": "flushed between steps (256 MB write)",
                      **({"eos": "rho e = %g P + %g P^2/rho" % (e["eos_a"], e["eos_b"]), "mass": "lumped",
                          "newton_checks_per_step": n_checks[0]} if eos else {"gamma": e["gamma"]})},
           "steps_per_s": 1e3 * args.steps / tot, "p50_ms": _pctl(times, 50), "p99_ms": _pctl(times, 99),
           "roofline": roof, "cpu_baseline": cpu,
           "e2e": {"value": case.n_free * iters / (np.sum(e2e) / 1e3), "unit": UNIT, "h2d_bytes_per_step": bytes_in,
                   "d2h_bytes_per_step": bytes_out, "ms_per_step": float(np.mean(e2e))},
           "gpu_launches": launches, "clocks": clk}
    print(json.dumps(out))
    P.ps_mesh_free(m)
    P.ps_ctx_destroy(ctx)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "headline":
        run_headline(args)
    elif args.workload in ("c1", "c3", "periodic"):
        run_single(args, args.workload)
    elif args.workload == "c4":
        run_batch(args)
    elif args.workload == "c5":
        run_served(args)
    elif args.workload == "projection":
        run_projection(args)
    elif args.workload == "eos":
        run_projection(args, eos=True)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
