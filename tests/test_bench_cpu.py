"""Host-side logic of bench.py that needs no GPU: the whole-job aggregation
over ranks (world_size 2 over gloo on CPU: max time, summed work), the
reference arm's rank > 0 behaviour, the clock-sample parser, and the served
bench's request stream prepared ahead in a thread pool."""
import os
import socket

import numpy as np
import pytest

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t, w = bench.aggregate(10.0 + 5 * rank, 100 * (rank + 1))
    q.put((rank, t, w))
    dist.destroy_process_group()


def test_aggregate_two_ranks_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, t, w in res:
        assert t == 15.0          # max over ranks
        assert w == 300.0         # sum over ranks


def test_aggregate_single_process_is_identity():
    assert bench.aggregate(3.5, 7) == (3.5, 7.0)


def test_reference_arm_rank1_exits_without_output(capsys, monkeypatch):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = type("A", (), {"n": 4, "steps": 1, "warmup": 0, "gpus": 2})()
    bench.run_reference(args)
    assert capsys.readouterr().out == ""


def test_reference_arm_rank0_prints_one_json_line(capsys, monkeypatch):
    import json
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("WORLD_SIZE", "1")
    args = type("A", (), {"n": 6, "steps": 2, "warmup": 0, "gpus": 1})()
    bench.run_reference(args)
    out = capsys.readouterr().out.strip().splitlines()
    assert len(out) == 1
    d = json.loads(out[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == bench.UNIT
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
    # the reference arm describes the headline workload with the main arm's config
    from paper_2301_08357_gb300 import synthetic as S
    assert d["config"] == bench.headline_config(S.make_c3(6))
    assert d["config"]["workload"].startswith("c3_3d_kuhn_6^3")


def test_clock_parser():
    lines = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
             "0, 1965, 2070, 1300.0, 0x4, Not Active, Not Active, Not Active, Active",
             "0, 2070, 2070, 1100.0, 0x0, Not Active, Not Active, Not Active, Not Active",
             "garbage line"]
    c = bench.parse_clocks(lines)
    assert c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"] and c["samples"] == 3
    assert bench.parse_clocks([]) is None


def test_fp64_flop_model():
    """The FP64 roofline's peak and per-pass flop count (C2: 1,572,864 tets,
    274,625 nodes; 74 flops per consistent tet, 36 per lumped tet)."""
    class St:
        n_elems, n_nodes, dim = 1572864, 274625, 3
    assert abs(bench.FP64_PEAK_TFLOPS - 152 * 4 * 2.07e-3) < 1e-12
    inc = St.n_elems * 4 / St.n_nodes
    assert bench.fp64_flops(St, False, False) == pytest.approx(74 * St.n_elems + (inc + 3) * St.n_nodes)
    assert bench.fp64_flops(St, True, True) == pytest.approx(36 * St.n_elems + (inc + 4) * St.n_nodes)

    class St2:
        n_elems, n_nodes, dim = 8192, 4225, 2
    assert bench.fp64_flops(St2, False, False) == pytest.approx(50 * 8192 + (8192 * 3 / 4225 + 3) * 4225)


def test_drift_ahead_matches_the_sequential_stream():
    """The served bench prepares each case's next request in a thread pool
    while the current one is in flight; every case must still draw its
    seeded random stream in the order of a plain sequential loop."""
    from paper_2301_08357_gb300 import synthetic as S
    steps = 4
    seq_cases = [S.make_served_case(c, lo=1e3, hi=4e3, median=2e3) for c in range(3)]
    seq = []
    for c in seq_cases:
        st, out = (c.beta.copy(), c.b.copy()), []
        for _ in range(steps - 1):
            st = S.served_step_drift(c, *st)
            out.append(st)
        seq.append(out)
    cases = [S.make_served_case(c, lo=1e3, hi=4e3, median=2e3) for c in range(3)]
    ahead = bench._DriftAhead(S, cases, workers=3)
    state = [(c.beta.copy(), c.b.copy()) for c in cases]
    got = [[] for _ in cases]
    for ci in range(len(cases)):
        ahead.prime(ci, state[ci])
    for k in range(1, steps):                # cases finishing in a shuffled order each step
        for ci in ([2, 0, 1] if k % 2 else [1, 2, 0]):
            state[ci] = ahead.take(ci)
            got[ci].append(state[ci])
            if k + 1 < steps:
                ahead.prime(ci, state[ci])
    ahead.close()
    for a, b in zip(seq, got):
        for (beta1, b1), (beta2, b2) in zip(a, b):
            assert np.array_equal(beta1, beta2) and np.array_equal(b1, b2)
