"""Host-side logic of bench.py that needs no GPU: the whole-job aggregation
over ranks (world_size 2 over gloo on CPU: max time, summed work), the
reference arm's rank > 0 behaviour, and the clock-sample parser."""
import os
import socket

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
