"""Host-side logic of bench.py on CPU: the replicas-only multi-process timing (gloo, world
size 2) and the roofline arithmetic."""
import json
import math
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r "took" 0.1 + 0.05 r seconds for 7296 slice-steps of its own problem
    t = bench.slowest_rank(0.1 + 0.05 * rank, world)
    q.put((rank, t, world * 7296 / t))
    dist.destroy_process_group()


def test_replicas_take_the_slowest_rank_gloo():
    pytest.importorskip("torch")
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, v in out:
        assert t == pytest.approx(0.15)                    # max over ranks, seen by every rank
        assert v == pytest.approx(2 * 7296 / 0.15)         # whole-job throughput


def test_single_process_needs_no_process_group():
    import bench
    assert bench.slowest_rank(0.25, 1) == 0.25


def test_roofline_arithmetic():
    import bench
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    # {name: (launches, total ms, flops, bytes)}
    stats = {"ring_nl_f32": (10, 10.0, 0.0, 10 * 906e6), "nl_pre": (10, 1.0, 0.0, 10 * 300e6),
             "leg_fwd_tc": (10, 4.0, 10 * 4.04e9, 10 * 258e6)}
    r = bench.roofline(stats)
    assert r["kernel"] == "ring_nl_f32" and r["bound"] == "hbm"
    assert r["achieved"] == pytest.approx(906e6 / 1e-3 / 1e9)          # 906 MB per 1 ms launch
    assert r["frac"] == pytest.approx(r["achieved"] / peaks["hbm_gbs"])
    ratio = bench.NCU_TRAFFIC_RATIO["ring_nl_f32"][0]
    assert r["traffic"]["bytes_per_launch"] == pytest.approx(ratio * 906e6)
    assert math.isclose(sum(k["share_of_timed"] for k in r["kernels"].values()), 1.0)
    # a tensor-core kernel dominating: six bf16 products per useful flop against the sustained peak
    r2 = bench.roofline({"leg_fwd_tc": (4, 4.0, 4 * 4.04e9, 4 * 258e6)})
    assert r2["bound"] == "tensor"
    assert r2["achieved"] == pytest.approx(6 * 4.04e9 / 1e-3 / 1e12)
    assert r2["frac"] == pytest.approx(r2["achieved"] / peaks["bf16_tflops_sustained"])
