"""The N > 1 launch path on the CPU: two gloo ranks, each with its own copy of the work,
reduce only their timings (MAX) -- the path itself needs no exchange."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, ms, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    value, total_ms, w = bench.whole_job(1_000_000, 4, ms[rank], dist, "cpu")
    out[rank] = (value, total_ms, w)
    dist.destroy_process_group()


def test_weak_scaling_reduction_two_ranks():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    ms = [10.0, 25.0]
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, ms, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        value, total_ms, w = out[r]
        assert w == 2 and total_ms == 25.0                 # the slowest rank sets the time
        assert value == pytest.approx(1_000_000 * 4 * 2 / 0.025)


def test_single_rank_without_process_group():
    value, total_ms, w = bench.whole_job(10, 3, 2.0)
    assert w == 1 and total_ms == 2.0 and value == pytest.approx(15000.0)


def test_clock_summary_keeps_the_timed_window():
    """Samples outside the timed region are dropped; throttle reasons inside it are kept."""
    c = bench.ClockSampler(0)
    row = lambda mhz, cap: [str(mhz), "2070", "900", "Not Active", "Not Active", "Not Active", cap]
    c.rows = [(0.0, row(1000, "Not Active")), (1.0, row(2070, "Active")),
              (1.1, row(2060, "Not Active")), (2.0, row(500, "Not Active"))]
    c.mark(0.9, 1.2)
    s = c.summary()
    assert s["samples"] == 2 and s["sm_mhz"] == 2065.0 and s["reasons"] == ["sw_power_cap"]
    assert s["window"] == "inside the timed region"
    c.mark(1.5, 1.6)                       # no sample inside: the two nearest, labelled so
    s = c.summary()
    assert s["samples"] == 2 and s["window"].startswith("nearest")
