"""The N > 1 path on the CPU: gloo ranks split the points and the dose targets, compute
their shares, and one all-gather reassembles the outputs (the compute here is the CPU
oracle, standing in for each rank's GPU: what is tested is the partition, the gather and
the whole-job timing reduction)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import bench
from paper_2507_00294_gb300 import shard
from paper_2507_00294_gb300 import workloads as w


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _timing_rank(rank, world, port, ms, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    value, total_ms, wsz = bench.whole_job(1_000_000, 4, ms[rank], dist, "cpu")
    out[rank] = (value, total_ms, wsz)
    dist.destroy_process_group()


def _spawn(target, world, *args):
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=target, args=(r, world, port) + args + (out,)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(180)
        assert p.exitcode == 0
    return dict(out)


def test_strong_scaling_reduction_two_ranks():
    out = _spawn(_timing_rank, 2, [10.0, 25.0])
    for r in range(2):
        value, total_ms, wsz = out[r]
        assert wsz == 2 and total_ms == 25.0                 # the slowest rank sets the time
        assert value == pytest.approx(1_000_000 * 4 / 0.025)  # the whole job's work, once


def test_single_rank_without_process_group():
    value, total_ms, wsz = bench.whole_job(10, 3, 2.0)
    assert wsz == 1 and total_ms == 2.0 and value == pytest.approx(15000.0)


SPLIT_SPEC = dict(nx=7, ny=6, order=w.SERPENTINE)
SPLIT_POINTS = 1300                    # three point tiles of 512: a ragged last tile
SPLIT_TIMES = (9.5e-6, 30e-6, 42e-6, 80e-6)


def _oracle_problem():
    import sys
    sys.path.insert(0, os.path.dirname(__file__))
    from parity_util import oracle_problem
    spec = w.ScanSpec(**SPLIT_SPEC)
    rng = np.random.default_rng(9)
    pts = np.column_stack([rng.uniform(-1e-9, 4e-9, SPLIT_POINTS), rng.uniform(-1e-9, 3.5e-9, SPLIT_POINTS)])
    return spec, pts, oracle_problem(spec)


def _split_rank(rank, world, port, out):
    import torch.distributed as dist
    import oracle
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    spec, pts, (src, Ds, D, Q0) = _oracle_problem()
    tt = np.asarray(SPLIT_TIMES) / spec.dwell_s

    def field_fn(p0, p1):
        return torch.from_numpy(oracle.field(src, Ds, D, Q0, pts[p0:p1, 0], pts[p0:p1, 1], tt, threads=1))

    def dose_fn(j0, j1):
        return torch.from_numpy(oracle.dose(src, Ds, D, Q0, targets=np.arange(j0, j1), threads=1))

    field, dose = shard.field_and_dose(rank, world, len(pts), src.n, field_fn, dose_fn, dist)
    out[rank] = (field.numpy(), dose.numpy())
    dist.destroy_process_group()


def _grid_split_rank(rank, world, port, out):
    import torch.distributed as dist
    import oracle
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    spec, pts, (src, Ds, D, Q0) = _oracle_problem()
    tt = np.asarray(SPLIT_TIMES) / spec.dwell_s
    costs = [int(np.searchsorted(src.ts, t, side="left")) * len(pts) for t in tt]

    def field_fn(snaps):
        if not snaps:
            return torch.zeros((0, len(pts)), dtype=torch.float64)
        return torch.from_numpy(oracle.field(src, Ds, D, Q0, pts[:, 0], pts[:, 1], tt[snaps], threads=1))

    def dose_fn(j0, j1):
        return torch.from_numpy(oracle.dose(src, Ds, D, Q0, targets=np.arange(j0, j1), threads=1))

    field, dose = shard.grid_field_and_dose(rank, world, costs, src.n, field_fn, dose_fn, dist)
    out[rank] = (field.numpy(), dose.numpy())
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3, 5])
def test_snapshot_split_gathered_equals_one_rank(world):
    """The grid form of the split: every rank keeps all points and takes a set of the
    snapshots; the rows gathered back in snapshot order equal the one-rank field bit for
    bit on every rank (and the dose as in the point split).  Five ranks for four
    snapshots: one rank takes none and still joins the gather."""
    import oracle
    spec, pts, (src, Ds, D, Q0) = _oracle_problem()
    tt = np.asarray(SPLIT_TIMES) / spec.dwell_s
    whole_f = oracle.field(src, Ds, D, Q0, pts[:, 0], pts[:, 1], tt)
    whole_d = oracle.dose(src, Ds, D, Q0)
    out = _spawn(_grid_split_rank, world)
    for r in range(world):
        f, d = out[r]
        assert f.shape == whole_f.shape and d.shape == whole_d.shape
        assert np.array_equal(f, whole_f) and np.array_equal(d, whole_d)


def test_snapshot_sets_partition_and_balance():
    costs = [64 * (j + 1) * 16384 for j in range(64)]          # the bench's row snapshots
    for world in (1, 2, 3, 4, 8, 64, 70):
        sets = shard.snapshot_sets(costs, world)
        assert len(sets) == world
        assert sorted(j for x in sets for j in x) == list(range(len(costs)))
        assert all(x == sorted(x) for x in sets)
        if world <= 8:
            load = [sum(costs[j] for j in x) for x in sets]
            assert max(load) <= 1.02 * sum(costs) / world


@pytest.mark.parametrize("world", [2, 3])
def test_split_field_and_dose_gathered_equals_one_rank(world):
    """Every rank holds the gathered field and dose, bit for bit equal to the one-rank
    evaluation of the whole job."""
    import oracle
    spec, pts, (src, Ds, D, Q0) = _oracle_problem()
    tt = np.asarray(SPLIT_TIMES) / spec.dwell_s
    whole_f = oracle.field(src, Ds, D, Q0, pts[:, 0], pts[:, 1], tt)
    whole_d = oracle.dose(src, Ds, D, Q0)
    out = _spawn(_split_rank, world)
    for r in range(world):
        f, d = out[r]
        assert f.shape == whole_f.shape and d.shape == whole_d.shape
        assert np.array_equal(f, whole_f) and np.array_equal(d, whole_d)


def test_point_and_dose_ranges_partition_and_balance():
    for n_pts in (1, 511, 512, 16384, 1_000_003):
        for world in (1, 2, 3, 8):
            pr = shard.point_ranges(n_pts, world)
            assert pr[0][0] == 0 and pr[-1][1] == n_pts
            assert all(a[1] == b[0] for a, b in zip(pr, pr[1:]))          # contiguous, disjoint
            assert all(p0 % shard.POINT_TILE == 0 for p0, _ in pr)       # whole tiles
            tiles = [(p1 - p0 + 511) // 512 for p0, p1 in pr]
            assert max(tiles) - min(tiles) <= 1
    for n in (2, 4096, 65536):
        for world in (2, 4, 8):
            dr = shard.dose_ranges(n, world)
            assert dr[0][0] == 0 and dr[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(dr, dr[1:]))
            work = [(j1 * (j1 - 1) - j0 * (j0 - 1)) / 2 for j0, j1 in dr]   # sum of j over the range
            if n >= 4096 * world // 2:
                assert max(work) <= 1.25 * sum(work) / world


def test_lpt_assignment_balances_uneven_scans():
    costs = [w.n_visits(s) * s.nx * s.nx for s in w.batched_specs(512, seed=4)]
    for world in (2, 4, 8):
        parts = shard.lpt_assign(costs, world)
        assert sorted(k for p in parts for k in p) == list(range(len(costs)))
        load = [sum(costs[k] for k in p) for p in parts]
        # LPT is within 4/3 of the optimum; the optimum is at least the mean and the largest job
        bound = max(sum(costs) / world, max(costs))
        assert max(load) <= 4 / 3 * bound


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
