"""Batches of scans evaluated on grids of points (dd_batch_create_grid: grid tiles of
32 x 32 points with the separable degree-2 form in FP32-mixed) against the oracle and
against the same points given as lists."""
import numpy as np
import pytest

from paper_2507_00294_gb300 import binding as b
from paper_2507_00294_gb300 import workloads as w
from parity_util import assert_fp64, assert_mixed, oracle_field, oracle_pairs

pytestmark = pytest.mark.gpu


def grid_pts(g):
    x0, y0, dx, dy, nc, nr = g
    c = np.arange(int(nc), dtype=np.float64) * dx + x0
    r = np.arange(int(nr), dtype=np.float64) * dy + y0
    yy, xx = np.meshgrid(r, c, indexing="ij")
    return np.stack([xx.reshape(-1), yy.reshape(-1)], axis=1)


def uneven_grid_batch(seed=5, n_scans=16):
    """Scans of the batched workload's kinds at small sizes, each on its own grid: the
    probe grid, ragged sizes (not multiples of 32), a grid off the probe lattice (pitch/3,
    shifted origin), a negative spacing, an empty grid, and snapshots during and after."""
    rng = np.random.default_rng(seed)
    specs, grids, times = [], [], []
    for k in range(n_scans):
        n = int(rng.integers(5, 40))
        s = w.ScanSpec(n, n, D_m2s=float(10 ** rng.uniform(-15, -12)), dwell_s=float(10 ** rng.uniform(-7, -5)),
                       sigma_m=float(rng.uniform(0.05e-9, 0.2e-9)), order=w.RANDOM, seed=k,
                       keep_fraction=float(rng.uniform(0.2, 1.0)))
        p = s.pitch_m
        kind = k % 5
        if kind == 0:
            g = (0.0, 0.0, p, p, n, n)
        elif kind == 1:
            g = (0.0, 0.0, p / 2, p / 2, 2 * n + 3, n + 7)
        elif kind == 2:
            g = (-0.37 * p, 0.21 * p, p / 3, p / 3, 40, 35)
        elif kind == 3:
            g = ((n - 1) * p, 0.0, -p, p, n, 33)
        else:
            g = (0.0, 0.0, p, p, 0 if k == 4 else 3, 5)
        nv = w.n_visits(s)
        specs.append(s)
        grids.append(g)
        times.append([nv * s.dwell_s, (0.4 * nv + 0.5) * s.dwell_s, 3.0 * nv * s.dwell_s][k % 3])
    return specs, grids, np.array(times)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_uneven_grid_batch_full(cuda, prec):
    specs, grids, times = uneven_grid_batch()
    scans = [b.Scan(s) for s in specs]
    plan = b.Batch(scans, None, times, prec, grids=grids)
    out = plan.run(device=cuda).cpu().numpy()
    again = plan.run(device=cuda).cpu().numpy()          # graph replay
    np.testing.assert_array_equal(out, again)
    host = plan.run(out=np.empty(plan.total))            # host output
    np.testing.assert_array_equal(out, host)
    for k, (s, g) in enumerate(zip(specs, grids)):
        got = out[plan.offsets[k]:plan.offsets[k + 1]]
        pts = grid_pts(g)
        assert len(got) == len(pts)
        if len(pts) == 0:
            continue
        ref = oracle_field(s, pts, times[k:k + 1])[0]
        if prec == "fp64":
            assert_fp64(got, ref, "grid batch scan %d" % k)
        else:
            assert_mixed(got, ref, ref.max(), "grid batch scan %d" % k)


def test_batched_512_scans_grid_against_point_list_and_oracle(cuda):
    """The 512-scan workload on each scan's probe grid: the grid plan (32 x 32 tiles,
    separable form) within the mixed tolerance of the point-list plan everywhere, and
    against the oracle on 4 seeded points of 48 scans."""
    import torch
    jobs = w.batched_scans()
    scans = [b.Scan(j.scan) for j in jobs]
    times = np.array([j.times[0] for j in jobs])
    grids = [(0.0, 0.0, j.scan.pitch_m, j.scan.pitch_m, j.scan.nx, j.scan.ny) for j in jobs]
    for j, g in zip(jobs, grids):
        assert np.array_equal(grid_pts(g), j.pts_xy)
    gplan = b.Batch(scans, None, times, "mixed", grids=grids)
    gout = gplan.run(device=cuda).cpu().numpy()
    offs = np.concatenate([[0], np.cumsum([len(j.pts_xy) for j in jobs])]).astype(np.int64)
    lplan = b.Batch(scans, offs, times, "mixed")
    lout = lplan.run(torch.from_numpy(np.concatenate([j.pts_xy for j in jobs])).cuda()).cpu().numpy()
    assert np.array_equal(gplan.offsets, offs)
    m = lout > 1e-6 * np.repeat([lout[offs[k]:offs[k + 1]].max() for k in range(len(jobs))], np.diff(offs))
    # two FP32-mixed evaluations, each within the mixed tolerance of the exact field
    assert np.max(np.abs(gout[m] / lout[m] - 1.0)) <= 1e-5
    rng = np.random.default_rng(8)
    for k in rng.choice(len(jobs), 48, replace=False):
        j = jobs[k]
        ip = rng.integers(0, len(j.pts_xy), 4)
        ref = oracle_pairs(j.scan, j.pts_xy, j.times, ip, np.zeros(4, int))
        got = gout[offs[k]:offs[k + 1]][ip]
        assert_mixed(got, ref, ref.max(), "grid 512 scan %d" % k)


def test_grid_batch_tensor_core_part(cuda):
    """Scans whose grids reach 64 x 64 points, where the plan sums each scan's older visits
    on the tensor cores (dd_field_tc.cuh, one table entry per scan) and the rest on the grid
    tiles: a probe grid, a ragged pitch/2 grid of 2 x 2 tensor-core tiles, an off-lattice
    grid, during and after the scan; every point within the mixed tolerance of the FP64
    plan, and seeded points against the oracle."""
    rng = np.random.default_rng(17)
    specs, grids, times = [], [], []
    for k in range(6):
        n = int(rng.integers(64, 101))
        s = w.ScanSpec(n, n, D_m2s=float(10 ** rng.uniform(-14, -12)), dwell_s=float(10 ** rng.uniform(-7, -6)),
                       sigma_m=0.1e-9, order=w.RANDOM, seed=40 + k, keep_fraction=float(rng.uniform(0.3, 1.0)))
        p = s.pitch_m
        g = [(0.0, 0.0, p, p, n, n), (0.0, 0.0, p / 2, p / 2, 2 * n + 3, 2 * n - 5),
             (-0.37 * p, 0.21 * p, 0.7 * p, 0.7 * p, 97, 130)][k % 3]
        nv = w.n_visits(s)
        specs.append(s)
        grids.append(g)
        times.append([nv * s.dwell_s, (0.7 * nv + 0.5) * s.dwell_s, 4.0 * nv * s.dwell_s][k % 3])
    times = np.array(times)
    scans = [b.Scan(s) for s in specs]
    split = [int(b.dd_field_grid_split(sc, *g, times[k:k + 1])[0]) for k, (sc, g) in enumerate(zip(scans, grids))]
    assert sum(x > 0 for x in split) >= 4, split          # the contraction takes part
    plan = b.Batch(scans, None, times, "mixed", grids=grids)
    out = plan.run(device=cuda).cpu().numpy()
    np.testing.assert_array_equal(out, plan.run(device=cuda).cpu().numpy())   # graph replay
    ref64 = b.Batch(scans, None, times, "fp64", grids=grids).run(device=cuda).cpu().numpy()
    for k, (s, g) in enumerate(zip(specs, grids)):
        got = out[plan.offsets[k]:plan.offsets[k + 1]]
        r64 = ref64[plan.offsets[k]:plan.offsets[k + 1]]
        assert_mixed(got, r64, r64.max(), "tc grid batch scan %d vs fp64" % k)
        pts = grid_pts(g)
        ip = rng.integers(0, len(pts), 24)
        ref = oracle_pairs(s, pts, times[k:k + 1], ip, np.zeros(len(ip), int))
        assert_fp64(r64[ip], ref, "tc grid batch scan %d fp64" % k)
        assert_mixed(got[ip], ref, r64.max(), "tc grid batch scan %d" % k)
