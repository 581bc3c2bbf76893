"""The work split of the multi-GPU path, run on one GPU: each rank's share (a range of
point tiles for the field, a range of dose targets) evaluated through the C-ABI one after
the other, concatenated, and compared with the whole job in one call and with the oracle.
(The shares never wait on one another, so running them in turn on one GPU is the same
computation as running them on several.)"""
import numpy as np
import pytest

from paper_2507_00294_gb300 import binding as b
from paper_2507_00294_gb300 import shard
from paper_2507_00294_gb300 import workloads as w
from parity_util import assert_fp64, assert_mixed, oracle_dose, oracle_pairs, peak_lower_bound

pytestmark = pytest.mark.gpu


def _close(a, c, rtol):
    m = np.abs(c) > 0
    assert np.all(a[~m] == 0.0)
    return np.max(np.abs(a[m] / c[m] - 1.0)) <= rtol


@pytest.mark.parametrize("world", [2, 3, 8])
def test_split_shares_equal_the_whole_job(cuda, world):
    import torch
    job = w.raster_64_supersampled()
    scan = b.Scan(job.scan)
    n = len(scan)
    pts = torch.from_numpy(job.pts_xy).to(cuda)
    for prec, rtol in (("mixed", 2e-6), ("fp64", 1e-13)):
        whole = b.dd_field_at_times(scan, pts, job.times, prec).cpu().numpy()
        whole_d = b.dd_per_probe_dose(scan, prec, device=cuda).cpu().numpy()
        parts = [b.dd_field_at_times(scan, pts[p0:p1].contiguous(), job.times, prec).cpu().numpy()
                 for p0, p1 in shard.point_ranges(len(job.pts_xy), world)]
        dparts = [b.dd_per_probe_dose_range(scan, j0, j1, prec, device=cuda).cpu().numpy()
                  for j0, j1 in shard.dose_ranges(n, world)]
        split = np.concatenate(parts, axis=1)
        split_d = np.concatenate(dparts)
        assert split.shape == whole.shape and split_d.shape == whole_d.shape
        assert _close(split, whole, rtol), prec
        assert _close(split_d[1:], whole_d[1:], rtol) and split_d[0] == 0.0, prec
        # and against the oracle on seeded pairs
        ip, it = w.sample_pairs(len(job.pts_xy), len(job.times), 512, seed=world)
        ref = oracle_pairs(job.scan, job.pts_xy, job.times, ip, it)
        if prec == "fp64":
            assert_fp64(split[it, ip], ref, "split field fp64")
        else:
            assert_mixed(split[it, ip], ref, peak_lower_bound(job.scan, job.times)[it], "split field mixed")


@pytest.mark.parametrize("spec", [w.ScanSpec(40, 30, order=w.RANDOM, seed=5),
                                  w.ScanSpec(20, 20, order=w.RANDOM, seed=6, blank_s=2e-7)])
def test_dose_ranges_against_the_oracle(cuda, spec):
    """Target ranges that start and end inside dose tiles, the empty range and the last
    visit alone, both precisions, uniform (lag-table) and general timing."""
    scan = b.Scan(spec)
    n = len(scan)
    ref = oracle_dose(spec)
    for j0, j1 in ((0, n), (0, 1), (1, 2), (100, 300), (257, min(n, 811)), (n - 1, n), (5, 5)):
        for prec in ("fp64", "mixed"):
            got = b.dd_per_probe_dose_range(scan, j0, j1, prec, device=cuda).cpu().numpy()
            assert got.shape == (j1 - j0,)
            if j1 == j0:
                continue
            if prec == "fp64":
                assert_fp64(got, ref[j0:j1], "dose range fp64")
            else:
                keep = np.arange(j0, j1) > 0
                if np.any(ref[j0:j1][keep] >= 1e-6 * ref.max()):
                    assert_mixed(got[keep], ref[j0:j1][keep], ref.max(), "dose range mixed")
                else:                                       # below the tolerance's floor
                    assert np.all(np.abs(got[keep]) <= 1e-6 * ref.max())
    with pytest.raises(b.DDError) as e:
        b.dd_per_probe_dose_range(scan, 3, n + 1, "mixed", device=cuda)
    assert e.value.status == b.DD_EINVAL


@pytest.mark.parametrize("world", [2, 3, 8])
def test_grid_snapshot_sets_equal_the_whole_job(cuda, world):
    """The grid form of the split: each rank keeps the whole 128 x 128 grid of the 64 x 64
    raster and evaluates the snapshot set the pair-count deal gives it (one call per set,
    the tensor-core contraction inside every call that reaches it); the sets put back at
    their indices against the whole job in one call -- FP64 within 1e-12, FP32-mixed
    within the mixed tolerance of the FP64 field at every point -- and the mixed rows
    against the oracle on seeded pairs."""
    job = w.raster_64_supersampled()
    scan = b.Scan(job.scan)
    p = job.scan.pitch_m
    x0, y0, dx, dy, nc, nr = 0.0, 0.0, p / 2, p / 2, 128, 128
    n_pts = nc * nr
    assert np.array_equal(job.pts_xy, w.grid_points(128, p / 2))          # the same points, row-major
    _, ts, _ = scan.visits()
    nact = np.searchsorted(ts, job.times, side="left")
    sets = shard.snapshot_sets([int(a) * n_pts for a in nact], world)
    assert sorted(k for s in sets for k in s) == list(range(len(job.times)))

    def on_grid(times, prec):
        return b.dd_field_on_grid(scan, x0, y0, dx, dy, nc, nr, np.ascontiguousarray(times), prec,
                                  device=cuda).cpu().numpy()

    whole64 = on_grid(job.times, "fp64")
    for prec in ("fp64", "mixed"):
        split = np.full_like(whole64, np.nan)
        for s in sets:
            if s:
                split[s] = on_grid(job.times[s], prec)
        assert not np.isnan(split).any()
        if prec == "fp64":
            assert_fp64(split, whole64, "snapshot split fp64")
        else:
            assert_mixed(split, whole64, whole64.max(axis=1), "snapshot split mixed vs fp64")
            ip, it = w.sample_pairs(n_pts, len(job.times), 512, seed=world)
            ref = oracle_pairs(job.scan, job.pts_xy, job.times, ip, it)
            assert_mixed(split[it, ip], ref, peak_lower_bound(job.scan, job.times)[it], "snapshot split vs oracle")
