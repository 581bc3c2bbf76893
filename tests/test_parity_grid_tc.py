"""The tensor-core part of the FP32-mixed grid field (the older visits' degree-2 and degree-4
pair terms as BF16-split matrix products, dd_field_tc.cuh): taken where it applies, and the
field it gives against the oracle and against the FP64 path."""
import numpy as np
import pytest

from paper_2507_00294_gb300 import binding as b
from paper_2507_00294_gb300 import workloads as w
from parity_util import assert_fp64, assert_mixed, oracle_pairs, oracle_problem, peak_lower_bound

pytestmark = pytest.mark.gpu


def on_grid(spec, g, times, prec, profile=False):
    import torch
    scan = b.Scan(spec)
    if profile:
        b.dd_profile_reset()
        b.dd_profile_enable(True)
    try:
        out = b.dd_field_on_grid(scan, *g, np.asarray(times), prec, device=torch.device("cuda", 0))
        torch.cuda.synchronize()
    finally:
        if profile:
            b.dd_profile_enable(False)
    launched = b.dd_profile_read() if profile else {}
    return out.cpu().numpy(), launched


def grid_pts(x0, y0, dx, dy, nc, nr):
    c = np.arange(nc, dtype=np.float64) * dx + x0
    r = np.arange(nr, dtype=np.float64) * dy + y0
    yy, xx = np.meshgrid(r, c, indexing="ij")
    return np.stack([xx.reshape(-1), yy.reshape(-1)], axis=1)


def check_against_oracle_and_fp64(spec, g, times, n_samples, seed, what, fp64_vs_oracle=True):
    """Mixed on the grid: sampled (point, snapshot) pairs against the oracle and every
    point against the FP64 path (itself within 1e-12 of the oracle on the samples, unless
    fp64_vs_oracle is False)."""
    gm, launched = on_grid(spec, g, times, "mixed", profile=True)
    assert "field_grid_tc" in launched, what + ": the tensor-core contraction did not run"
    g64, _ = on_grid(spec, g, times, "fp64")
    pts = grid_pts(*g)
    problem = oracle_problem(spec)
    ip, it = w.sample_pairs(len(pts), len(times), n_samples, seed=seed)
    ref = oracle_pairs(spec, pts, times, ip, it, problem)
    peak = peak_lower_bound(spec, times, problem)
    if fp64_vs_oracle:
        assert_fp64(g64[it, ip], ref, what + " fp64")
    assert_mixed(gm[it, ip], ref, peak[it], what + " mixed vs oracle")
    assert_mixed(gm, g64, g64.max(axis=1), what + " mixed vs fp64, every point")
    return gm, g64


def test_ragged_tiles_off_lattice_serpentine(cuda):
    """200 x 150 points (2 x 2 tiles of 128, ragged on both sides), an origin off the probe
    lattice and a spacing of 0.4 pitch over a 40 x 36 serpentine scan, snapshots inside,
    at the end of and long after the scan."""
    spec = w.ScanSpec(40, 36, order=w.SERPENTINE)
    n = w.n_visits(spec)
    g = (-3.37e-9, -2.21e-9, 0.2e-9, 0.2e-9, 200, 150)
    times = np.array([0.6 * n, n - 0.3, float(n), 4.0 * n]) * spec.dwell_s
    check_against_oracle_and_fp64(spec, g, times, 3000, 5, "ragged serpentine")


def test_random_order_blanker_and_per_visit_dwells(cuda):
    """Random order over a 70 % mask, dwells drawn per visit over a decade and a blanker
    dead time per jump: the prefix the contraction takes comes from the longest dwell."""
    base = w.ScanSpec(48, 48, order=w.RANDOM, seed=5, keep_fraction=0.7, blank_s=3e-7, blank_s_per_m=400.0)
    n = w.n_visits(base)
    rng = np.random.default_rng(11)
    spec = base.with_(dwell_per_visit=10 ** rng.uniform(-6.5, -5.5, n))
    _, ts, taus = b.Scan(spec).visits()
    end = ts[-1] + taus[-1]
    # half a dwell away from every visit boundary (where the field's time derivative at
    # the beam is large and start times off the dwell lattice round differently)
    times = np.array([ts[n // 2] + 0.5 * taus[n // 2], ts[(4 * n) // 5] + 0.5 * taus[(4 * n) // 5],
                      end + 0.5 * spec.dwell_s, 3.0 * end])
    g = (0.0, 0.0, 0.25e-9, 0.25e-9, 96, 96)
    # The start times are running sums of 1,613 irregular dwells and dead times, which the
    # library (in seconds) and the oracle (in dwells) round differently: up to about 4e-11
    # dwell apart by the end of the scan, which moves the field half a dwell after the last
    # visit by 5.5e-12 -- the FP64 path's parity is checked on scans whose start times both
    # sides form alike (test_next_items); here the FP64 path is the per-point reference.
    check_against_oracle_and_fp64(spec, g, times, 3000, 6, "random blanker", fp64_vs_oracle=False)


def test_bench_grid_snapshot_groups_and_repeat(cuda):
    """The 64 x 64 raster at 128 x 128 points and its 64 row snapshots: every point within
    the mixed tolerance of the FP64 path, the samples against the oracle, and bit-identical
    on a second call (deterministic order of the partial sums)."""
    job = w.raster_64_supersampled()
    p = job.scan.pitch_m
    g = (0.0, 0.0, p / 2, p / 2, 128, 128)
    gm, _ = check_against_oracle_and_fp64(job.scan, g, job.times, 4096, 2, "bench grid")
    again, launched = on_grid(job.scan, g, job.times, "mixed", profile=True)
    np.testing.assert_array_equal(again, gm)
    # both forms ran: degree 2 (the oldest visits) and degree 4 (the band after them)
    assert "field_grid_tc" in launched and "field_grid_tc4" in launched


def test_grid256_raster_sixteen_tiles(cuda):
    """A 256 x 256 raster (65,536 visits) on a 512 x 512 grid at pitch/2 (16 tiles) at the
    end of the scan and 16x later: samples against the oracle."""
    spec = w.ScanSpec(256, 256)
    n = w.n_visits(spec)
    p = spec.pitch_m
    g = (0.0, 0.0, p / 2, p / 2, 512, 512)
    times = np.array([float(n), 16.0 * n]) * spec.dwell_s
    gm, launched = on_grid(spec, g, times, "mixed", profile=True)
    assert "field_grid_tc" in launched
    pts = grid_pts(*g)
    problem = oracle_problem(spec)
    ip, it = w.sample_pairs(len(pts), len(times), 600, seed=9)
    ref = oracle_pairs(spec, pts, times, ip, it, problem)
    assert_mixed(gm[it, ip], ref, peak_lower_bound(spec, times, problem)[it], "grid256 mixed")


def test_tensor_core_wait_timeout_is_reported(cuda, monkeypatch):
    """Failure detection without a GPU fault: with DD_FAULT=field_tc_wait no MMA is issued,
    the contraction's bounded completion waits run out, its CTAs release their tensor
    memory and write NaN, and dd_field_check reports DD_ETIMEOUT; the next call is normal."""
    spec = w.ScanSpec(32, 32)
    n = w.n_visits(spec)
    g = (0.0, 0.0, 0.25e-9, 0.25e-9, 64, 64)
    times = np.array([4.0 * n]) * spec.dwell_s
    monkeypatch.setenv("DD_FAULT", "field_tc_wait")
    bad, launched = on_grid(spec, g, times, "mixed", profile=True)
    assert "field_grid_tc" in launched
    with pytest.raises(b.DDError) as e:
        b.dd_field_check()
    assert e.value.status == b.DD_ETIMEOUT
    assert np.isnan(bad).any()
    monkeypatch.delenv("DD_FAULT")
    good, _ = on_grid(spec, g, times, "mixed")
    b.dd_field_check()
    g64, _ = on_grid(spec, g, times, "fp64")
    assert_mixed(good, g64, g64.max(axis=1), "after the timeout")
