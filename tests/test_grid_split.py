"""dd_field_grid_split (host-only): the prefixes of visits that dd_field_on_grid sums on the
tensor cores in FP32-mixed precision.  The contraction relies on every such visit's pair
term being on the degree-2 exponent series (h = rho^2 dq <= 0.04) at every grid point, or
on the degree-4 series (h <= 0.33) for the band after the degree-2 prefix; these tests
evaluate h in FP64 from the oracle's visit list and check that, that each prefix is as long
as the library's stated bound allows, and the simple properties of a prefix."""
import numpy as np
import pytest

from paper_2507_00294_gb300 import binding as b
from paper_2507_00294_gb300 import workloads as w
from parity_util import oracle_problem

L2H, L4H = 0.04, 0.33
MIN_DQ = 1e-8            # per pitch^2: the degree-4 coefficients stay in the FP32 normal range


def grid_corners(g):
    x0, y0, dx, dy, nc, nr = g
    xs = np.array([x0, x0 + (nc - 1) * dx])
    ys = np.array([y0, y0 + (nr - 1) * dy])
    return xs, ys


def visit_geometry(spec, t_dwell):
    """Per visit at snapshot t (in dwells): started, dwell over, dq = 1/w0 - 1/w1 [1/m^2]
    (Eq. 1/2 widths w = 2 sigma^2 + 4 D t), from the oracle's visit list."""
    src, Ds, D, _ = oracle_problem(spec)
    dT = t_dwell - src.ts
    over = dT > src.taus
    w1 = 2 * Ds + 4 * D * dT
    w0 = 2 * Ds + 4 * D * np.where(over, dT - src.taus, 0.0)
    with np.errstate(divide="ignore", invalid="ignore"):
        dq = np.where(dT > 0, 1.0 / w0 - 1.0 / w1, np.inf)
    return src, dT > 0, over, dq


def check_split(spec, g, times):
    scan = b.Scan(spec)
    K, K2 = b.dd_field_grid_split(scan, *g, times, degree2=True)
    assert np.all(K2 <= K)
    gx, gy = grid_corners(g)
    src, _, _, _ = visit_geometry(spec, 0.0)
    # the largest squared distance between the grid's box and the visits' box
    ex = max(gx.max() - src.xs.min(), src.xs.max() - gx.min())
    ey = max(gy.max() - src.ys.min(), src.ys.max() - gy.min())
    R2 = ex * ex + ey * ey
    Ds, D = spec.sigma_m ** 2, spec.D_m2s * spec.dwell_s
    c = 4 * D * src.taus.max()
    for k, t in enumerate(np.asarray(times) / spec.dwell_s):
        src, started, over, dq = visit_geometry(spec, t)
        n_started = int(started.sum())
        assert 0 <= K[k] <= n_started
        for n_pre, limit, what in ((K2[k], L2H, "degree-2"), (K[k], L4H, "degree-4")):
            if n_pre > 0:
                i = np.arange(n_pre)
                assert np.all(over[i]), "a visit still under the beam in the prefix"
                # each visit's own farthest grid corner: on the series at every point
                r2 = np.maximum.reduce([(cx - src.xs[i]) ** 2 + (cy - src.ys[i]) ** 2 for cx in gx for cy in gy])
                assert np.all(r2 * dq[i] <= limit), "a prefix visit off the %s series" % what
            if 0 < n_pre < n_started and (limit == L2H or K[k] > K2[k]):
                # the first visit after the prefix fails the stated bound (prefix is maximal)
                j = n_pre
                w1 = 2 * Ds + 4 * D * (t - src.ts[j])
                assert (w1 <= c) or (c / ((w1 - c) * w1)) * R2 > limit * (1 - 1e-3)
        if K[k] > K2[k]:
            band = np.arange(K2[k], K[k])
            assert np.all(dq[band] * spec.pitch_m ** 2 >= MIN_DQ)
    return K


def test_bench_grid_prefix():
    job = w.raster_64_supersampled()
    p = job.scan.pitch_m
    K = check_split(job.scan, (0.0, 0.0, p / 2, p / 2, 128, 128), job.times)
    assert np.all(np.diff(K) >= 0)
    assert K[0] == 0 and K[-1] > 3000            # early rows: none; the last row: most visits


def test_irregular_dwells_and_blanker_prefix():
    base = w.ScanSpec(40, 40, order=w.RANDOM, seed=3, keep_fraction=0.8, blank_s=2e-7, blank_s_per_m=300.0)
    n = w.n_visits(base)
    rng = np.random.default_rng(5)
    spec = base.with_(dwell_per_visit=10 ** rng.uniform(-6.5, -5.5, n))
    T = spec.dwell_per_visit.sum() + n * 2e-7
    times = np.array([0.3, 0.7, 1.0, 2.5, 10.0]) * T
    K = check_split(spec, (-1e-9, 2e-9, 0.3e-9, 0.25e-9, 90, 100), times)
    assert K[-1] == n                            # long after the scan every visit qualifies


def test_interleaved_off_grid_and_small_grids():
    spec = w.ScanSpec(32, 32, order=w.INTERLEAVED, interleave_stride=4, D_m2s=1e-13)
    n = w.n_visits(spec)
    times = np.array([0.5 * n, n - 0.5, 3.0 * n]) * spec.dwell_s
    check_split(spec, (3e-9, -2e-9, 0.17e-9, 0.21e-9, 64, 70), times)
    scan = b.Scan(spec)
    # below 64 points in either direction the grid takes the CUDA-core tile only
    assert np.all(b.dd_field_grid_split(scan, 0.0, 0.0, 1e-10, 1e-10, 63, 200, times) == 0)
    assert np.all(b.dd_field_grid_split(scan, 0.0, 0.0, 1e-10, 1e-10, 200, 63, times) == 0)
    # no snapshot before any dwell is over qualifies anything
    assert np.all(b.dd_field_grid_split(scan, 0.0, 0.0, 1e-10, 1e-10, 64, 64, np.array([0.0, 0.5e-6])) == 0)


def test_split_rejects_bad_arguments():
    scan = b.Scan(w.ScanSpec(4, 4))
    with pytest.raises(b.DDError) as e:
        b.dd_field_grid_split(scan, float("nan"), 0.0, 1e-10, 1e-10, 64, 64, np.array([1e-6]))
    assert e.value.status == b.DD_EINVAL
    with pytest.raises(b.DDError):
        b.dd_field_grid_split(scan, 0.0, 0.0, 1e-10, 1e-10, 64, 64, np.array([float("inf")]))
    assert len(b.dd_field_grid_split(scan, 0.0, 0.0, 1e-10, 1e-10, 64, 64, np.array([]))) == 0
