"""The field on a rectilinear grid of points (dd_field_on_grid) against the oracle and
against the same points given as a list (dd_field_at_times)."""
import numpy as np
import pytest

from paper_2507_00294_gb300 import binding as b
from paper_2507_00294_gb300 import workloads as w
from parity_util import assert_fp64, assert_mixed, oracle_field, oracle_pairs, peak_lower_bound

pytestmark = pytest.mark.gpu


def grid_pts(x0, y0, dx, dy, nc, nr):
    """The grid's points in row-major order, each coordinate one product and one sum."""
    c = np.arange(nc, dtype=np.float64) * dx + x0
    r = np.arange(nr, dtype=np.float64) * dy + y0
    yy, xx = np.meshgrid(r, c, indexing="ij")
    return np.stack([xx.reshape(-1), yy.reshape(-1)], axis=1)


def on_grid(spec, g, times, prec):
    import torch
    scan = b.Scan(spec)
    out = b.dd_field_on_grid(scan, *g, np.asarray(times), prec, device=torch.device("cuda", 0))
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_bench_workload_grid_sampled_and_equal_to_point_list(cuda):
    """The 64x64 raster at 128x128 points (pitch/2) and its 64 row snapshots: the FP64
    path is bit for bit the point-list result; FP32-mixed against the oracle on 4096
    seeded pairs and within the mixed tolerance of the point-list result everywhere."""
    import torch
    job = w.raster_64_supersampled()
    p = job.scan.pitch_m
    g = (0.0, 0.0, p / 2, p / 2, 128, 128)
    pts = grid_pts(*g)
    assert np.array_equal(pts, job.pts_xy)
    scan = b.Scan(job.scan)
    lst64 = b.dd_field_at_times(scan, torch.from_numpy(pts).cuda(), job.times, "fp64").cpu().numpy()
    g64 = on_grid(job.scan, g, job.times, "fp64")
    np.testing.assert_array_equal(g64, lst64)
    gm = on_grid(job.scan, g, job.times, "mixed")
    lstm = b.dd_field_at_times(scan, torch.from_numpy(pts).cuda(), job.times, "mixed").cpu().numpy()
    assert_mixed(gm, lst64, lst64.max(axis=1), "grid vs list (fp64) mixed")
    ip, it = w.sample_pairs(len(pts), len(job.times), 4096, seed=2)
    ref = oracle_pairs(job.scan, pts, job.times, ip, it)
    assert_mixed(gm[it, ip], ref, peak_lower_bound(job.scan, job.times)[it], "grid mixed")
    assert_fp64(g64[it, ip], ref, "grid fp64")
    # the separable form and the tensor-core contraction of the older visits (BF16 pieces,
    # FP32 accumulation in another order) change only the FP32 rounding: both results
    # within a few 1e-6 of each other
    rel = np.abs(gm - lstm)[lstm > 1e-6 * lstm.max(axis=1, keepdims=True)] / lstm[lstm > 1e-6 * lstm.max(axis=1, keepdims=True)]
    assert rel.max() <= 5e-6


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_ragged_off_lattice_grids(cuda, prec):
    """Grids whose width is not a multiple of 128 columns and height not of 4 rows, with
    an origin and spacing off the probe lattice (split offsets), a negative spacing, and
    snapshots on and off the dwell lattice: every point against the oracle."""
    cases = [
        (w.ScanSpec(12, 10, order=w.SERPENTINE), (-0.37e-9, 0.21e-9, 0.5e-9 / 3, 0.5e-9 / 3, 200, 7)),
        (w.ScanSpec(9, 9, order=w.RANDOM, seed=4, D_m2s=1e-15), (4.5e-9, -0.2e-9, -0.25e-9, 0.125e-9, 37, 45)),
        (w.ScanSpec(16, 16, order=w.INTERLEAVED, interleave_stride=4, D_m2s=1e-12), (0.0, 0.0, 0.5e-9, 0.5e-9, 16, 16)),
        (w.ScanSpec(20, 3, keep_fraction=0.5, seed=1), (0.0, 0.0, 0.25e-9, 0.25e-9, 129, 13)),
    ]
    for spec, g in cases:
        n = w.n_visits(spec)
        times = np.array([0.5 * n, n - 0.3, float(n), 4.0 * n]) * spec.dwell_s
        pts = grid_pts(*g)
        ref = oracle_field(spec, pts, times)
        got = on_grid(spec, g, times, prec)
        if prec == "fp64":
            assert_fp64(got, ref, "ragged grid fp64")
        else:
            assert_mixed(got, ref, ref.max(axis=1), "ragged grid mixed")


@pytest.mark.parametrize("D", [6e-14, 1e-15])
def test_class_limits_on_a_grid_row(cuda, D):
    """One visit seen at the end of its dwell and half a dwell later from a 6001 x 2 grid
    whose columns sweep h = rho^2 dq over 0 .. 3.5 (every series class and its limits,
    the cross term on and off), plus a second row one pitch away: every point against the
    oracle in FP32-mixed."""
    spec = w.ScanSpec(1, 1, D_m2s=D)
    tau, p = spec.dwell_s, spec.pitch_m
    s, kappa = spec.sigma_m ** 2 / p ** 2, spec.D_m2s * tau / p ** 2
    dq = 1.0 / (2 * s) - 1.0 / (2 * s + 4 * kappa)
    xmax = p * np.sqrt(3.5 / dq)
    g = (0.0, 0.0, xmax / 6000, p, 6001, 2)
    times = np.array([tau, 1.5 * tau])
    ref = oracle_field(spec, grid_pts(*g), times)
    assert_mixed(on_grid(spec, g, times, "mixed"), ref, ref.max(axis=1), "grid class limits")


def test_grid_empty_and_invalid(cuda):
    import torch
    scan = b.Scan(w.ScanSpec(4, 4))
    out = b.dd_field_on_grid(scan, 0.0, 0.0, 1e-10, 1e-10, 0, 5, np.array([1e-6]), "mixed", device=cuda)
    assert out.shape == (1, 0)
    with pytest.raises(b.DDError) as e:
        b.dd_field_on_grid(scan, float("nan"), 0.0, 1e-10, 1e-10, 3, 3, np.array([1e-6]), "mixed", device=cuda)
    assert e.value.status == b.DD_EINVAL
