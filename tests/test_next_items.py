"""Multi-frame acquisitions, live-mode snapshot streams and headless maps (GPU)."""
import numpy as np
import pytest

from paper_2507_00294_gb300 import binding as b
from paper_2507_00294_gb300 import workloads as w
from parity_util import assert_fp64, assert_mixed, oracle_dose, oracle_field

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("frames", [2, 4])
def test_multi_frame_field_and_dose(cuda, frames):
    spec = b.multi_frame_spec(w.ScanSpec(8, 8, order=w.SERPENTINE), frames)
    assert len(b.Scan(spec)) == 64 * frames
    pts = w.grid_points(16, spec.pitch_m / 2)
    end = 64 * frames * spec.dwell_s
    times = np.array([0.5 * end, end])
    ref = oracle_field(spec, pts, times)
    assert_fp64(b.dd_field_at_times(b.Scan(spec), pts, times, "fp64"), ref, "multi-frame fp64")
    assert_mixed(b.dd_field_at_times(b.Scan(spec), pts, times, "mixed"), ref, ref.max(axis=1), "multi-frame")
    dref = oracle_dose(spec)
    assert_fp64(b.dd_per_probe_dose(b.Scan(spec), "fp64"), dref, "multi-frame dose")


def test_live_mode_snapshot_stream(cuda):
    job = w.live_mode(12, 5e-6)
    assert len(job.times) == 12 * 12 // 5
    ref = oracle_field(job.scan, job.pts_xy, job.times)
    got = b.dd_field_at_times(b.Scan(job.scan), job.pts_xy, job.times, "mixed")
    assert_mixed(got, ref, ref.max(axis=1), "live mode")


def _levels_from_definition(field, decades=6.0):
    """Grey levels restated from their definition (log10 of the field over its maximum,
    six decades onto 0..255), and the unrounded level, for the comparison below."""
    top = float(np.max(field))
    lv = 255.0 * (1.0 + np.log10(np.maximum(field, top * 10.0 ** -decades) / top) / decades)
    return np.clip(np.floor(lv + 0.5), 0, 255).astype(np.uint8), lv


def test_headless_maps(cuda, tmp_path):
    """Fig. 1-style maps: the field behind each PGM matches the oracle's (mixed tolerance),
    and each image equals the oracle field quantised the same way, except by one grey level
    where the oracle's unrounded level lies within the field tolerance of a rounding edge."""
    from paper_2507_00294_gb300 import figures
    spec = w.ScanSpec(16, 16, order=w.INTERLEAVED, interleave_stride=4)
    pts, times, field = figures.fig1_field(spec)
    ref = oracle_field(spec, pts, times).reshape(field.shape)
    for i in range(2):
        assert_mixed(field[i], ref[i], ref[i].max(), "fig1 map %d" % i)
    paths = figures.fig1_maps(spec, str(tmp_path))
    head = b"P5\n32 32\n255\n"
    for i, p in enumerate(paths):
        data = open(p, "rb").read()
        assert data.startswith(head) and len(data) == len(head) + 32 * 32
        img = np.frombuffer(data[len(head):], np.uint8).reshape(32, 32)
        want, lv = _levels_from_definition(ref[i])
        assert img.max() == 255 and img.min() < 255
        # a 1e-5 relative field error moves a level by at most 255 * 2 * 4.4e-6 / 6 = 4e-4
        edge = np.abs((lv - np.floor(lv)) - 0.5) < 1e-3
        diff = np.abs(img.astype(int) - want.astype(int))
        assert np.all(diff[~edge] == 0), "grey levels differ away from a rounding edge"
        assert np.all(diff <= 1)


@pytest.mark.parametrize("spec", [
    w.ScanSpec(12, 12, order=w.RANDOM, seed=21, blank_s=3e-7),
    w.ScanSpec(16, 16, order=w.RANDOM, seed=22, keep_fraction=0.4, blank_s=1e-7, blank_s_per_m=400.0,
               D_m2s=2e-13),
    w.ScanSpec(10, 10, order=w.RASTER, mask=(np.arange(100).reshape(10, 10) % 7 != 3).astype(np.uint8),
               blank_s_per_m=1000.0, flyback_s=5e-7),
    w.ScanSpec(12, 12, order=w.INTERLEAVED, interleave_stride=3, blank_s=2e-7, D_m2s=1e-15),
])
def test_blanker_travel_field_and_dose(cuda, spec):
    """Random, subsampled, masked and interleaved scans with the blanker's dead time before
    every jump longer than one pitch (constant and distance-proportional): field and dose,
    both precisions, against the oracle."""
    assert not np.allclose(np.diff(b.Scan(spec).visits()[1]), spec.dwell_s)   # dead time present
    pts = w.grid_points(2 * spec.nx, spec.pitch_m / 2)
    _, ts, taus = b.Scan(spec).visits()
    end = ts[-1] + taus[-1]
    # half a dwell away from every visit boundary: there the field's derivative in t is
    # large at the beam, and start times off the dwell lattice carry different roundings
    # in seconds (library) and in dwells (oracle), some 1e-13 of a dwell after a hundred
    # dead times -- 5e-12 of a lag of 0.02 dwell
    k = len(ts) // 3
    times = np.array([ts[k] + 0.5 * taus[k], end + 0.5 * spec.dwell_s, 3 * end])
    ref = oracle_field(spec, pts, times)
    assert_fp64(b.dd_field_at_times(b.Scan(spec), pts, times, "fp64"), ref, "blanker field fp64")
    assert_mixed(b.dd_field_at_times(b.Scan(spec), pts, times, "mixed"), ref, ref.max(axis=1),
                 "blanker field mixed")
    dref = oracle_dose(spec)
    d64 = b.dd_per_probe_dose(b.Scan(spec), "fp64")
    assert d64[0] == 0.0
    assert_fp64(d64, dref, "blanker dose fp64")
    dmx = b.dd_per_probe_dose(b.Scan(spec), "mixed")
    assert_mixed(dmx[1:], dref[1:], dref.max(), "blanker dose mixed")
