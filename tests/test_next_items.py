"""Multi-frame acquisitions, live-mode snapshot streams and headless maps (GPU)."""
import numpy as np
import pytest

import oracle
from paper_2507_00294_gb300 import binding as b
from paper_2507_00294_gb300 import workloads as w
from parity_util import assert_fp64, assert_mixed, oracle_field, oracle_sources

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
    dref = oracle.dose(oracle_sources(spec), spec.sigma_m ** 2, spec.D_m2s, spec.Q0)
    assert_fp64(b.dd_per_probe_dose(b.Scan(spec), "fp64"), dref, "multi-frame dose")


def test_live_mode_snapshot_stream(cuda):
    job = w.live_mode(12, 5e-6)
    assert len(job.times) == 12 * 12 // 5
    ref = oracle_field(job.scan, job.pts_xy, job.times)
    got = b.dd_field_at_times(b.Scan(job.scan), job.pts_xy, job.times, "mixed")
    assert_mixed(got, ref, ref.max(axis=1), "live mode")


def test_headless_maps(cuda, tmp_path):
    from paper_2507_00294_gb300 import figures
    paths = figures.fig1_maps(w.ScanSpec(16, 16, order=w.INTERLEAVED, interleave_stride=4), str(tmp_path))
    for p in paths:
        data = open(p, "rb").read()
        assert data.startswith(b"P5\n32 32\n255\n") and len(data) == len(b"P5\n32 32\n255\n") + 32 * 32
        img = np.frombuffer(data[-32 * 32:], np.uint8)
        assert img.max() == 255 and img.min() < 255
