"""Host-side descriptors of the surrogate (no GPU): the input maps and scalars, the
background / last-visits split, and the scan draw."""
import math

import numpy as np

from paper_2507_00294_gb300 import surrogate as sur
from paper_2507_00294_gb300 import workloads as w


def test_scan_inputs_time_map_and_scalars():
    specs = sur.draw_scans(5, seed=3)
    tmap, scal = sur.scan_inputs(specs)
    assert tmap.shape == (5, sur.CANVAS, sur.CANVAS) and scal.shape == (5, 3)
    for k, s in enumerate(specs):
        g = sur.visit_list(s)
        nv = len(g)
        iy, ix = g // s.nx, g % s.nx
        # 1 / age at the end of the scan: the last visit 1, the first 1 / n
        np.testing.assert_array_equal(tmap[k, iy, ix], (1.0 / (nv - np.arange(nv))).astype(np.float32))
        assert tmap[k, iy[-1], ix[-1]] == 1.0
        other = np.ones((sur.CANVAS, sur.CANVAS), bool)
        other[iy, ix] = False
        assert np.all(tmap[k][other] == -1.0)
        np.testing.assert_allclose(scal[k, 0], (math.log10(s.D_m2s) + 13.5) / 1.5, rtol=1e-6)
        np.testing.assert_allclose(scal[k, 1], math.log10(s.dwell_s) + 6.0, rtol=1e-6, atol=1e-6)
        np.testing.assert_allclose(scal[k, 2], s.D_m2s * s.dwell_s / s.pitch_m ** 2, rtol=1e-6)
        assert s.sigma_m == sur.PROBE_SIGMA


def test_split_scan_partitions_the_visits():
    spec = sur.draw_scans(1, seed=9)[0]
    g = sur.visit_list(spec)
    n = len(g)
    bg, t_bg, near, t_near = sur.split_scan(spec)
    k = min(sur.K_EXACT, n - 1)
    np.testing.assert_array_equal(np.concatenate([bg.custom_visit, near.custom_visit]), g)
    assert len(near.custom_visit) == k and bg.order == w.CUSTOM and near.order == w.CUSTOM
    # the background seen at the scan's end, the last visits at k dwells in their own clock
    assert t_bg == n * spec.dwell_s and t_near == k * spec.dwell_s
    bg2, _, near2, _ = sur.split_scan(spec, k=5)
    assert len(near2.custom_visit) == 5 and len(bg2.custom_visit) == n - 5


def test_background_plane_constants():
    # the surrogate's scans: sigma 0.1 nm at the 0.5 nm pitch
    assert math.isclose(sur.S_DIM, (0.1e-9 / 0.5e-9) ** 2, rel_tol=1e-12)
    assert sur.REAL_IN == 6 and sur.LAYERS[0][0] >= sur.REAL_IN
