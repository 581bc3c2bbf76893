"""Pins for the oracle's scan orders and visit times (Sec. 1 scan strategies, Eq. 5
visit order).  Expected sequences are written out by hand from the definitions."""
import numpy as np

from oracle import scan


def test_raster_and_serpentine_small():
    assert scan.visit_order(3, 2, scan.RASTER) == [0, 1, 2, 3, 4, 5]
    assert scan.visit_order(3, 3, scan.SERPENTINE) == [0, 1, 2, 5, 4, 3, 6, 7, 8]
    assert scan.visit_order(1, 3, scan.SERPENTINE) == [0, 1, 2]


def test_interleaved_small():
    assert scan.visit_order(4, 4, scan.INTERLEAVED, stride=2) == [
        0, 2, 8, 10, 1, 3, 9, 11, 4, 6, 12, 14, 5, 7, 13, 15]
    # ragged: stride 3 on a 4 x 4 grid
    assert scan.visit_order(4, 4, scan.INTERLEAVED, stride=3) == [
        0, 3, 12, 15, 1, 13, 2, 14, 4, 7, 5, 6, 8, 11, 9, 10]
    # stride 1 is raster
    assert scan.visit_order(5, 3, scan.INTERLEAVED, stride=1) == list(range(15))


def test_splitmix64_published_outputs():
    g = scan.splitmix64(0)
    assert [next(g) for _ in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4,
                                           0x06C45D188009454F]


def test_random_order_is_a_seeded_permutation():
    a = scan.visit_order(16, 16, scan.RANDOM, seed=42)
    b = scan.visit_order(16, 16, scan.RANDOM, seed=42)
    c = scan.visit_order(16, 16, scan.RANDOM, seed=43)
    assert a == b and a != c
    assert sorted(a) == list(range(256))


def test_keep_fraction_and_mask():
    n = 10 * 10
    for f in (0.1, 0.37, 0.5, 0.999):
        v = scan.visit_order(10, 10, scan.RANDOM, seed=9, keep_fraction=f)
        assert len(v) == int(np.floor(f * n + 0.5))
        assert v == scan.permutation(n, 9)[:len(v)]
        r = scan.visit_order(10, 10, scan.RASTER, seed=9, keep_fraction=f)
        assert sorted(r) == sorted(v) and r == sorted(r)
    mask = np.zeros((3, 4), dtype=np.uint8)
    mask[0, 1] = mask[1, 3] = mask[2, 0] = 1
    assert scan.visit_order(4, 3, scan.SERPENTINE, mask=mask) == [1, 7, 8]


def test_visit_times():
    tau, fb = 1e-6, 0.25e-6
    v = scan.visit_order(3, 2, scan.RASTER)
    ts, taus = scan.visit_times(v, 3, scan.RASTER, tau)
    assert list(ts) == [k * tau for k in range(6)] and np.all(taus == tau)
    ts, _ = scan.visit_times(v, 3, scan.RASTER, tau, flyback=fb)
    np.testing.assert_allclose(ts, [0, tau, 2 * tau, 3 * tau + fb, 4 * tau + fb, 5 * tau + fb],
                               rtol=1e-15)
    ts, taus = scan.visit_times([0, 1, 2], 3, scan.RANDOM, tau, dwell_per_visit=[1e-6, 2e-6, 5e-7])
    np.testing.assert_allclose(ts, [0, 1e-6, 3e-6], rtol=1e-15)


def test_visit_times_with_blanker_travel():
    """Dead time of the blanker before a jump longer than one pitch (worked by hand on a
    4-wide grid): 0 -> 1 and 1 -> 5 are neighbours (no dead time), 5 -> 2 is a diagonal
    jump of sqrt(2) pitches, 2 -> 15 jumps (1, 3) pitches = sqrt(10)."""
    tau, blank, per_m, p = 1e-6, 0.3e-6, 200.0, 0.5e-9
    v = [0, 1, 5, 2, 15]
    ts, taus = scan.visit_times(v, 4, scan.CUSTOM, tau, pitch=p, blank=blank, blank_per_m=per_m)
    d1 = 0.3e-6 + 200.0 * 0.5e-9 * 1.4142135623730951
    d2 = 0.3e-6 + 200.0 * 0.5e-9 * 3.1622776601683795
    np.testing.assert_allclose(ts, [0.0, 1e-6, 2e-6, 3e-6 + d1, 4e-6 + d1 + d2], rtol=1e-15)
    assert np.all(taus == tau)
    # with a flyback too, a raster row change pays both
    v = scan.visit_order(3, 2, scan.RASTER)
    ts, _ = scan.visit_times(v, 3, scan.RASTER, tau, flyback=0.25e-6, pitch=p, blank=blank)
    np.testing.assert_allclose(ts, [0, tau, 2 * tau, 3 * tau + 0.25e-6 + blank,
                                    4 * tau + 0.25e-6 + blank, 5 * tau + 0.25e-6 + blank], rtol=1e-15)


def test_sources_positions():
    xs, ys, ts, taus, g = scan.sources(3, 2, 0.5e-9, 1e-6, order=scan.SERPENTINE)
    assert list(g) == [0, 1, 2, 5, 4, 3]
    np.testing.assert_array_equal(xs, np.array([0, 1, 2, 2, 1, 0]) * 0.5e-9)
    np.testing.assert_array_equal(ys, np.array([0, 0, 0, 1, 1, 1]) * 0.5e-9)


def test_vectorised_raster_sources_equal_the_list_builder():
    """The vectorised raster sources used by the maximum-size parity test equal the
    oracle's list-based builder bit for bit (positions, start times, dwells)."""
    from paper_2507_00294_gb300 import workloads as w
    from parity_util import raster_sources
    for nx, ny in [(1, 1), (37, 23), (128, 3)]:
        spec = w.ScanSpec(nx, ny, dwell_s=0.7e-6)
        xs, ys, ts, taus, _ = scan.sources(nx, ny, spec.pitch_m, spec.dwell_s)
        fast = raster_sources(spec)
        for a, b_ in zip((xs, ys, ts, taus), (fast.xs, fast.ys, fast.ts, fast.taus)):
            assert np.array_equal(a, b_)
