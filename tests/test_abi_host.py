"""C-ABI checks that need no GPU: the library loads, exports every entry point that
include/dd.h declares, builds scans exactly like the oracle's independent scan code,
and rejects bad arguments."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import scan as oscan
from paper_2507_00294_gb300 import binding as b
from paper_2507_00294_gb300 import workloads as w

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "dd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dd_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    lib = b.load()
    names = declared_functions()
    assert "dd_create_scan" in names and "dd_field_at_times" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def _compare_with_oracle(spec):
    s = b.Scan(spec)
    g, t, tau = s.visits()
    xs, ys, ts, taus, og = oscan.sources(
        spec.nx, spec.ny, spec.pitch_m, spec.dwell_s, order=spec.order,
        stride=spec.interleave_stride, seed=spec.seed, keep_fraction=spec.keep_fraction,
        mask=spec.mask, custom=spec.custom_visit, flyback=spec.flyback_s,
        dwell_per_visit=spec.dwell_per_visit, blank=spec.blank_s, blank_per_m=spec.blank_s_per_m)
    np.testing.assert_array_equal(g, og)
    np.testing.assert_array_equal(t, ts)      # same FP64 recipe on both sides: bit-exact
    np.testing.assert_array_equal(tau, taus)
    return s


@pytest.mark.parametrize("order,stride", [(w.RASTER, 1), (w.SERPENTINE, 1), (w.INTERLEAVED, 4),
                                          (w.INTERLEAVED, 3), (w.RANDOM, 1)])
@pytest.mark.parametrize("nx,ny", [(1, 1), (7, 5), (16, 16), (33, 20)])
def test_scan_orders_match_oracle(order, stride, nx, ny):
    _compare_with_oracle(w.ScanSpec(nx, ny, order=order, interleave_stride=stride, seed=1234))


def test_scan_subsets_flyback_and_dwell_match_oracle():
    _compare_with_oracle(w.ScanSpec(20, 20, order=w.RANDOM, seed=99, keep_fraction=0.37))
    _compare_with_oracle(w.ScanSpec(20, 17, order=w.SERPENTINE, seed=5, keep_fraction=0.5))
    mask = (np.arange(12 * 9).reshape(9, 12) % 3 != 1).astype(np.uint8)
    _compare_with_oracle(w.ScanSpec(12, 9, order=w.INTERLEAVED, interleave_stride=2, mask=mask))
    _compare_with_oracle(w.ScanSpec(10, 6, order=w.RASTER, flyback_s=3e-7))
    _compare_with_oracle(w.ScanSpec(10, 6, order=w.SERPENTINE, flyback_s=1e-7, mask=mask[:6, :10]))
    rng = np.random.default_rng(3)
    _compare_with_oracle(w.ScanSpec(8, 8, dwell_per_visit=10 ** rng.uniform(-7, -5, 64)))


def test_scan_blanker_travel_matches_oracle():
    """Blanker dead time before jumps longer than one pitch: random, subsampled, masked,
    interleaved and raster-with-flyback scans, constant and distance-proportional parts."""
    mask = (np.arange(12 * 9).reshape(9, 12) % 5 != 2).astype(np.uint8)
    rng = np.random.default_rng(4)
    for spec in (w.ScanSpec(16, 16, order=w.RANDOM, seed=7, blank_s=2e-7),
                 w.ScanSpec(20, 20, order=w.RANDOM, seed=8, keep_fraction=0.3, blank_s_per_m=300.0),
                 w.ScanSpec(12, 9, order=w.RASTER, mask=mask, blank_s=1e-7, blank_s_per_m=50.0),
                 w.ScanSpec(12, 12, order=w.INTERLEAVED, interleave_stride=3, blank_s=5e-8),
                 w.ScanSpec(10, 6, order=w.SERPENTINE, flyback_s=3e-7, blank_s=1e-7,
                            keep_fraction=0.6, seed=2),
                 w.ScanSpec(9, 9, order=w.RANDOM, seed=3, blank_s=1e-7,
                            dwell_per_visit=10 ** rng.uniform(-7, -5, 81))):
        _compare_with_oracle(spec)
    s = b.Scan(w.ScanSpec(4, 4, order=w.RANDOM, seed=1, blank_s=1e-7))
    _, t, tau = s.visits()
    assert np.all(np.diff(t) >= tau[:-1] * (1 - 1e-12))    # dead time only adds


def test_destroyed_scans_storage_reused():
    """A destroyed scan's host storage is kept for the next scan: scans of growing and
    shrinking sizes and of every order, each built right after the previous one was
    destroyed, still match the oracle's visit lists and times exactly."""
    rng = np.random.default_rng(4)
    specs = [w.ScanSpec(40, 40), w.ScanSpec(3, 5, order=w.SERPENTINE), w.ScanSpec(64, 64, order=w.RANDOM, seed=9),
             w.ScanSpec(7, 7, order=w.INTERLEAVED, interleave_stride=2, keep_fraction=0.5, seed=3),
             w.ScanSpec(30, 20, order=w.SERPENTINE, flyback_s=2e-7),
             w.ScanSpec(6, 6, order=w.CUSTOM, custom_visit=np.array([35, 0, 7, 7, 14])),
             w.ScanSpec(12, 12, order=w.RANDOM, seed=5, dwell_per_visit=10 ** rng.uniform(-7, -5, 144)),
             w.ScanSpec(50, 50, order=w.RASTER, blank_s=1e-7)]
    for spec in specs + specs[::-1]:
        s = _compare_with_oracle(spec)
        assert len(s) == len(s.visits()[0])
        s.close()


def test_scan_rejects_negative_blanker_time():
    for kw in ({"blank_s": -1e-9}, {"blank_s_per_m": -1.0}, {"blank_s": float("nan")}):
        with pytest.raises(b.DDError) as e:
            b.Scan(w.ScanSpec(4, 4, **kw))
        assert e.value.status == b.DD_EINVAL
    _compare_with_oracle(w.ScanSpec(5, 5, order=w.CUSTOM, custom_visit=np.array([24, 0, 12, 3, 3, 7])))


def test_random_order_uses_splitmix64_fisher_yates():
    s = b.Scan(w.ScanSpec(9, 9, order=w.RANDOM, seed=2024))
    assert list(s.visits()[0]) == oscan.permutation(81, 2024)


@pytest.mark.parametrize("field,value", [("nx", 0), ("pitch_m", 0.0), ("sigma_m", -1.0),
                                         ("D_m2s", float("nan")), ("dwell_s", 0.0),
                                         ("keep_fraction", 0.0), ("keep_fraction", 1.5),
                                         ("order", 9), ("flyback_s", -1.0)])
def test_invalid_descriptions_rejected(field, value):
    spec = w.ScanSpec(4, 4)
    setattr(spec, field, value)
    with pytest.raises(b.DDError) as e:
        b.Scan(spec)
    assert e.value.status == b.DD_EINVAL


def test_invalid_combinations_rejected():
    with pytest.raises(b.DDError):
        b.Scan(w.ScanSpec(4, 4, order=w.RANDOM, flyback_s=1e-7))      # flyback only for raster
    with pytest.raises(b.DDError):
        b.Scan(w.ScanSpec(4, 4, keep_fraction=0.5, mask=np.ones(16, np.uint8)))
    with pytest.raises(b.DDError):
        b.Scan(w.ScanSpec(4, 4, order=w.CUSTOM, custom_visit=np.array([0, 16])))
    with pytest.raises(b.DDError):
        b.Scan(w.ScanSpec(4, 4, mask=np.zeros(16, np.uint8)))          # visits nothing
    with pytest.raises(b.DDError):
        b.Scan(w.ScanSpec(3, 3, dwell_per_visit=np.array([1e-6] * 8 + [0.0])))


def test_null_and_size_arguments_rejected_without_gpu():
    lib = b.load()
    assert lib.dd_create_scan(None, None) == b.DD_EINVAL
    assert b"NULL" in lib.dd_last_error()
    lib.dd_destroy(None)                          # NULL-safe
    s = b.Scan(w.ScanSpec(2, 2))
    out = np.zeros(4)
    pts = np.zeros(8)
    t = np.array([1e-6])
    assert lib.dd_field_at_times(None, pts.ctypes.data, 4, t.ctypes.data, 1, 1, out.ctypes.data, None) == b.DD_EINVAL
    assert lib.dd_field_at_times(s.handle, pts.ctypes.data, -1, t.ctypes.data, 1, 1, out.ctypes.data, None) == b.DD_EINVAL
    assert lib.dd_field_at_times(s.handle, pts.ctypes.data, 4, t.ctypes.data, 1, 7, out.ctypes.data, None) == b.DD_EINVAL
    assert lib.dd_field_at_times(s.handle, None, 4, t.ctypes.data, 1, 1, out.ctypes.data, None) == b.DD_EINVAL
    # empty requests are no-ops that touch no device
    assert lib.dd_field_at_times(s.handle, None, 0, None, 0, 1, None, None) == b.DD_OK
    assert lib.dd_per_probe_dose(s.handle, 5, out.ctypes.data, None) == b.DD_EINVAL
    fb = b.Scan(w.ScanSpec(3, 3, flyback_s=1e-7))
    # the allocation-free dose keeps to uniform dwells (checked before any device work)
    assert lib.dd_per_probe_dose_noalloc(fb.handle, 1, out.ctypes.data, None) == b.DD_ENOTSUP


def test_double_destroy_is_harmless():
    lib = b.load()
    s = b.Scan(w.ScanSpec(3, 3))
    h = s.handle
    lib.dd_destroy(h)
    lib.dd_destroy(h)             # second call finds no live handle: no-op
    s.handle = None
