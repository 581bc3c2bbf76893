"""The FP32-mixed tile's test of whether a point's offset from the tile origin is exact in
one FP32 value: with xi an integer (|xi| < 2^24) and f a fraction (|f| <= 1/2, itself
FP32), x = fl(xi + f) lost no bit exactly when fl(x - xi) == f.  Checked here in FP32
arithmetic against the exact sum in FP64 (which holds xi + f exactly)."""
import numpy as np


def _exact_by_test(xi, f):
    x = (xi + f).astype(np.float32)                      # FP32 add, one rounding
    return (x - xi).astype(np.float32) == f


def _exact_truth(xi, f):
    x = (xi + f).astype(np.float32)
    return x.astype(np.float64) == xi.astype(np.float64) + f.astype(np.float64)


def test_exactness_test_matches_the_exact_sum():
    rng = np.random.default_rng(7)
    n = 2_000_000
    xi = rng.integers(-8192, 8193, n).astype(np.float32)
    # fractions: grid-like (k/2, k/4, k/3, k/10 + 0.1 style) and random FP32 values
    kinds = [rng.integers(-2, 3, n) / 4.0, rng.integers(-1, 2, n) / 3.0,
             rng.uniform(-0.5, 0.5, n), (rng.integers(0, 3, n) / 3.0 + 0.1) % 1.0 - 0.5]
    for f in kinds:
        f = np.asarray(f, dtype=np.float32)
        assert np.array_equal(_exact_by_test(xi, f), _exact_truth(xi, f))
    # halves and quarters of the grid are always exact; generic fractions far from the
    # origin are not
    q = (rng.integers(-2, 3, n) / 4.0).astype(np.float32)
    assert _exact_by_test(xi, q).all()
    g = rng.uniform(-0.5, 0.5, n).astype(np.float32)
    far = np.abs(xi) >= 4096
    assert not _exact_by_test(xi[far], g[far]).all()


def test_split_offset_error_bound():
    """dx from the split point offsets, emulated step by step in FP32 (point as float-float
    (hi, lo) of x in pitch units, rint, integer offsets from an integer origin, one add for
    the fraction), within 2^-24 |dx| + 2^-25 pitch of the exact difference, for points
    anywhere on an 8192-pitch grid; the single FP32 offset from the tile origin is not."""
    rng = np.random.default_rng(3)
    n = 1_000_000
    x = rng.uniform(-2.0, 8194.0, n)                          # point, pitch units (FP64)
    v = rng.integers(0, 8192, n).astype(np.float64)           # visit on the probe grid
    org = rng.uniform(0.0, 8192.0, n)                         # tile's first point
    f32 = np.float32
    hi = x.astype(f32)
    lo = (x - hi.astype(np.float64)).astype(f32)
    ox = np.rint(org.astype(f32)).astype(f32)
    ix = np.rint(hi).astype(f32)
    fx = ((hi - ix).astype(f32) + lo).astype(f32)
    xi = (ix - ox).astype(f32)
    nv = (-(v.astype(f32) - ox)).astype(f32)
    dx = (((xi + nv).astype(f32)) + fx).astype(f32).astype(np.float64)
    exact = x - v
    err = np.abs(dx - exact)
    assert np.all(err <= 2.0 ** -24 * np.abs(exact) + 2.0 ** -25), err.max()
    # one FP32 offset per point from the tile origin: errors grow with the distance to it
    single = ((x - org).astype(f32) - (v - org).astype(f32)).astype(np.float64)
    assert np.max(np.abs(single - exact)) > 1e-4
