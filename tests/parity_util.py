"""Helpers for the GPU-vs-oracle parity tests (inputs come from workloads.py; expected
values only from oracle/)."""
import numpy as np

import oracle
from oracle import scan as oscan

FP64_RTOL = 1e-12          # GPU FP64 vs oracle, every point with |psi| >= 1e-290
MIXED_RTOL = 1e-5          # GPU FP32-mixed vs oracle where psi >= 1e-6 of the map's peak


def oracle_problem(spec):
    """The scan as the oracle evaluates it, with time measured in dwells.

    Eq. 1/2 depend on time only through D (t - t_i), D tau_i and Q0 / D, so measuring
    time in units of the dwell tau (t' = t / tau, D' = D tau, Q0' = Q0 tau) leaves every
    field value unchanged, in u/m^2.  It does change the oracle's rounding: in seconds a
    start time t_k = k tau carries an FP64 rounding of ulp(t_k), which long into a scan is
    no longer small against a one-dwell lag (1.4e-11 of it at t = 65 ms, tau = 1 us: the
    dose of a 256 x 256 scan at its last visits then moves by 3e-12), whereas in dwells
    t'_k = k and every lag on the dwell lattice are exact.  Returns (sources with times in
    dwells, Ds, D', Q0')."""
    tau = spec.dwell_s
    dpv = None if spec.dwell_per_visit is None else np.asarray(spec.dwell_per_visit, np.float64) / tau
    xs, ys, ts, taus, _ = oscan.sources(
        spec.nx, spec.ny, spec.pitch_m, 1.0, order=spec.order,
        stride=spec.interleave_stride, seed=spec.seed, keep_fraction=spec.keep_fraction,
        mask=spec.mask, custom=spec.custom_visit, flyback=spec.flyback_s / tau,
        dwell_per_visit=dpv, blank=spec.blank_s / tau, blank_per_m=spec.blank_s_per_m / tau)
    return oracle.Sources(xs, ys, ts, taus), spec.sigma_m ** 2, spec.D_m2s * tau, spec.Q0 * tau


def raster_sources(spec):
    """Sources of a full raster scan with a uniform dwell, from the definition (visit k is
    grid index k and starts at k * dwell) in vectorised form, in SI units, for grids too
    large for the oracle's list-based scan builder; equal to the oracle's SI sources on such
    specs (checked in test_oracle_scan.py)."""
    assert spec.order == oscan.RASTER and spec.keep_fraction == 1.0 and spec.mask is None
    assert spec.flyback_s == 0.0 and spec.dwell_per_visit is None
    n = spec.nx * spec.ny
    g = np.arange(n, dtype=np.int64)
    ts = np.arange(n, dtype=np.int64).astype(np.float64) * spec.dwell_s
    return oracle.Sources((g % spec.nx).astype(np.float64) * spec.pitch_m,
                          (g // spec.nx).astype(np.float64) * spec.pitch_m, ts,
                          np.full(n, spec.dwell_s, dtype=np.float64))


def oracle_field(spec, pts, times, problem=None):
    src, Ds, D, Q0 = problem or oracle_problem(spec)
    return oracle.field(src, Ds, D, Q0, pts[:, 0], pts[:, 1], np.asarray(times) / spec.dwell_s)


def oracle_pairs(spec, pts, times, ip, it, problem=None):
    src, Ds, D, Q0 = problem or oracle_problem(spec)
    return oracle.field_pairs(src, Ds, D, Q0, pts[ip, 0], pts[ip, 1], np.asarray(times)[it] / spec.dwell_s)


def oracle_dose(spec, targets=None, problem=None):
    src, Ds, D, Q0 = problem or oracle_problem(spec)
    return oracle.dose(src, Ds, D, Q0, targets=targets)


def peak_lower_bound(spec, times, problem=None):
    """Oracle field at the probe visited last before each time: <= that map's peak."""
    src, Ds, D, Q0 = problem or oracle_problem(spec)
    tt = np.asarray(times) / spec.dwell_s
    idx = np.clip(np.searchsorted(src.ts, tt, side="left") - 1, 0, src.n - 1)
    return oracle.field_pairs(src, Ds, D, Q0, src.xs[idx], src.ys[idx], tt)


def assert_fp64(got, ref, what=""):
    got = np.asarray(got); ref = np.asarray(ref)
    assert got.shape == ref.shape
    zero = ref == 0.0
    assert np.all(got[zero] == 0.0), what + ": nonzero where the oracle is exactly 0"
    m = np.abs(ref) >= 1e-290
    rel = np.abs(got[m] - ref[m]) / np.abs(ref[m])
    worst = rel.max() if rel.size else 0.0
    if worst > FP64_RTOL:
        k = np.argwhere(m)[np.argmax(rel)]
        raise AssertionError("%s: FP64 max rel err %.3e at index %s (got %.17g, oracle %.17g)"
                             % (what, worst, tuple(int(i) for i in k), got[tuple(k)], ref[tuple(k)]))
    return worst


def assert_mixed(got, ref, peak, what=""):
    """peak: per-row (snapshot) peak or a lower bound of it, shape [n_t] or scalar."""
    got = np.asarray(got); ref = np.asarray(ref)
    thr = 1e-6 * np.asarray(peak)
    if ref.ndim == 2:
        thr = np.broadcast_to(np.reshape(thr, (-1, 1)), ref.shape)
    assert np.all(got[ref == 0.0] == 0.0), what + ": nonzero where the oracle is exactly 0"
    m = (ref >= thr) & (ref > 0.0)
    assert m.sum() > 0
    rel = np.abs(got[m] - ref[m]) / ref[m]
    worst = rel.max()
    if worst > MIXED_RTOL:
        k = np.argwhere(m)[np.argmax(rel)]
        raise AssertionError("%s: mixed max rel err %.3e (median %.3e) at index %s (got %.9g, oracle %.9g)"
                             % (what, worst, np.median(rel), tuple(int(i) for i in k), got[tuple(k)],
                                ref[tuple(k)]))
    return worst
