"""Pins for the oracle's single-probe field (Eq. 1-4) and cumulative field (Eq. 5).

None of these retype the oracle's formulas.  They check it against:
  * the time integral of the 2D heat kernel for a Gaussian deposit of variance D_s per
    axis, released at rate Q0 during the dwell (Fick's law, Eq. 6, solved by Green's
    function), integrated by mpmath at 30 digits;
  * conservation of the deposited amount (area integral = Q0 x time the beam was on);
  * the PDE of Eq. 6 itself, by finite differences;
  * the late-time point-source limit;
  * brute-force sums of that Green's-function integral over tiny scans (Eq. 5);
  * symmetries of the cumulative field (mirror, time shift, scale invariance).
"""
import math

import numpy as np
import pytest

import oracle
from oracle import scan

mp = pytest.importorskip("mpmath")
integrate = pytest.importorskip("scipy.integrate")

Ds = (0.1e-9) ** 2
D = 6e-14
Q0 = 1.0
TAU = 1e-6


def green_time_integral(rho2, dt, tau, Ds_, D_, Q0_, dps=30):
    """int over the beam-on window of Q0 * 2D Gaussian of variance Ds + 2D(age) per axis."""
    mp.mp.dps = dps
    rho2, dt, tau = mp.mpf(rho2), mp.mpf(dt), mp.mpf(tau)
    Ds_, D_, Q0_ = mp.mpf(Ds_), mp.mpf(D_), mp.mpf(Q0_)
    if dt <= 0:
        return mp.mpf(0)
    lo = dt - tau if dt > tau else mp.mpf(0)      # ages of the deposits still present

    def kern(age):
        var = Ds_ + 2 * D_ * age
        return Q0_ / (2 * mp.pi * var) * mp.e ** (-rho2 / (2 * var))
    # split at a few ages so the quadrature resolves the early, sharply peaked part
    # (small ages for points near the probe, the largest ages for far points)
    # mpmath's quad stops on an absolute tolerance, so integrate kern / peak where the
    # peak is the larger end value, then scale back
    peak = max(kern(lo), kern(dt))
    span = dt - lo
    fr = sorted(set([mp.mpf(10) ** -k for k in range(1, 14)]
                    + [1 - mp.mpf(10) ** -k for k in range(1, 14)] + [mp.mpf(1) / 2]))
    pts = [lo] + [lo + span * f for f in fr] + [dt]
    return peak * mp.quad(lambda a: kern(a) / peak, pts)


CASES = [(r, dt, tau) for r in (0.0, 0.05e-9, 0.2e-9, 0.5e-9, 1.3e-9, 3e-9)
         for dt, tau in ((0.3e-6, 1e-6), (1e-6, 1e-6), (1.7e-6, 1e-6), (40e-6, 1e-6),
                         (5000e-6, 1e-6), (2.5e-7, 1e-7))]


@pytest.mark.parametrize("r,dt,tau", CASES)
def test_phi_equals_green_function_time_integral(r, dt, tau):
    ref = float(green_time_integral(r * r, dt, tau, Ds, D, Q0))
    got = float(oracle.phi(r * r, dt, tau, Ds, D, Q0))
    if ref < 1e-280:
        assert got < 1e-270
        return
    assert abs(got / ref - 1.0) < 1e-12, (r, dt, tau, got, ref)


@pytest.mark.parametrize("r", [0.0, 0.15e-9])
@pytest.mark.parametrize("lag", [0.5, 1e3, 1e5, 1e7, 6.7e7])
def test_phi_long_after_the_dwell_slow_diffusion(r, lag):
    """Eq. 3/4 (rho = 0) and Eq. 2 long after the dwell, with slow diffusion
    (D tau / pitch^2 = 1e-6 at a 0.5 nm pitch): the logarithm's argument is then
    1 + O(1e-8), where forming the ratio before the logarithm would lose ~1e-8 of relative
    accuracy; against the Green's-function time integral at 40 digits."""
    D_slow = 1e-6 * (0.5e-9) ** 2 / TAU
    dt = lag * TAU
    ref = float(green_time_integral(r * r, dt, TAU, Ds, D_slow, Q0, dps=40))
    got = float(oracle.phi(r * r, dt, TAU, Ds, D_slow, Q0))
    assert abs(got / ref - 1.0) < 1e-13, (r, lag, got, ref)


def test_phi_causal_and_continuous_at_rho0():
    assert oracle.phi(1e-20, 0.0, TAU, Ds, D, Q0) == 0.0          # t = t_i
    assert oracle.phi(1e-20, -1e-7, TAU, Ds, D, Q0) == 0.0        # not started
    for dt in (0.5e-6, 1e-6, 3e-6, 1e-3):
        p0 = float(oracle.phi(0.0, dt, TAU, Ds, D, Q0))
        pe = float(oracle.phi(1e-12 * Ds, dt, TAU, Ds, D, Q0))
        assert abs(pe / p0 - 1.0) < 1e-9


@pytest.mark.parametrize("dt,tau", [(0.4e-6, 1e-6), (1e-6, 1e-6), (3e-6, 1e-6), (2e-4, 1e-6)])
def test_mass_conservation_single_probe(dt, tau):
    # 2 pi int_0^inf phi(rho) rho d rho = Q0 * (time the beam was on)
    f = lambda r: 2 * math.pi * r * float(oracle.phi(r * r, dt, tau, Ds, D, Q0))
    width = math.sqrt(2 * Ds + 4 * D * dt)
    brk = [0.0, 0.5 * math.sqrt(Ds), 2 * math.sqrt(Ds), width, 4 * width, 12 * width]
    total = sum(integrate.quad(f, a, b, epsabs=0, epsrel=1e-12, limit=200)[0]
                for a, b in zip(brk[:-1], brk[1:]))
    assert abs(total / (Q0 * min(dt, tau)) - 1.0) < 1e-9


@pytest.mark.parametrize("dt", [0.3e-6, 0.8e-6, 2.0e-6, 9e-6])
@pytest.mark.parametrize("r", [0.07e-9, 0.3e-9, 0.9e-9])
def test_fick_pde_residual(dt, r):
    # d phi/dt - D lap phi = Q0 * Gaussian(D_s) while the beam is on, 0 after (Eq. 6)
    tau = 1e-6
    def ph(x, y, t):
        return float(oracle.phi(x * x + y * y, t, tau, Ds, D, Q0))
    x0, y0 = r * 0.6, r * 0.8
    ht = 1e-4 * dt
    hx = 2e-3 * math.sqrt(Ds + 2 * D * dt)
    dphidt = (ph(x0, y0, dt + ht) - ph(x0, y0, dt - ht)) / (2 * ht)
    c = ph(x0, y0, dt)
    lap = (ph(x0 + hx, y0, dt) + ph(x0 - hx, y0, dt) + ph(x0, y0 + hx, dt)
           + ph(x0, y0 - hx, dt) - 4 * c) / (hx * hx)
    src = Q0 / (2 * math.pi * Ds) * math.exp(-(x0 * x0 + y0 * y0) / (2 * Ds)) if dt < tau else 0.0
    scale = abs(dphidt) + abs(D * lap) + abs(src)
    assert abs(dphidt - D * lap - src) < 2e-5 * scale


def test_late_time_point_source_limit():
    # t >> tau: phi -> Q0 tau / (4 pi D (t - t_i)) exp(-rho^2 / (4 D (t - t_i)))
    for r in (0.0, 1e-9, 5e-9):
        for dt in (1e-3, 1e-2):
            got = float(oracle.phi(r * r, dt, TAU, Ds, D, Q0))
            approx = Q0 * TAU / (4 * math.pi * D * dt) * math.exp(-r * r / (4 * D * dt))
            assert abs(got / approx - 1.0) < 5 * TAU / dt


def brute_field(xs, ys, ts, taus, px, py, t):
    return float(sum(green_time_integral((px - x) ** 2 + (py - y) ** 2, t - ti, tau, Ds, D, Q0)
                     for x, y, ti, tau in zip(xs, ys, ts, taus)))


def test_cumulative_field_brute_force_tiny_scans():
    p = 0.5e-9
    for nx, ny, order in ((1, 1, scan.RASTER), (2, 1, scan.RASTER), (3, 1, scan.SERPENTINE),
                          (2, 2, scan.RANDOM)):
        xs, ys, ts, taus, _ = scan.sources(nx, ny, p, TAU, order=order, seed=7)
        src = oracle.Sources(xs, ys, ts, taus)
        pts = np.array([[0.0, 0.0], [0.25e-9, 0.1e-9], [1.0e-9, 0.5e-9], [3e-9, -1e-9]])
        times = np.array([0.5e-6, 1.0e-6, 2.5e-6, 7e-6])
        got = oracle.field(src, Ds, D, Q0, pts[:, 0], pts[:, 1], times)
        # the (point, time) pair list form, on every pair, against the same brute force
        ip_all, it_all = np.meshgrid(np.arange(len(pts)), np.arange(len(times)))
        pairs = oracle.field_pairs(src, Ds, D, Q0, pts[ip_all.ravel(), 0], pts[ip_all.ravel(), 1],
                                   times[it_all.ravel()]).reshape(len(times), len(pts))
        for it, t in enumerate(times):
            for ip in range(len(pts)):
                ref = brute_field(xs, ys, ts, taus, pts[ip, 0], pts[ip, 1], t)
                for val in (got[it, ip], pairs[it, ip]):
                    if ref < 1e-250:
                        assert val < 1e-240
                    else:
                        assert abs(val / ref - 1.0) < 1e-12


def test_raster_field_mirror_symmetry():
    # mirroring x -> (nx-1)p - x maps the raster scan onto the right-to-left raster
    nx, ny, p = 6, 5, 0.5e-9
    xs, ys, ts, taus, g = scan.sources(nx, ny, p, TAU)
    mirrored = [(gi // nx) * nx + (nx - 1 - gi % nx) for gi in g]
    xm, ym, tm, taum, _ = scan.sources(nx, ny, p, TAU, order=scan.CUSTOM, custom=mirrored)
    rng = np.random.default_rng(5)
    px = rng.uniform(-1e-9, (nx + 1) * p, 40)
    py = rng.uniform(-1e-9, (ny + 1) * p, 40)
    times = np.array([3e-6, 17e-6, 30e-6, 200e-6])
    a = oracle.field(oracle.Sources(xs, ys, ts, taus), Ds, D, Q0, px, py, times)
    b = oracle.field(oracle.Sources(xm, ym, tm, taum), Ds, D, Q0, (nx - 1) * p - px, py, times)
    assert np.max(np.abs(a / b - 1.0)) < 1e-12


def test_time_shift_and_scale_invariance():
    nx, ny, p = 4, 3, 0.5e-9
    xs, ys, ts, taus, _ = scan.sources(nx, ny, p, TAU, order=scan.SERPENTINE)
    px = np.array([0.1e-9, 0.7e-9, 1.6e-9]); py = np.array([0.0, 0.4e-9, 1.1e-9])
    times = np.array([2.2e-6, 5e-6, 12e-6, 40e-6])
    base = oracle.field(oracle.Sources(xs, ys, ts, taus), Ds, D, Q0, px, py, times)
    shifted = oracle.field(oracle.Sources(xs, ys, ts + 3e-3, taus), Ds, D, Q0, px, py, times + 3e-3)
    assert np.max(np.abs(shifted / base - 1.0)) < 1e-9
    lam = 3.0   # lengths x lam, D x lam^2: 4 pi D psi / Q0 is unchanged
    scaled = oracle.field(oracle.Sources(xs * lam, ys * lam, ts, taus), Ds * lam ** 2, D * lam ** 2, Q0,
                          px * lam, py * lam, times)
    assert np.max(np.abs(scaled * lam ** 2 / base - 1.0)) < 1e-12


def test_field_is_sum_over_visits_and_dose_matches_field():
    nx, ny, p = 5, 4, 0.5e-9
    xs, ys, ts, taus, _ = scan.sources(nx, ny, p, TAU, order=scan.INTERLEAVED, stride=2)
    src = oracle.Sources(xs, ys, ts, taus)
    # the dwell-start dose of visit j is the field at (r_j, t_j)
    dose = oracle.dose(src, Ds, D, Q0)
    fp = oracle.field_pairs(src, Ds, D, Q0, xs, ys, ts)
    assert dose[0] == 0.0
    assert np.max(np.abs(dose[1:] / fp[1:] - 1.0)) < 1e-15
    # splitting the visits into two groups and adding the two fields gives the same field
    px = np.array([0.3e-9, 1.2e-9]); py = np.array([0.2e-9, 0.9e-9]); times = np.array([9e-6, 25e-6])
    whole = oracle.field(src, Ds, D, Q0, px, py, times)
    part = lambda sl: oracle.field(oracle.Sources(xs[sl], ys[sl], ts[sl], taus[sl]), Ds, D, Q0, px, py, times)
    assert np.max(np.abs((part(slice(0, 7)) + part(slice(7, None))) / whole - 1.0)) < 1e-14


@pytest.mark.parametrize("r,lag", [(0.0, 1.0), (0.5e-9, 1.0), (0.5e-9, 2.0), (1.1e-9, 37.0), (3e-9, 65015.0),
                                   (0.7e-9, 0.4)])
def test_phi_in_dwell_units(r, lag):
    """Time measured in dwells (t' = t / tau, D' = D tau, Q0' = Q0 tau), the form the parity
    tests hand to the oracle, gives phi unchanged: Eq. 1/2 see time only through D (t - t_i),
    D tau and Q0 / D."""
    si = float(oracle.phi(r * r, lag * TAU, TAU, Ds, D, Q0))
    dw = float(oracle.phi(r * r, lag, 1.0, Ds, D * TAU, Q0 * TAU))
    assert dw == pytest.approx(si, rel=2e-14)


def test_dose_late_in_a_long_scan_against_40_digits():
    """Dwell-start dose of visit 65016 of a 256 x 256 serpentine scan (D = 5.58e-14 m^2/s,
    0.065 s into the scan): the oracle fed with time in dwells against a 40-digit mpmath
    sum of Eq. 2 over all 65016 earlier visits.  With start times in seconds, each lag
    carries the rounding of t_k (1.4e-11 of a dwell here), and the oracle was off by
    3.3e-12 -- beyond the FP64 parity tolerance."""
    import sys
    import os
    sys.path.insert(0, os.path.dirname(__file__))
    from parity_util import oracle_dose
    from paper_2507_00294_gb300 import workloads as w
    spec = w.precision_study(w.SERPENTINE, 3).scan
    j = 65016
    got = float(oracle_dose(spec, np.array([j]))[0])
    order = scan.visit_order(spec.nx, spec.ny, spec.order)
    mp.mp.dps = 40
    p, Dm, Dsm, tau = mp.mpf(spec.pitch_m), mp.mpf(spec.D_m2s), mp.mpf(spec.sigma_m) ** 2, mp.mpf(spec.dwell_s)
    gj = order[j]
    acc = mp.mpf(0)
    for i in range(j):
        gi = order[i]
        r2 = ((gj % spec.nx - gi % spec.nx) ** 2 + (gj // spec.nx - gi // spec.nx) ** 2) * p * p
        lag = j - i                       # beam of visit i off since (lag - 1) dwells (Eq. 2)
        acc += mp.e1(r2 / (2 * Dsm + 4 * Dm * lag * tau)) - mp.e1(r2 / (2 * Dsm + 4 * Dm * (lag - 1) * tau))
    want = float(acc * spec.Q0 / (4 * mp.pi * Dm))
    assert got == pytest.approx(want, rel=2e-14)
