"""Seeded synthetic workloads: scan parameters, evaluation points and snapshot times.

This module holds input recipes only -- no part of the field computation.  Both the
CUDA library (through the Python binding) and the CPU oracle consume what it returns,
so it must stay free of the method's arithmetic.  The shapes follow the paper's setting
(Sec. 1-3): square probe grids scanned in raster, interleaved, serpentine or random
order, a Gaussian probe, constant D and Q0, and snapshots along the scan.

All lengths are metres, times seconds, D in m^2/s, Q0 in u/s.
"""
from dataclasses import dataclass, field, replace
from typing import Optional

import numpy as np

RASTER, SERPENTINE, INTERLEAVED, RANDOM, CUSTOM = 0, 1, 2, 3, 4
ORDER_NAMES = {RASTER: "raster", SERPENTINE: "serpentine", INTERLEAVED: "interleaved",
               RANDOM: "random", CUSTOM: "custom"}

PITCH = 0.5e-9      # probe pitch [m]
SIGMA = 0.1e-9      # Gaussian probe sigma [m]  (D_s = sigma^2)
D_REF = 6e-14       # diffusion coefficient [m^2/s]
Q0 = 1.0            # deposition rate [u/s]
DWELL = 1e-6        # dwell time [s]


@dataclass
class ScanSpec:
    nx: int
    ny: int
    pitch_m: float = PITCH
    sigma_m: float = SIGMA
    D_m2s: float = D_REF
    Q0: float = Q0
    dwell_s: float = DWELL
    flyback_s: float = 0.0
    order: int = RASTER
    interleave_stride: int = 1
    seed: int = 0
    keep_fraction: float = 1.0
    mask: Optional[np.ndarray] = None
    custom_visit: Optional[np.ndarray] = None
    dwell_per_visit: Optional[np.ndarray] = None
    blank_s: float = 0.0          # blanker dead time before a jump longer than one pitch [s]
    blank_s_per_m: float = 0.0    # and per metre of that jump [s/m]

    def with_(self, **kw):
        return replace(self, **kw)


@dataclass
class FieldJob:
    """One scan, the points the field is wanted at, and the snapshot times."""
    scan: ScanSpec
    pts_xy: np.ndarray          # [n_pts, 2] metres
    times: np.ndarray           # [n_t] seconds
    name: str = ""
    extra: dict = field(default_factory=dict)


def grid_points(n, step, origin=(0.0, 0.0)):
    """n x n points k * step (k = 0..n-1) in row-major order (y outer, x inner)."""
    k = np.arange(n, dtype=np.float64) * step
    yy, xx = np.meshgrid(k + origin[1], k + origin[0], indexing="ij")
    return np.stack([xx.reshape(-1), yy.reshape(-1)], axis=1)


def n_visits(spec: ScanSpec) -> int:
    if spec.custom_visit is not None and spec.order == CUSTOM:
        return len(spec.custom_visit)
    if spec.mask is not None:
        return int(np.count_nonzero(spec.mask))
    n = spec.nx * spec.ny
    if spec.keep_fraction < 1.0:
        return max(int(np.floor(spec.keep_fraction * n + 0.5)), 1)
    return n


def small_raster_16():
    """16x16 raster, field on the probe grid at the end of each of the 256 dwells."""
    s = ScanSpec(16, 16)
    times = (np.arange(256, dtype=np.float64) + 1.0) * s.dwell_s
    return FieldJob(s, grid_points(16, s.pitch_m), times, name="raster16_probe-grid_256-snapshots")


def raster_64_supersampled():
    """64x64 raster, field on a 2x supersampled 128x128 grid (pitch/2) at the end of
    every scan row (64 snapshots)."""
    s = ScanSpec(64, 64)
    times = 64.0 * (np.arange(64, dtype=np.float64) + 1.0) * s.dwell_s
    return FieldJob(s, grid_points(128, s.pitch_m / 2), times,
                    name="raster64_pts128x128_64-row-snapshots")


def precision_study(order, d_index, seed=3):
    """256x256 grid, one of the four scan orders, D from 8 seeded log-uniform draws in
    [1e-15, 1e-12]; field on the probe grid at the end of the scan and at 16x that time."""
    rng = np.random.default_rng(seed)
    Ds = 10.0 ** rng.uniform(-15.0, -12.0, size=8)
    stride = 4 if order == INTERLEAVED else 1
    s = ScanSpec(256, 256, D_m2s=float(Ds[d_index]), order=order, interleave_stride=stride,
                 seed=seed * 1000 + 17)
    n = 256 * 256
    times = np.array([n * s.dwell_s, 16.0 * n * s.dwell_s])
    return FieldJob(s, grid_points(256, s.pitch_m), times,
                    name="grid256_%s_D%.2e" % (ORDER_NAMES[order], s.D_m2s))


def batched_specs(n_scans=512, seed=4, n_min=32, n_max=128):
    """Scan descriptions of the uneven batch: n ~ U{n_min..n_max}; D log-uniform
    [1e-15, 1e-12] m^2/s; dwell log-uniform [1e-7, 1e-5] s; sigma ~ U[0.05, 0.2] nm; keep
    fraction f ~ U[0.1, 1] of the positions, visited in seeded random order."""
    rng = np.random.default_rng(seed)
    specs = []
    for k in range(n_scans):
        n = int(rng.integers(n_min, n_max + 1))
        D = float(10.0 ** rng.uniform(-15.0, -12.0))
        tau = float(10.0 ** rng.uniform(-7.0, -5.0))
        sigma = float(rng.uniform(0.05e-9, 0.2e-9))
        f = float(rng.uniform(0.1, 1.0))
        specs.append(ScanSpec(n, n, sigma_m=sigma, D_m2s=D, dwell_s=tau, order=RANDOM,
                              seed=seed * 100003 + k, keep_fraction=f))
    return specs


def batched_scans(n_scans=512, seed=4, n_min=32, n_max=128):
    """The uneven batch of batched_specs, each evaluated on its n x n probe grid at the
    end of its scan."""
    jobs = []
    for k, s in enumerate(batched_specs(n_scans, seed, n_min, n_max)):
        nv = n_visits(s)
        jobs.append(FieldJob(s, grid_points(s.nx, s.pitch_m), np.array([nv * s.dwell_s]),
                             name="batch%03d_n%d" % (k, s.nx)))
    return jobs


def live_mode(n, frame_s, dwell_s=DWELL):
    """n x n raster, field on the probe grid at every frame time across the scan (the
    runtime-vs-probe-count setting of Fig. 2: frame time delta_t, pixel = probe pitch)."""
    s = ScanSpec(n, n, dwell_s=dwell_s)
    end = n * n * dwell_s
    times = np.arange(1, int(np.floor(end / frame_s + 1e-9)) + 1, dtype=np.float64) * frame_s
    return FieldJob(s, grid_points(n, s.pitch_m), times, name="live%dx%d_frame%.0eus" % (n, n, frame_s * 1e6))


def sample_pairs(n_pts, n_t, count, seed):
    """Seeded (point index, time index) pairs, without replacement where possible."""
    rng = np.random.default_rng(seed)
    total = n_pts * n_t
    flat = rng.choice(total, size=min(count, total), replace=False)
    return flat % n_pts, flat // n_pts


def causal_pairs(visit_starts, times, n_pts):
    """Number of causal (source, point, snapshot) triples: sources with t_i < t."""
    visit_starts = np.sort(np.asarray(visit_starts))
    return int(n_pts * np.searchsorted(visit_starts, np.asarray(times), side="left").sum())
