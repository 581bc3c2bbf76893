"""Scan orders and visit times, written independently for the oracle (test infrastructure).

The paper (Sec. 1) names raster scans, alternating/interleaved scans that skip fixed
grid points, random scans, and subsampling with a beam blanker; Eq. 5 sums the probes
in the order they are visited, each starting when the previous dwell ends (Sec. 2).
Readings used here (they are restated in the design notes):
  * grid index g = iy * nx + ix, probe at (ix * pitch, iy * pitch);
  * raster: rows in order, each left to right;
  * serpentine ("alternating"): even rows left to right, odd rows right to left;
  * interleaved with stride S: S*S passes over the sub-lattices (py, px) in raster
    order of (py, px); each pass visits the positions with iy % S == py and
    ix % S == px in raster order;
  * random: Fisher-Yates shuffle driven by SplitMix64 (Steele, Lea & Flood, 2014);
    the swap index for position i is floor(u * (i + 1) / 2^64) for the next 64-bit
    output u;
  * keep fraction f < 1: the kept set is the first round(f * N) entries of that
    seeded permutation; the random order visits them in permutation order, the
    other orders visit them in their own sequence;
  * an explicit mask removes positions whose mask entry is 0;
  * visit k starts at t_k = k * tau with a uniform dwell and no dead time; otherwise
    t_{k+1} = t_k + tau_k (+ flyback when raster/serpentine visits change row)
    (+ the blanker's travel time, blank + blank_per_m * jump length in metres, when the
    beam jumps more than one pitch to the next visit: the blanker of Sec. 1 keeps the beam
    off while the probe moves over positions it does not visit).
"""
import math

import numpy as np

RASTER, SERPENTINE, INTERLEAVED, RANDOM, CUSTOM = 0, 1, 2, 3, 4
_M64 = (1 << 64) - 1


def splitmix64(seed):
    """Generator of SplitMix64 outputs for a 64-bit seed."""
    state = seed & _M64
    while True:
        state = (state + 0x9E3779B97F4A7C15) & _M64
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
        yield z ^ (z >> 31)


def permutation(n, seed):
    """Fisher-Yates permutation of range(n) driven by SplitMix64(seed)."""
    perm = list(range(n))
    gen = splitmix64(seed)
    for i in range(n - 1, 0, -1):
        j = (next(gen) * (i + 1)) >> 64
        perm[i], perm[j] = perm[j], perm[i]
    return perm


def base_order(nx, ny, order, stride=1, seed=0, custom=None):
    if order == RASTER:
        return [iy * nx + ix for iy in range(ny) for ix in range(nx)]
    if order == SERPENTINE:
        out = []
        for iy in range(ny):
            cols = range(nx) if iy % 2 == 0 else range(nx - 1, -1, -1)
            out.extend(iy * nx + ix for ix in cols)
        return out
    if order == INTERLEAVED:
        out = []
        for py in range(stride):
            for px in range(stride):
                for iy in range(py, ny, stride):
                    for ix in range(px, nx, stride):
                        out.append(iy * nx + ix)
        return out
    if order == RANDOM:
        return permutation(nx * ny, seed)
    if order == CUSTOM:
        return [int(g) for g in custom]
    raise ValueError("unknown order")


def visit_order(nx, ny, order, stride=1, seed=0, keep_fraction=1.0, mask=None, custom=None):
    """Grid indices in visit order."""
    seq = base_order(nx, ny, order, stride, seed, custom)
    if mask is not None:
        m = np.asarray(mask).reshape(-1)
        seq = [g for g in seq if m[g] != 0]
    if keep_fraction < 1.0:
        n = nx * ny
        k = int(np.floor(keep_fraction * n + 0.5))
        k = max(k, 1)
        perm = permutation(n, seed)
        if order == RANDOM:
            seq = perm[:k]
        else:
            kept = set(perm[:k])
            seq = [g for g in seq if g in kept]
    return seq


def visit_times(visits, nx, order, dwell, flyback=0.0, dwell_per_visit=None, pitch=0.0,
                blank=0.0, blank_per_m=0.0):
    """Start time t_k [s] and dwell tau_k [s] of each visit."""
    n = len(visits)
    if dwell_per_visit is None and flyback == 0.0 and blank == 0.0 and blank_per_m == 0.0:
        ts = [k * dwell for k in range(n)]
        return np.array(ts, dtype=np.float64), np.full(n, dwell, dtype=np.float64)
    taus = (np.full(n, dwell, dtype=np.float64) if dwell_per_visit is None
            else np.asarray(dwell_per_visit, dtype=np.float64))
    ts = np.zeros(n, dtype=np.float64)
    t = 0.0
    for k in range(n):
        ts[k] = t
        t = t + float(taus[k])
        if k + 1 == n:
            break
        here, there = int(visits[k]), int(visits[k + 1])
        if flyback != 0.0 and order in (RASTER, SERPENTINE) and here // nx != there // nx:
            t = t + flyback
        if blank != 0.0 or blank_per_m != 0.0:
            jx = there % nx - here % nx
            jy = there // nx - here // nx
            if jx * jx + jy * jy > 1:                  # not the neighbouring position
                t = t + (blank + blank_per_m * (pitch * math.sqrt(jx * jx + jy * jy)))
    return ts, taus


def sources(nx, ny, pitch, dwell, order=RASTER, stride=1, seed=0, keep_fraction=1.0,
            mask=None, custom=None, flyback=0.0, dwell_per_visit=None, blank=0.0, blank_per_m=0.0):
    """Probe visits as (xs, ys, ts, taus) arrays in SI units, plus the visit list."""
    v = visit_order(nx, ny, order, stride, seed, keep_fraction, mask, custom)
    ts, taus = visit_times(v, nx, order, dwell, flyback, dwell_per_visit, pitch, blank, blank_per_m)
    g = np.asarray(v, dtype=np.int64)
    xs = (g % nx).astype(np.float64) * pitch
    ys = (g // nx).astype(np.float64) * pitch
    return xs, ys, ts, taus, g
