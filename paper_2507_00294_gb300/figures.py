"""Headless cumulative-damage maps (the start-of-scan / end-of-scan pictures of Fig. 1),
written as binary PGM images.  There is no graphics stack: the field is computed by the
library (dd_field_at_times) and scaled to 8-bit grey levels on the host."""
import os

import numpy as np

from . import binding as b
from . import workloads as w


def gray_levels(field, log_decades=6.0):
    """8-bit grey levels of a 2-D field: log10 of the field relative to its maximum, over
    `log_decades` decades (values below that floor are black, the maximum is white)."""
    f = np.asarray(field, dtype=np.float64)
    top = f.max()
    if top > 0:
        v = np.log10(np.maximum(f, top * 10.0 ** -log_decades) / top) / log_decades + 1.0
    else:
        v = np.zeros_like(f)
    return np.clip(np.round(v * 255.0), 0, 255).astype(np.uint8)


def write_pgm(path, img):
    """Binary PGM (P5) of an 8-bit image [rows, cols]."""
    img = np.ascontiguousarray(img, dtype=np.uint8)
    with open(path, "wb") as fh:
        fh.write(b"P5\n%d %d\n255\n" % (img.shape[1], img.shape[0]))
        fh.write(img.tobytes())
    return path


def fig1_field(spec, supersample=2, early_fraction=0.1, prec="mixed"):
    """Field on a `supersample`-times finer grid over the scanned area after
    `early_fraction` of the visits and at the end of the scan: (points [n*n, 2] metres,
    times [2] seconds, field [2, n, n] u/m^2)."""
    n = max(spec.nx, spec.ny) * supersample
    pts = w.grid_points(n, spec.pitch_m / supersample)
    scan = b.Scan(spec)
    _, ts, taus = scan.visits()
    k = max(1, int(len(ts) * early_fraction))
    times = np.array([ts[k - 1] + taus[k - 1], ts[-1] + taus[-1]])
    field = b.dd_field_at_times(scan, pts, times, prec).reshape(2, n, n)
    scan.close()
    return pts, times, field


def fig1_maps(spec, out_dir, supersample=2, early_fraction=0.1, prec="mixed"):
    """The two maps of fig1_field as PGM files in out_dir; returns their paths."""
    os.makedirs(out_dir, exist_ok=True)
    _, _, field = fig1_field(spec, supersample, early_fraction, prec)
    return [write_pgm(os.path.join(out_dir, name), gray_levels(field[i]))
            for i, name in enumerate(("damage_early.pgm", "damage_end.pgm"))]
