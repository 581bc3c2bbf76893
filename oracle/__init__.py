"""CPU oracle for the cumulative damage-diffusion field.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this package; the product library never does, and the
two share no code.  The arithmetic lives in ``dd_oracle.c`` (plain C, FP64, SI units);
this module compiles it with gcc on first use and marshals numpy arrays through ctypes.
Scan orders and visit times are reimplemented independently in ``oracle/scan.py``.

Paper: Javadi Rad et al., "Fast Simulation of Damage Diffusion Distribution in STEM",
Sec. 2, Eq. 1-5.
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dd_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libdd_oracle.so")
_lock = threading.Lock()
_lib = None

_D = ctypes.c_double
_I64 = ctypes.c_int64
_PD = ctypes.POINTER(ctypes.c_double)
_PI64 = ctypes.POINTER(ctypes.c_int64)


def build(force=False):
    """Compile dd_oracle.c into oracle/_build/libdd_oracle.so (gcc, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-fno-fast-math",
           "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        lib.ddo_e1.restype = _D
        lib.ddo_e1.argtypes = [_D]
        lib.ddo_e1_diff.restype = _D
        lib.ddo_e1_diff.argtypes = [_D, _D]
        lib.ddo_e1_diff_quad.restype = _D
        lib.ddo_e1_diff_quad.argtypes = [_D, _D]
        lib.ddo_e1_diff_log.restype = _D
        lib.ddo_e1_diff_log.argtypes = [_D, _D]
        lib.ddo_phi.restype = _D
        lib.ddo_phi.argtypes = [_D, _D, _D, _D, _D, _D]
        lib.ddo_field.restype = None
        lib.ddo_field.argtypes = [_I64, _PD, _PD, _PD, _PD, _D, _D, _D,
                                  _I64, _PD, _PD, _I64, _PD, _PD, ctypes.c_int]
        lib.ddo_field_pairs.restype = None
        lib.ddo_field_pairs.argtypes = [_I64, _PD, _PD, _PD, _PD, _D, _D, _D,
                                        _I64, _PD, _PD, _PD, _PD, ctypes.c_int]
        lib.ddo_dose.restype = None
        lib.ddo_dose.argtypes = [_I64, _PD, _PD, _PD, _PD, _D, _D, _D,
                                 _I64, _PI64, _PD, ctypes.c_int]
        lib.ddo_max_threads.restype = ctypes.c_int
        _lib = lib
        return lib


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ptr(a):
    return a.ctypes.data_as(_PD)


def max_threads():
    return int(_load().ddo_max_threads())


def e1(x):
    """E_1(x) (definition below Eq. 2): A&S 5.1.11 series / A&S 5.1.22 fraction."""
    lib = _load()
    x = np.asarray(x, dtype=np.float64)
    return np.vectorize(lib.ddo_e1, otypes=[np.float64])(x)


def e1_diff(a, b):
    """E_1(a) - E_1(b) for 0 <= a <= b."""
    lib = _load()
    return np.vectorize(lib.ddo_e1_diff, otypes=[np.float64])(np.asarray(a, float), np.asarray(b, float))


def e1_diff_quad(a, b):
    """int_a^b e^-u/u du by adaptive Gauss-Legendre quadrature in ln u."""
    lib = _load()
    return np.vectorize(lib.ddo_e1_diff_quad, otypes=[np.float64])(np.asarray(a, float), np.asarray(b, float))


def e1_diff_log(a, ell):
    """E_1(a) - E_1(a e^ell) by quadrature of int_0^ell exp(-a e^y) dy."""
    lib = _load()
    return np.vectorize(lib.ddo_e1_diff_log, otypes=[np.float64])(np.asarray(a, float), np.asarray(ell, float))


def phi(rho2, dt, tau, Ds, D, Q0):
    """Single-probe field, Eq. 1-4 (SI units): rho2 [m^2], dt = t - t_i [s]."""
    lib = _load()
    return np.vectorize(lambda r, t, ta: lib.ddo_phi(r, t, ta, Ds, D, Q0), otypes=[np.float64])(
        np.asarray(rho2, float), np.asarray(dt, float), np.asarray(tau, float))


class Sources:
    """Probe visits in visit order (SI): positions xs, ys [m], start ts [s], dwell taus [s]."""

    def __init__(self, xs, ys, ts, taus):
        self.xs, self.ys, self.ts, self.taus = _f64(xs), _f64(ys), _f64(ts), _f64(taus)
        n = len(self.xs)
        assert len(self.ys) == n and len(self.ts) == n and len(self.taus) == n
        self.n = n


def field(src, Ds, D, Q0, px, py, times, threads=0):
    """psi(p, t) of Eq. 5 on every (time, point): returns array [n_t, n_pts]."""
    lib = _load()
    px, py, times = _f64(px), _f64(py), _f64(times)
    out = np.empty((len(times), len(px)), dtype=np.float64)
    lib.ddo_field(src.n, _ptr(src.xs), _ptr(src.ys), _ptr(src.ts), _ptr(src.taus), Ds, D, Q0,
                  len(px), _ptr(px), _ptr(py), len(times), _ptr(times), _ptr(out), int(threads))
    return out


def field_pairs(src, Ds, D, Q0, px, py, pt, threads=0):
    """psi(p_k, t_k) of Eq. 5 for a list of (point, time) pairs."""
    lib = _load()
    px, py, pt = _f64(px), _f64(py), _f64(pt)
    out = np.empty(len(px), dtype=np.float64)
    lib.ddo_field_pairs(src.n, _ptr(src.xs), _ptr(src.ys), _ptr(src.ts), _ptr(src.taus), Ds, D, Q0,
                        len(px), _ptr(px), _ptr(py), _ptr(pt), _ptr(out), int(threads))
    return out


def dose(src, Ds, D, Q0, targets=None, threads=0):
    """Dwell-start dose psi_{j-1}(r_j, t_j) for the listed visit indices (all by default)."""
    lib = _load()
    if targets is None:
        targets = np.arange(src.n, dtype=np.int64)
    targets = np.ascontiguousarray(np.asarray(targets, dtype=np.int64))
    out = np.empty(len(targets), dtype=np.float64)
    lib.ddo_dose(src.n, _ptr(src.xs), _ptr(src.ys), _ptr(src.ts), _ptr(src.taus), Ds, D, Q0,
                 len(targets), targets.ctypes.data_as(_PI64), _ptr(out), int(threads))
    return out
