"""Python binding of libdd.so (include/dd.h): argument marshalling only.

Every computation happens in the CUDA library; this module converts numpy arrays and
torch tensors to pointers, calls the C entry point of the same name and raises on a
non-zero status.  If libdd.so cannot be built or loaded the import fails loudly:
there is no fallback implementation.
"""
import ctypes
import os

import numpy as np

from . import build as _build

DD_OK, DD_EINVAL, DD_ENOMEM, DD_ECUDA, DD_ETIMEOUT, DD_ENOTSUP = 0, -1, -2, -3, -4, -5
DD_RASTER, DD_SERPENTINE, DD_INTERLEAVED, DD_RANDOM, DD_CUSTOM = 0, 1, 2, 3, 4
DD_FP64, DD_MIXED = 0, 1
PRECISIONS = {"fp64": DD_FP64, "mixed": DD_MIXED, DD_FP64: DD_FP64, DD_MIXED: DD_MIXED}


class DDError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("dd status %d: %s" % (status, msg))
        self.status = status


class dd_scan_desc(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("pitch_m", ctypes.c_double), ("sigma_m", ctypes.c_double), ("D_m2s", ctypes.c_double),
        ("Q0", ctypes.c_double), ("dwell_s", ctypes.c_double), ("flyback_s", ctypes.c_double),
        ("order", ctypes.c_int32), ("interleave_stride", ctypes.c_int32),
        ("seed", ctypes.c_uint64), ("keep_fraction", ctypes.c_double),
        ("mask", ctypes.POINTER(ctypes.c_uint8)),
        ("custom_visit", ctypes.POINTER(ctypes.c_int32)), ("n_custom", ctypes.c_int32),
        ("dwell_per_visit", ctypes.POINTER(ctypes.c_double)),
        ("blank_s", ctypes.c_double), ("blank_s_per_m", ctypes.c_double),
    ]


_VP = ctypes.c_void_p
_I64 = ctypes.c_int64
_lib = None


def lib_path():
    return _build.LIB


def load(build_if_missing=True):
    """Load libdd.so (building it first if needed) and declare the C signatures."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build_if_missing else _build.LIB
    if not os.path.exists(path):
        raise ImportError("libdd.so not found at %s: build it with paper_2507_00294_gb300.build" % path)
    lib = ctypes.CDLL(path)
    lib.dd_create_scan.argtypes = [ctypes.POINTER(dd_scan_desc), ctypes.POINTER(_VP)]
    lib.dd_scan_size.argtypes = [_VP, ctypes.POINTER(_I64)]
    lib.dd_scan_visits.argtypes = [_VP, _VP, _VP, _VP]
    lib.dd_field_at_times.argtypes = [_VP, _VP, _I64, _VP, _I64, ctypes.c_int, _VP, _VP]
    lib.dd_per_probe_dose.argtypes = [_VP, ctypes.c_int, _VP, _VP]
    lib.dd_field_on_grid.argtypes = [_VP, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                     _I64, _I64, _VP, _I64, ctypes.c_int, _VP, _VP]
    lib.dd_field_on_grid.restype = ctypes.c_int
    lib.dd_field_batch.argtypes = [_VP, ctypes.c_int32, _VP, _VP, _VP, ctypes.c_int, _VP, _VP]
    lib.dd_per_probe_dose_range.argtypes = [_VP, ctypes.c_int, _I64, _I64, _VP, _VP]
    lib.dd_per_probe_dose_range.restype = ctypes.c_int
    lib.dd_per_probe_dose_noalloc.argtypes = [_VP, ctypes.c_int, _VP, _VP]
    lib.dd_per_probe_dose_noalloc.restype = ctypes.c_int
    lib.dd_batch_create.argtypes = [_VP, ctypes.c_int32, _VP, _VP, ctypes.c_int, ctypes.POINTER(_VP)]
    lib.dd_batch_create_grid.argtypes = [_VP, ctypes.c_int32, _VP, _VP, _VP, ctypes.c_int, ctypes.POINTER(_VP)]
    lib.dd_batch_create_grid.restype = ctypes.c_int
    lib.dd_batch_run.argtypes = [_VP, _VP, _VP, _VP]
    lib.dd_batch_tune.argtypes = [_VP, _VP, ctypes.POINTER(ctypes.c_int32)]
    lib.dd_batch_info.argtypes = [_VP, ctypes.POINTER(_I64), ctypes.POINTER(_I64), ctypes.POINTER(ctypes.c_int32)]
    for name in ("dd_batch_create", "dd_batch_run", "dd_batch_tune", "dd_batch_info"):
        getattr(lib, name).restype = ctypes.c_int
    lib.dd_batch_destroy.argtypes = [_VP]
    lib.dd_batch_destroy.restype = None
    i32 = ctypes.c_int32
    lib.dd_sur_conv3x3.argtypes = [_VP, _VP, _VP, _VP, _VP, i32, i32, i32, i32, i32, i32, i32, _VP]
    lib.dd_sur_wgrad.argtypes = [_VP, _VP, i32, i32, i32, i32, i32, i32, _VP, _I64, _VP, _VP]
    lib.dd_sur_mse.argtypes = [_VP, _VP, _I64, _VP, _VP, _VP, _VP]
    lib.dd_sur_wmse.argtypes = [_VP, _VP, _VP, _I64, _VP, _VP, _VP, _VP]
    lib.dd_sur_weights.argtypes = [_VP, _I64, _I64, ctypes.c_float, ctypes.c_float, ctypes.c_float, _VP, _VP]
    lib.dd_sur_adam.argtypes = [_VP, _VP, _VP, _VP, _I64, ctypes.c_float, ctypes.c_float,
                                ctypes.c_float, ctypes.c_float, i32, _VP, _VP, i32, i32, _VP]
    lib.dd_sur_planes.argtypes = [_VP, _VP, i32, i32, i32, _VP, _VP]
    lib.dd_sur_planes_bg.argtypes = [_VP, _VP, ctypes.c_float, i32, ctypes.c_float, ctypes.c_float, i32, i32, i32,
                                     _VP, _VP]
    lib.dd_sur_targets.argtypes = [_VP, _VP, _I64, _I64, ctypes.c_double, ctypes.c_float, ctypes.c_float, _VP, _VP]
    lib.dd_sur_fields.argtypes = [_VP, _VP, _I64, _I64, ctypes.c_float, ctypes.c_float, _VP, _VP]
    lib.dd_sur_spot_error.argtypes = [_VP, _VP, _VP, _VP, _VP, i32, i32, i32, ctypes.c_float, ctypes.c_float, _VP, _VP]
    lib.dd_sur_check.argtypes = []
    lib.dd_field_check.argtypes = []
    lib.dd_field_check.restype = ctypes.c_int
    lib.dd_field_grid_split.argtypes = [_VP, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                        _I64, _I64, _VP, _I64, _VP, _VP]
    lib.dd_field_grid_split.restype = ctypes.c_int
    for name in ("dd_sur_conv3x3", "dd_sur_wgrad", "dd_sur_mse", "dd_sur_wmse", "dd_sur_weights", "dd_sur_adam",
                 "dd_sur_planes", "dd_sur_planes_bg",
                 "dd_sur_targets", "dd_sur_fields", "dd_sur_spot_error", "dd_sur_check"):
        getattr(lib, name).restype = ctypes.c_int
    lib.dd_profile_enable.argtypes = [ctypes.c_int32]
    lib.dd_profile_reset.argtypes = []
    lib.dd_profile_read.argtypes = [_VP, _VP, _VP, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]
    for name in ("dd_profile_enable", "dd_profile_reset", "dd_profile_read"):
        getattr(lib, name).restype = ctypes.c_int
    lib.dd_destroy.argtypes = [_VP]
    lib.dd_destroy.restype = None
    lib.dd_last_error.restype = ctypes.c_char_p
    lib.dd_version.restype = ctypes.c_char_p
    for name in ("dd_create_scan", "dd_scan_size", "dd_scan_visits", "dd_field_at_times",
                 "dd_per_probe_dose", "dd_field_batch"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(status, what):
    if status != DD_OK:
        raise DDError(status, "%s: %s" % (what, load().dd_last_error().decode()))


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr(x, dtype):
    """(pointer, keepalive) for a numpy array / torch tensor of the given dtype."""
    if x is None:
        return None, None
    if _is_torch(x):
        import torch
        want = {np.float64: torch.float64, np.int32: torch.int32, np.int64: torch.int64}[dtype]
        if x.dtype != want or not x.is_contiguous():
            raise TypeError("expected a contiguous %s tensor" % want)
        return ctypes.c_void_p(x.data_ptr()), x
    a = np.ascontiguousarray(np.asarray(x, dtype=dtype))
    return ctypes.c_void_p(a.ctypes.data), a


def _stream(stream, *tensors):
    if stream is not None:
        return ctypes.c_void_p(stream if isinstance(stream, int) else stream.cuda_stream)
    for t in tensors:
        if t is not None and _is_torch(t) and t.is_cuda:
            import torch
            return ctypes.c_void_p(torch.cuda.current_stream(t.device).cuda_stream)
    return ctypes.c_void_p(0)


class Scan:
    """A dd_scan built from a workloads.ScanSpec (or anything with the same fields)."""

    def __init__(self, spec):
        lib = load()
        d = dd_scan_desc()
        d.nx, d.ny = int(spec.nx), int(spec.ny)
        d.pitch_m, d.sigma_m, d.D_m2s = spec.pitch_m, spec.sigma_m, spec.D_m2s
        d.Q0, d.dwell_s, d.flyback_s = spec.Q0, spec.dwell_s, spec.flyback_s
        d.order, d.interleave_stride = int(spec.order), int(spec.interleave_stride)
        d.seed, d.keep_fraction = int(spec.seed) & ((1 << 64) - 1), float(spec.keep_fraction)
        d.blank_s = float(getattr(spec, "blank_s", 0.0))
        d.blank_s_per_m = float(getattr(spec, "blank_s_per_m", 0.0))
        self._keep = []
        if spec.mask is not None:
            m = np.ascontiguousarray(np.asarray(spec.mask, dtype=np.uint8).reshape(-1))
            self._keep.append(m)
            d.mask = m.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
        if spec.custom_visit is not None:
            c = np.ascontiguousarray(np.asarray(spec.custom_visit, dtype=np.int32))
            self._keep.append(c)
            d.custom_visit = c.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
            d.n_custom = len(c)
        if spec.dwell_per_visit is not None:
            w = np.ascontiguousarray(np.asarray(spec.dwell_per_visit, dtype=np.float64))
            self._keep.append(w)
            d.dwell_per_visit = w.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        h = ctypes.c_void_p()
        _check(lib.dd_create_scan(ctypes.byref(d), ctypes.byref(h)), "dd_create_scan")
        self._keep = None
        self.handle = h
        self.spec = spec

    def __len__(self):
        n = ctypes.c_int64()
        _check(load().dd_scan_size(self.handle, ctypes.byref(n)), "dd_scan_size")
        return n.value

    def visits(self):
        """(grid_index int32, t_start_s, dwell_s) in visit order."""
        n = len(self)
        g = np.empty(n, np.int32)
        t = np.empty(n, np.float64)
        w = np.empty(n, np.float64)
        _check(load().dd_scan_visits(self.handle, g.ctypes.data, t.ctypes.data, w.ctypes.data),
               "dd_scan_visits")
        return g, t, w

    def close(self):
        if getattr(self, "handle", None) is not None and _lib is not None:
            _lib.dd_destroy(self.handle)
            self.handle = None

    def __del__(self):
        self.close()


def multi_frame_spec(spec, frames):
    """Multi-frame acquisition (Sec. 1): the scan's own visit order repeated `frames` times
    with the dwell divided by `frames`, as a custom-order scan description."""
    from dataclasses import replace
    if frames < 1:
        raise ValueError("frames must be >= 1")
    g, _, tau = Scan(spec).visits()
    if spec.dwell_per_visit is not None:
        per = np.tile(np.asarray(tau) / frames, frames)
    else:
        per = None
    return replace(spec, order=DD_CUSTOM, custom_visit=np.tile(g, frames), keep_fraction=1.0, mask=None,
                   dwell_s=spec.dwell_s / frames, dwell_per_visit=per, flyback_s=0.0)


def dd_create_scan(spec):
    return Scan(spec)


def dd_field_at_times(scan, pts_xy_m, times_s, prec="mixed", out=None, stream=None):
    """psi at every (time, point); returns `out` ([n_t, n_pts] float64, numpy or torch).

    With a `stream` and only page-locked host buffers the host copies stay enqueued on
    that stream: synchronise it before reading `out`."""
    n_pts = (pts_xy_m.shape[0] if hasattr(pts_xy_m, "shape") else len(pts_xy_m))
    n_t = len(times_s)
    if out is None:
        if _is_torch(pts_xy_m) and pts_xy_m.is_cuda:
            import torch
            out = torch.empty((n_t, n_pts), dtype=torch.float64, device=pts_xy_m.device)
        else:
            out = np.empty((n_t, n_pts), dtype=np.float64)
    p, kp = _ptr(pts_xy_m, np.float64)
    t, kt = _ptr(times_s, np.float64)
    o, ko = _ptr(out, np.float64)
    st = load().dd_field_at_times(scan.handle, p, n_pts, t, n_t, PRECISIONS[prec], o,
                                  _stream(stream, pts_xy_m, out))
    _check(st, "dd_field_at_times")
    return out


def dd_field_on_grid(scan, x0, y0, dx, dy, n_cols, n_rows, times_s, prec="mixed", out=None, stream=None,
                     device=None):
    """Field on the grid (x0 + c dx, y0 + r dy), c < n_cols, r < n_rows: out [n_t, n_rows * n_cols]
    (row-major points).  times_s: numpy or torch; out: host numpy unless `device` is given."""
    t, kt = _ptr(times_s, np.float64)
    n_t = int(times_s.shape[0]) if _is_torch(times_s) else len(np.asarray(times_s).reshape(-1))
    n_pts = int(n_cols) * int(n_rows)
    if out is None:
        if device is not None:
            import torch
            out = torch.empty((n_t, n_pts), dtype=torch.float64, device=device)
        else:
            out = np.empty((n_t, n_pts), dtype=np.float64)
    o, ko = _ptr(out, np.float64)
    _check(load().dd_field_on_grid(scan.handle, float(x0), float(y0), float(dx), float(dy), int(n_cols),
                                   int(n_rows), t, n_t, PRECISIONS[prec], o, _stream(stream, out)),
           "dd_field_on_grid")
    return out


def dd_per_probe_dose(scan, prec="mixed", out=None, stream=None, device=None):
    """Dwell-start dose of every visit, in visit order."""
    n = len(scan)
    if out is None:
        if device is not None:
            import torch
            out = torch.empty(n, dtype=torch.float64, device=device)
        else:
            out = np.empty(n, dtype=np.float64)
    o, ko = _ptr(out, np.float64)
    _check(load().dd_per_probe_dose(scan.handle, PRECISIONS[prec], o, _stream(stream, out)),
           "dd_per_probe_dose")
    return out


def dd_per_probe_dose_range(scan, j0, j1, prec="mixed", out=None, stream=None, device=None):
    """Dwell-start dose of visits j0 <= j < j1 (out[j - j0])."""
    m = int(j1) - int(j0)
    if out is None:
        if device is not None:
            import torch
            out = torch.empty(m, dtype=torch.float64, device=device)
        else:
            out = np.empty(m, dtype=np.float64)
    o, ko = _ptr(out, np.float64)
    _check(load().dd_per_probe_dose_range(scan.handle, PRECISIONS[prec], int(j0), int(j1), o,
                                           _stream(stream, out)), "dd_per_probe_dose_range")
    return out


def dd_per_probe_dose_noalloc(scan, out, prec="mixed", stream=None):
    """Dwell-start dose into a device tensor `out` without any device allocation
    (scratch in the library's fixed 8 MiB area; at most 16384 visits)."""
    o, ko = _ptr(out, np.float64)
    _check(load().dd_per_probe_dose_noalloc(scan.handle, PRECISIONS[prec], o, _stream(stream, out)),
           "dd_per_probe_dose_noalloc")
    return out


def dd_field_batch(scans, pt_offsets, pts_xy_m, times_s, prec="mixed", out=None, stream=None):
    """Field of many scans, each at its own points and single time; out[pt_offsets[k]:...]."""
    n_scans = len(scans)
    handles = (ctypes.c_void_p * n_scans)(*[s.handle.value for s in scans])
    offs = np.ascontiguousarray(np.asarray(pt_offsets, dtype=np.int64))
    times = np.ascontiguousarray(np.asarray(times_s, dtype=np.float64))
    total = int(offs[-1])
    if out is None:
        if _is_torch(pts_xy_m) and pts_xy_m.is_cuda:
            import torch
            out = torch.empty(total, dtype=torch.float64, device=pts_xy_m.device)
        else:
            out = np.empty(total, dtype=np.float64)
    p, kp = _ptr(pts_xy_m, np.float64)
    o, ko = _ptr(out, np.float64)
    st = load().dd_field_batch(handles, n_scans, offs.ctypes.data, p, times.ctypes.data,
                               PRECISIONS[prec], o, _stream(stream, pts_xy_m, out))
    _check(st, "dd_field_batch")
    return out


class Batch:
    """A dd_batch plan: many scans, each at its own points and one time, one graph launch.
    With grids ([n_scans, 6]: x0, y0, dx, dy [m], columns, rows) the points are each scan's
    grid (dd_batch_create_grid) and run() takes pts_xy_m=None."""

    def __init__(self, scans, pt_offsets, times_s, prec="mixed", grids=None):
        lib = load()
        self.scans = list(scans)                  # the plan reads them: keep them alive
        n = len(self.scans)
        self._handles = (ctypes.c_void_p * n)(*[s.handle.value for s in self.scans])
        times = np.ascontiguousarray(np.asarray(times_s, dtype=np.float64))
        h = ctypes.c_void_p()
        if grids is None:
            self.offsets = np.ascontiguousarray(np.asarray(pt_offsets, dtype=np.int64))
            _check(lib.dd_batch_create(self._handles, n, self.offsets.ctypes.data, times.ctypes.data,
                                       PRECISIONS[prec], ctypes.byref(h)), "dd_batch_create")
        else:
            g = np.asarray(grids, dtype=np.float64).reshape(n, 6)
            xy = np.ascontiguousarray(g[:, :4])
            wh = np.ascontiguousarray(g[:, 4:].astype(np.int64))
            self.offsets = np.concatenate([[0], np.cumsum(wh[:, 0] * wh[:, 1])]).astype(np.int64)
            _check(lib.dd_batch_create_grid(self._handles, n, xy.ctypes.data, wh.ctypes.data, times.ctypes.data,
                                            PRECISIONS[prec], ctypes.byref(h)), "dd_batch_create_grid")
        self.on_grid = grids is not None
        self.handle = h
        self.total = int(self.offsets[-1])

    def run(self, pts_xy_m=None, out=None, stream=None, device=None):
        if out is None:
            if _is_torch(pts_xy_m) and pts_xy_m.is_cuda:
                import torch
                out = torch.empty(self.total, dtype=torch.float64, device=pts_xy_m.device)
            elif device is not None:
                import torch
                out = torch.empty(self.total, dtype=torch.float64, device=device)
            else:
                out = np.empty(self.total, dtype=np.float64)
        p, kp = _ptr(pts_xy_m, np.float64)
        o, ko = _ptr(out, np.float64)
        _check(load().dd_batch_run(self.handle, p, o, _stream(stream, pts_xy_m, out)), "dd_batch_run")
        return out

    def tune(self, pts_xy_m=None):
        p, kp = _ptr(pts_xy_m, np.float64)
        v = ctypes.c_int32()
        _check(load().dd_batch_tune(self.handle, p, ctypes.byref(v)), "dd_batch_tune")
        return v.value

    def info(self):
        n, pairs, v = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
        _check(load().dd_batch_info(self.handle, ctypes.byref(n), ctypes.byref(pairs), ctypes.byref(v)),
               "dd_batch_info")
        return {"items": n.value, "pairs": pairs.value, "variant": v.value}

    def close(self):
        if getattr(self, "handle", None) is not None and _lib is not None:
            _lib.dd_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        self.close()


def _dp(t):
    """Device pointer of a torch tensor (None -> NULL)."""
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _cs(stream, t):
    import torch
    if stream is not None:
        return ctypes.c_void_p(stream if isinstance(stream, int) else stream.cuda_stream)
    return ctypes.c_void_p(torch.cuda.current_stream(t.device).cuda_stream)


def dd_sur_conv3x3(x, w, bias, mask, out, epilogue, dilation=1, stream=None):
    """x [B,H,W,cin] bf16, w [cout,9,cin] bf16 -> out (see include/dd.h)."""
    B, H, W, cin = x.shape
    cout = w.shape[0]
    _check(load().dd_sur_conv3x3(_dp(x), _dp(w), _dp(bias), _dp(mask), _dp(out), B, H, W, cin, cout,
                                 int(dilation), int(epilogue), _cs(stream, x)), "dd_sur_conv3x3")
    return out


def dd_field_grid_split(scan, x0, y0, dx, dy, n_cols, n_rows, times_s, degree2=False):
    """Per snapshot, the number of leading visits dd_field_on_grid sums on the tensor cores
    (FP32-mixed); host-only.  degree2: also return how many of them in the degree-2 form."""
    t = np.ascontiguousarray(np.asarray(times_s, dtype=np.float64).reshape(-1))
    out = np.zeros(len(t), dtype=np.int64)
    out2 = np.zeros(len(t), dtype=np.int64)
    _check(load().dd_field_grid_split(scan.handle, float(x0), float(y0), float(dx), float(dy), int(n_cols),
                                      int(n_rows), t.ctypes.data, len(t), out.ctypes.data, out2.ctypes.data),
           "dd_field_grid_split")
    return (out, out2) if degree2 else out


def dd_field_check():
    """Synchronise the device; raise DDError (DD_ETIMEOUT) if a tensor-core contraction of
    dd_field_on_grid gave up waiting for its MMAs since the last check."""
    _check(load().dd_field_check(), "dd_field_check")


def dd_sur_check():
    """Synchronise the device; raise DDError (DD_ETIMEOUT) if a tensor-memory convolution
    gave up waiting for its MMAs since the last check."""
    _check(load().dd_sur_check(), "dd_sur_check")


def dd_sur_wgrad(x, dz, part, grad, dilation=1, stream=None):
    B, H, W, cin = x.shape
    cout = dz.shape[3]
    _check(load().dd_sur_wgrad(_dp(x), _dp(dz), B, H, W, cin, cout, int(dilation), _dp(part), part.numel(),
                               _dp(grad), _cs(stream, x)), "dd_sur_wgrad")
    return grad


def dd_sur_mse(pred, target, dz, block_sums, loss_sum, stream=None):
    _check(load().dd_sur_mse(_dp(pred), _dp(target), pred.numel(), _dp(dz), _dp(block_sums), _dp(loss_sum),
                             _cs(stream, pred)), "dd_sur_mse")


def dd_sur_adam(param, grad, m, v, lr, step, beta1=0.9, beta2=0.999, eps=1e-8, w_bf16=None, w_flip=None,
                cin=0, cout=0, stream=None):
    _check(load().dd_sur_adam(_dp(param), _dp(grad), _dp(m), _dp(v), param.numel(), lr, beta1, beta2, eps,
                              int(step), _dp(w_bf16), _dp(w_flip), cin, cout, _cs(stream, param)), "dd_sur_adam")


def dd_sur_planes(tmap, scal, x, stream=None):
    B, H, W = tmap.shape
    _check(load().dd_sur_planes(_dp(tmap), _dp(scal), B, H, W, _dp(x), _cs(stream, tmap)), "dd_sur_planes")
    return x


def dd_sur_planes_bg(tmap, scal3, s_dim, k_exact, mu, sigma, x, stream=None):
    B, H, W = tmap.shape
    _check(load().dd_sur_planes_bg(_dp(tmap), _dp(scal3), s_dim, k_exact, mu, sigma, B, H, W, _dp(x),
                                   _cs(stream, tmap)), "dd_sur_planes_bg")
    return x


def dd_sur_wmse(pred, target, weight, dz, block_sums, loss_sum, stream=None):
    _check(load().dd_sur_wmse(_dp(pred), _dp(target), _dp(weight), pred.numel(), _dp(dz), _dp(block_sums),
                              _dp(loss_sum), _cs(stream, pred)), "dd_sur_wmse")


def dd_sur_weights(target, n_maps, hw, mu, sigma, alpha, out, stream=None):
    _check(load().dd_sur_weights(_dp(target), n_maps, hw, mu, sigma, alpha, _dp(out), _cs(stream, target)),
           "dd_sur_weights")


def dd_sur_targets(psi, scale, n_maps, hw, floor_rel_log10, mu, sigma, out, stream=None):
    _check(load().dd_sur_targets(_dp(psi), _dp(scale), n_maps, hw, floor_rel_log10, mu, sigma, _dp(out),
                                 _cs(stream, psi)), "dd_sur_targets")
    return out


def dd_sur_fields(pred, scale, n_maps, hw, mu, sigma, psi, stream=None):
    _check(load().dd_sur_fields(_dp(pred), _dp(scale), n_maps, hw, mu, sigma, _dp(psi), _cs(stream, pred)),
           "dd_sur_fields")
    return psi


def dd_sur_spot_error(pred, idx, exact, scale, n_maps, hw, k, mu, sigma, err, stream=None, add=None):
    _check(load().dd_sur_spot_error(_dp(pred), _dp(idx), _dp(exact), _dp(scale), None if add is None else _dp(add),
                                    n_maps, hw, k, mu, sigma, _dp(err), _cs(stream, pred)), "dd_sur_spot_error")
    return err


def dd_profile_enable(on=True):
    _check(load().dd_profile_enable(1 if on else 0), "dd_profile_enable")


def dd_profile_reset():
    _check(load().dd_profile_reset(), "dd_profile_reset")


def dd_profile_read(max_entries=64):
    """{kernel name: (launches, total device ms)} since the last reset."""
    names = ctypes.create_string_buffer(64 * max_entries)
    launches = np.zeros(max_entries, np.int64)
    ms = np.zeros(max_entries, np.float64)
    n = ctypes.c_int32()
    _check(load().dd_profile_read(names, launches.ctypes.data, ms.ctypes.data, max_entries,
                                  ctypes.byref(n)), "dd_profile_read")
    out = {}
    for k in range(min(n.value, max_entries)):
        nm = names.raw[64 * k:64 * k + 64].split(b"\0", 1)[0].decode()
        out[nm] = (int(launches[k]), float(ms[k]))
    return out


def version():
    return load().dd_version().decode()
