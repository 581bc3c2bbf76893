"""Learned surrogate of the final damage map, trained on the exact batched path.

A small convolutional network maps six input planes of a scan -- the visit-time map
(the inverse of each visit's age at the end of the scan, in dwells, where visited), the
visited mask, standardised log10 D and log10 dwell, and for every background visit its
own closed-form term at its position (Eq. 3/4, in the target's units) with a mask of those
visits -- on a 128 x 128 canvas at the probe pitch to the log10 of the dimensionless final
field (psi * 4 pi D / Q0), floored six decades below the map's own peak: values below that
floor change a map's relative L2 error by less than 1e-6, so the loss does not spend
capacity on them.  The probe sigma is fixed (0.1 nm) for the surrogate's scans: it is not
an input plane, and near the last visits the field depends on it.  The loss is the squared
log error weighted per pixel by the pixel's share of the map's squared norm (plus a small
uniform part), which to first order is the squared relative L2 error of the linear map,
the surrogate's accuracy measure.  Six 3x3 convolutions, 32 channels, ReLU, BF16
activations, FP32 accumulation and FP32 master weights; every layer, the loss, the
weight and data gradients and Adam run in the library's CUDA kernels (dd_sur_* in
include/dd.h).  This module only allocates buffers and sequences those calls.

The network learns the field of all but the last K_EXACT visits (the "background"); the
last K_EXACT visits, whose sharp, recent deposits carry most of a map's squared norm, are
added by the exact path (K_EXACT x 128^2 pair terms per map, against the full map's
n_visits x 128^2).  The exact path (dd_batch_*) generates the training fields and is also
the fallback: at inference every map gets k exact spot values, and a map whose estimated
relative L2 error exceeds the threshold is recomputed exactly.
"""
import math
import time

import numpy as np

from . import binding as b
from . import workloads as w

CANVAS = 128
LAYERS = [(16, 32), (32, 32), (32, 32), (32, 32), (32, 32), (32, 16)]   # (cin, cout), padded
# dilation of each 3x3 layer: the receptive field grows to 1 + 2 * sum = 127 pixels, the
# whole canvas, since the final field at a point depends on the whole scan history
DILATIONS = (1, 2, 4, 8, 16, 32)
REAL_IN, REAL_OUT = 6, 1
FLOOR_REL = -6.0          # target floor: log10 of the fraction of the map's peak
# fixed affine normalisation of the target log10 field: (log10 psi - MU) / SIGMA
MU, SIGMA = -3.0, 3.0
PROBE_SIGMA = 0.1e-9      # probe sigma of every surrogate scan [m]
S_DIM = (PROBE_SIGMA / w.PITCH) ** 2   # sigma^2 / pitch^2 of the surrogate's scans
LOSS_ALPHA = 0.9          # share of the loss weight that follows the pixel's squared field
K_EXACT = 64              # the last visits of a scan, added exactly to the network's background


def _torch():
    import torch
    return torch


_VISITS = {}


def visit_list(spec):
    """Grid indices of the scan's visits in visit order (built once per spec object)."""
    hit = _VISITS.get(id(spec))
    if hit is not None and hit[0] is spec:
        return hit[1]
    sc = b.Scan(spec)
    g, _, _ = sc.visits()
    sc.close()
    if len(_VISITS) > 100_000:
        _VISITS.clear()
    _VISITS[id(spec)] = (spec, g)
    return g


class Net:
    """Parameters (FP32 master + BF16 copies), Adam state and per-batch buffers."""

    def __init__(self, device, seed=0, dilations=DILATIONS):
        torch = _torch()
        self.device = device
        self.dil = tuple(dilations)
        rng = np.random.default_rng(seed)
        self.params, self.m, self.v, self.wb, self.wf, self.grads = [], [], [], [], [], []
        for k, (ci, co) in enumerate(LAYERS):
            real_ci = REAL_IN if k == 0 else ci
            real_co = REAL_OUT if k == len(LAYERS) - 1 else co
            wt = np.zeros((co, 9, ci), np.float32)
            wt[:real_co, :, :real_ci] = rng.standard_normal((real_co, 9, real_ci)) * math.sqrt(2.0 / (9 * real_ci))
            p = np.concatenate([wt.reshape(-1), np.zeros(co, np.float32)])
            self.params.append(torch.from_numpy(p).to(device))
            self.m.append(torch.zeros_like(self.params[-1]))
            self.v.append(torch.zeros_like(self.params[-1]))
            self.grads.append(torch.zeros_like(self.params[-1]))
            self.wb.append(torch.from_numpy(wt).to(device).to(torch.bfloat16).contiguous())
            self.wf.append(torch.from_numpy(np.ascontiguousarray(wt[:, ::-1, :].transpose(2, 1, 0)))
                           .to(device).to(torch.bfloat16).contiguous())
        self.step_count = 0
        self._B = None

    def _split(self, k):
        ci, co = LAYERS[k]
        return self.params[k][: co * 9 * ci], self.params[k][co * 9 * ci:]

    def buffers(self, B):
        torch = _torch()
        if self._B == B:
            return
        d, bf = self.device, torch.bfloat16
        H = W = CANVAS
        self.x = torch.zeros((B, H, W, 16), dtype=bf, device=d)
        self.acts = [self.x] + [torch.zeros((B, H, W, 32), dtype=bf, device=d) for _ in range(5)]
        self.pred = torch.zeros((B, H, W), dtype=torch.float32, device=d)
        self.dz6 = torch.zeros((B, H, W, 16), dtype=bf, device=d)
        self.dzs = [torch.zeros((B, H, W, 32), dtype=bf, device=d) for _ in range(2)]
        self.part = torch.zeros(608 * (32 * 9 * 32 + 32), dtype=torch.float32, device=d)
        nb = (B * H * W + 255) // 256
        self.block_sums = torch.zeros(nb, dtype=torch.float64, device=d)
        self.loss_sum = torch.zeros(1, dtype=torch.float64, device=d)
        self._B = B

    def forward(self):
        """pred (FP32 [B,H,W]) from self.x (BF16 [B,H,W,16])."""
        for k in range(5):
            _, bias = self._split(k)
            b.dd_sur_conv3x3(self.acts[k], self.wb[k], bias, None, self.acts[k + 1], 0, self.dil[k])
        _, bias = self._split(5)
        b.dd_sur_conv3x3(self.acts[5], self.wb[5], bias, None, self.pred, 1, self.dil[5])
        return self.pred

    def backward(self, target, weight=None):
        """(Weighted) squared error against target (FP32 [B,H,W]); fills self.grads; returns
        the loss tensor."""
        if weight is None:
            b.dd_sur_mse(self.pred, target, self.dz6, self.block_sums, self.loss_sum)
        else:
            b.dd_sur_wmse(self.pred, target, weight, self.dz6, self.block_sums, self.loss_sum)
        b.dd_sur_wgrad(self.acts[5], self.dz6, self.part, self.grads[5], self.dil[5])
        b.dd_sur_conv3x3(self.dz6, self.wf[5], None, self.acts[5], self.dzs[0], 2, self.dil[5])
        cur = 0
        for k in range(4, -1, -1):
            b.dd_sur_wgrad(self.acts[k], self.dzs[cur], self.part, self.grads[k], self.dil[k])
            if k > 0:
                b.dd_sur_conv3x3(self.dzs[cur], self.wf[k], None, self.acts[k], self.dzs[1 - cur], 2, self.dil[k])
                cur = 1 - cur
        return self.loss_sum

    def adam(self, lr):
        self.step_count += 1
        for k, (ci, co) in enumerate(LAYERS):
            n = co * 9 * ci
            p, g, m, v = self.params[k], self.grads[k], self.m[k], self.v[k]
            b.dd_sur_adam(p[:n], g[:n], m[:n], v[:n], lr, self.step_count, w_bf16=self.wb[k],
                          w_flip=self.wf[k], cin=ci, cout=co)
            b.dd_sur_adam(p[n:], g[n:], m[n:], v[n:], lr, self.step_count)

    def state(self):
        return [p.cpu().numpy().copy() for p in self.params]

    def save(self, path):
        """Checkpoint: FP32 master weights, Adam moments, step count and dilations (.npz)."""
        arrays = {"step": np.array(self.step_count), "dilations": np.array(self.dil)}
        for k in range(len(LAYERS)):
            arrays["p%d" % k] = self.params[k].cpu().numpy()
            arrays["m%d" % k] = self.m[k].cpu().numpy()
            arrays["v%d" % k] = self.v[k].cpu().numpy()
        np.savez(path, **arrays)

    @classmethod
    def load(cls, path, device):
        """Resume from a checkpoint written by save(); the BF16 copies are rebuilt."""
        torch = _torch()
        z = np.load(path)
        net = cls(device, dilations=tuple(int(d) for d in z["dilations"]))
        for k, (ci, co) in enumerate(LAYERS):
            net.params[k].copy_(torch.from_numpy(z["p%d" % k]))
            net.m[k].copy_(torch.from_numpy(z["m%d" % k]))
            net.v[k].copy_(torch.from_numpy(z["v%d" % k]))
            wt = z["p%d" % k][: co * 9 * ci].reshape(co, 9, ci)
            net.wb[k].copy_(torch.from_numpy(wt).to(torch.bfloat16))
            net.wf[k].copy_(torch.from_numpy(np.ascontiguousarray(wt[:, ::-1, :].transpose(2, 1, 0))).to(torch.bfloat16))
        net.step_count = int(z["step"])
        return net


# ----------------------------------------------------------------------- dataset

def draw_scans(n_maps, seed, n_min=32, n_max=128):
    """Scans with the batched workload's distributions (seeded), the probe sigma fixed at
    PROBE_SIGMA (it is not an input of the network)."""
    return [s.with_(sigma_m=PROBE_SIGMA)
            for s in w.batched_specs(n_scans=n_maps, seed=seed, n_min=n_min, n_max=n_max)]


def canvas_points(spec):
    return w.grid_points(CANVAS, spec.pitch_m)


def scan_inputs(specs):
    """Host-side input descriptors: time maps [N, H, W] (-1 unvisited) and scalars [N, 3]
    (standardised log10 D, standardised log10 dwell, kappa = D dwell / pitch^2)."""
    N = len(specs)
    tmap = np.full((N, CANVAS, CANVAS), -1.0, np.float32)
    scal = np.zeros((N, 3), np.float32)
    for k, s in enumerate(specs):
        g = visit_list(s)
        nv = len(g)
        iy, ix = g // s.nx, g % s.nx
        # inverse age of visit k at the end of the scan, in dwells: 1 / (nv - k) (the last
        # visit: 1).  Long after its dwell a visit's own dose falls as 1 / age, and BF16
        # keeps 1 / age to 0.2 % (a log of the age would lose ln(age) times more)
        tmap[k, iy, ix] = (1.0 / (nv - np.arange(nv, dtype=np.float64))).astype(np.float32)
        scal[k] = [(math.log10(s.D_m2s) + 13.5) / 1.5, math.log10(s.dwell_s) + 6.0,
                   s.D_m2s * s.dwell_s / s.pitch_m ** 2]
    return tmap, scal


def input_planes(tmap, scal, x):
    """The network's input planes (BF16 [B,H,W,16]) of a batch: the time map, the visited
    mask, standardised log D and log dwell, and each background visit's own closed-form
    term at its position with a mask of those visits (dd_sur_planes_bg)."""
    b.dd_sur_planes_bg(tmap, scal, S_DIM, K_EXACT, MU, SIGMA, x)
    return x


def field_scales(specs, device):
    """Per-map 4 pi D / Q0 (turns u/m^2 into the dimensionless field), FP64 on the device."""
    torch = _torch()
    return torch.tensor([4 * math.pi * s.D_m2s / s.Q0 for s in specs], dtype=torch.float64, device=device)


def split_scan(spec, k=None):
    """The scan's first n - k visits and its last k, as two custom-order scans of the same
    grid positions and dwell: (background spec, its snapshot time, near spec, its
    snapshot time).  The background is seen at the scan's end, n dwells; the near scan's
    visits start (n - k) dwells early in its own clock, so it is seen at k dwells (the field
    depends on t - t_i only).  Uniform dwell, no dead time (the surrogate's scans)."""
    g = visit_list(spec)
    n = len(g)
    k = max(1, min(K_EXACT if k is None else k, n - 1))
    kw = dict(order=w.CUSTOM, keep_fraction=1.0, mask=None)
    bg = spec.with_(custom_visit=np.ascontiguousarray(g[:n - k]), **kw)
    near = spec.with_(custom_visit=np.ascontiguousarray(g[n - k:]), **kw)
    return bg, n * spec.dwell_s, near, k * spec.dwell_s


def exact_fields(specs, device, prec="mixed", chunk=512, pts_index=None, times=None):
    """Exact fields psi [u/m^2] (FP64, device) on the canvas by the batched path, `chunk`
    scans per plan, at times[k] (default: the end of scan k); with pts_index ([N, k]
    canvas indices) only those points."""
    torch = _torch()
    outs = []
    for c0 in range(0, len(specs), chunk):
        sub = specs[c0:c0 + chunk]
        scans = [b.Scan(s) for s in sub]
        tt = (np.array([w.n_visits(s) * s.dwell_s for s in sub]) if times is None
              else np.asarray(times[c0:c0 + chunk], dtype=np.float64))
        if pts_index is None:
            # the canvas as each scan's grid of points (dd_batch_create_grid)
            plan = b.Batch(scans, None, tt, prec,
                           grids=[(0.0, 0.0, s.pitch_m, s.pitch_m, CANVAS, CANVAS) for s in sub])
            outs.append(plan.run(device=device))
        else:
            idx = pts_index[c0:c0 + chunk]
            allp = np.concatenate([canvas_points(s)[ix] for s, ix in zip(sub, idx)])
            offs = np.concatenate([[0], np.cumsum([len(ix) for ix in idx])]).astype(np.int64)
            plan = b.Batch(scans, offs, tt, prec)
            outs.append(plan.run(torch.from_numpy(np.ascontiguousarray(allp)).to(device)))
        plan.close()
        for s in scans:
            s.close()
    return torch.cat(outs) if outs else None


def loss_weights(target):
    """Per-pixel loss weights [N,H,W] (FP32, device) of normalised targets (dd_sur_weights)."""
    torch = _torch()
    wt = torch.empty_like(target)
    b.dd_sur_weights(target, target.shape[0], CANVAS * CANVAS, MU, SIGMA, LOSS_ALPHA, wt)
    return wt


def near_fields(specs, device, pts_index=None):
    """Exact field of each scan's last K_EXACT visits at its end [N, points] (u/m^2)."""
    parts = [split_scan(s) for s in specs]
    return exact_fields([p[2] for p in parts], device, pts_index=pts_index, times=[p[3] for p in parts])


def build_dataset(n_maps, seed, device):
    """(specs, tmap [N,H,W] f32, scal [N,2] f32, normalised target [N,H,W] f32) on the device;
    the target is (log10 of the dimensionless exact background field -- all visits but the
    last K_EXACT, at the scan's end -- floored at 1e-6 of the map's peak, - MU) / SIGMA."""
    torch = _torch()
    specs = draw_scans(n_maps, seed)
    tmap, scal = scan_inputs(specs)
    parts = [split_scan(s) for s in specs]
    psi = exact_fields([p[0] for p in parts], device, times=[p[1] for p in parts])
    target = torch.empty((n_maps, CANVAS, CANVAS), dtype=torch.float32, device=device)
    b.dd_sur_targets(psi, field_scales(specs, device), n_maps, CANVAS * CANVAS, FLOOR_REL, MU, SIGMA, target)
    return specs, torch.from_numpy(tmap).to(device), torch.from_numpy(scal).to(device), target


# ---------------------------------------------------------------------- training

def train(net, tmap, scal, target, epochs, batch=32, lr=2e-3, seed=0, log=None, weight=None):
    """Adam on the squared error of the normalised log10 field (weighted per pixel when
    `weight` [N,H,W] is given); returns the per-epoch mean losses."""
    torch = _torch()
    N = tmap.shape[0]
    net.buffers(batch)
    rng = np.random.default_rng(seed)
    losses = []
    for ep in range(epochs):
        order = rng.permutation(N)
        tot, cnt = 0.0, 0
        lr_ep = lr * (0.5 * (1 + math.cos(math.pi * ep / max(1, epochs))))
        for s0 in range(0, N - batch + 1, batch):
            idx = torch.from_numpy(order[s0:s0 + batch]).to(tmap.device)
            input_planes(tmap[idx].contiguous(), scal[idx].contiguous(), net.x)
            net.forward()
            loss = net.backward(target[idx].contiguous(), None if weight is None else weight[idx].contiguous())
            net.adam(lr_ep)
            tot += float(loss.item()) / (batch * CANVAS * CANVAS)
            cnt += 1
        losses.append(tot / max(1, cnt))
        if log:
            log("epoch %d loss %.4f" % (ep, losses[-1]))
    return losses


def predict(net, tmap, scal, batch=256):
    """Normalised log10-field predictions [N,H,W] (FP32) in batches of `batch` maps."""
    torch = _torch()
    N = tmap.shape[0]
    out = torch.empty((N, CANVAS, CANVAS), dtype=torch.float32, device=tmap.device)
    for s0 in range(0, N, batch):
        B = min(batch, N - s0)
        net.buffers(B)
        input_planes(tmap[s0:s0 + B].contiguous(), scal[s0:s0 + B].contiguous(), net.x)
        out[s0:s0 + B] = net.forward()
    return out


def fields_from_prediction(pred, specs):
    """psi [N, H*W] (u/m^2, FP64) from normalised predictions [N,H,W]."""
    torch = _torch()
    N = pred.shape[0]
    out = torch.empty((N, CANVAS * CANVAS), dtype=torch.float64, device=pred.device)
    b.dd_sur_fields(pred, field_scales(specs, pred.device), N, CANVAS * CANVAS, MU, SIGMA, out)
    return out


def map_errors(fields, exact):
    """Relative L2 error of each map (evaluation only)."""
    torch = _torch()
    return (torch.linalg.norm(fields - exact, dim=1) / torch.linalg.norm(exact, dim=1)).cpu().numpy()


def spot_points(specs, k_spot, seed=0):
    """Canvas indices [N, k_spot] of the exact spot checks: the positions of the last
    k_spot / 2 visits (near them sits most of a map's squared norm) and k_spot / 2 seeded
    canvas points."""
    rng = np.random.default_rng(seed)
    out = np.empty((len(specs), k_spot), np.int32)
    for m, s in enumerate(specs):
        g = visit_list(s)
        last = ((g // s.nx) * CANVAS + g % s.nx)[::-1][:k_spot // 2]
        out[m, :len(last)] = last
        out[m, len(last):] = rng.integers(0, CANVAS * CANVAS, k_spot - len(last))
    return out


def surrogate_fields(net, specs, tmap, scal, device, batch=256):
    """Fields [N, H*W] (u/m^2, FP64): the network's background plus the exact field of each
    scan's last K_EXACT visits; also returns the prediction and that exact part."""
    pred = predict(net, tmap, scal, batch)
    near = near_fields(specs, device).view(len(specs), -1)
    return fields_from_prediction(pred, specs) + near, pred, near


def infer_with_fallback(net, specs, tmap, scal, device, k_spot=64, threshold=1e-2, batch=256, seed=0):
    """Surrogate fields with exact spot checks; maps whose estimated relative L2 error
    exceeds `threshold` are recomputed by the exact batched path.  Returns
    (fields [N, H*W] u/m^2 FP64, fallback mask, estimated errors, seconds)."""
    torch = _torch()
    t0 = time.perf_counter()
    N = len(specs)
    fields, pred, near = surrogate_fields(net, specs, tmap, scal, device, batch)
    spot = spot_points(specs, k_spot, seed)
    ex_spot = exact_fields(specs, device, pts_index=spot)
    est = torch.empty(N, dtype=torch.float64, device=device)
    b.dd_sur_spot_error(pred, torch.from_numpy(spot).to(device), ex_spot, field_scales(specs, device), N,
                        CANVAS * CANVAS, k_spot, MU, SIGMA, est, add=near)
    est = est.cpu().numpy()
    bad = np.nonzero(~(est <= threshold))[0]
    if len(bad):
        fixed = exact_fields([specs[i] for i in bad], device).view(len(bad), -1)
        fields[torch.from_numpy(bad).to(device)] = fixed
    torch.cuda.synchronize(device)
    return fields, est > threshold, est, time.perf_counter() - t0
