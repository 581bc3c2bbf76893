"""Plain FP64 reference of the surrogate network (test infrastructure only).

The learned surrogate is a stack of six 3x3 convolutions ("same" zero padding, stride 1)
with ReLU after the first five, NHWC activations and weights laid out [Cout][3][3][Cin].
This module states the forward pass, the MSE loss and the backward pass directly from
their definitions with numpy einsum over the nine taps, so that the GPU kernels'
forward, data-gradient and weight-gradient results can be checked against it.

  forward:  z[b,y,x,o] = bias[o] + sum_{ky,kx,c} w[o,ky,kx,c] * xp[b, y+d*ky, x+d*kx, c]
            (xp = x zero-padded by d pixels on each side; d = dilation, 1 for a plain 3x3)
  dgrad:    dx[b,y,x,c] = sum_{ky,kx,o} dz[b, y-d(ky-1), x-d(kx-1), o] * w[o,ky,kx,c]
  wgrad:    dw[o,ky,kx,c] = sum_{b,y,x} dz[b,y,x,o] * xp[b, y+d*ky, x+d*kx, c];  dbias[o] = sum dz
"""
import numpy as np


def _pad(x, d):
    B, H, W, C = x.shape
    xp = np.zeros((B, H + 2 * d, W + 2 * d, C))
    xp[:, d:d + H, d:d + W, :] = x
    return xp


def conv3x3(x, w, b, dil=1):
    B, H, W, Ci = x.shape
    xp = _pad(x, dil)
    z = np.zeros((B, H, W, w.shape[0])) + b
    for ky in range(3):
        for kx in range(3):
            z += np.einsum("bhwc,oc->bhwo", xp[:, dil * ky:dil * ky + H, dil * kx:dil * kx + W, :], w[:, ky, kx, :])
    return z


def conv3x3_dgrad(dz, w, dil=1):
    B, H, W, Co = dz.shape
    dxp = np.zeros((B, H + 2 * dil, W + 2 * dil, w.shape[3]))
    for ky in range(3):
        for kx in range(3):
            dxp[:, dil * ky:dil * ky + H, dil * kx:dil * kx + W, :] += np.einsum("bhwo,oc->bhwc", dz, w[:, ky, kx, :])
    return dxp[:, dil:dil + H, dil:dil + W, :]


def conv3x3_wgrad(x, dz, dil=1):
    B, H, W, Ci = x.shape
    xp = _pad(x, dil)
    dw = np.zeros((dz.shape[3], 3, 3, Ci))
    for ky in range(3):
        for kx in range(3):
            dw[:, ky, kx, :] = np.einsum("bhwo,bhwc->oc", dz, xp[:, dil * ky:dil * ky + H, dil * kx:dil * kx + W, :])
    return dw, dz.sum(axis=(0, 1, 2))


def forward(params, x, dils=None):
    """params: list of (w, b); returns the list of layer outputs (post-activation; the last
    layer is linear).  dils: per-layer dilation (default 1)."""
    dils = dils or [1] * len(params)
    acts = [x]
    for k, (w, b) in enumerate(params):
        z = conv3x3(acts[-1], w, b, dils[k])
        acts.append(np.maximum(z, 0.0) if k < len(params) - 1 else z)
    return acts


def loss_and_grads(params, x, target, dils=None):
    """Mean squared error over every output element and its parameter gradients."""
    dils = dils or [1] * len(params)
    acts = forward(params, x, dils)
    pred = acts[-1]
    diff = pred - target
    loss = float(np.mean(diff ** 2))
    dz = 2.0 * diff / diff.size
    grads = [None] * len(params)
    for k in range(len(params) - 1, -1, -1):
        w, _ = params[k]
        grads[k] = conv3x3_wgrad(acts[k], dz, dils[k])
        if k > 0:
            da = conv3x3_dgrad(dz, w, dils[k])
            dz = da * (acts[k] > 0.0)          # ReLU of the previous layer
    return loss, grads
