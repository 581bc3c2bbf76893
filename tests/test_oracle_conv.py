"""Pins for the FP64 reference of the surrogate network: forward against torch's CPU
conv2d (a library routine) and gradients against torch autograd and central finite
differences of the reference's own loss."""
import numpy as np
import pytest

from oracle import conv_ref

torch = pytest.importorskip("torch")


def rand_params(rng, chans):
    return [(rng.standard_normal((co, 3, 3, ci)) * 0.3, rng.standard_normal(co) * 0.1)
            for ci, co in zip(chans[:-1], chans[1:])]


@pytest.mark.parametrize("dil", [1, 2, 3])
def test_conv_forward_matches_torch(dil):
    rng = np.random.default_rng(dil)
    x = rng.standard_normal((2, 7, 9, 5))
    w = rng.standard_normal((3, 3, 3, 5))
    b = rng.standard_normal(3)
    got = conv_ref.conv3x3(x, w, b, dil)
    ref = torch.nn.functional.conv2d(torch.from_numpy(x).permute(0, 3, 1, 2),
                                     torch.from_numpy(w).permute(0, 3, 1, 2), torch.from_numpy(b),
                                     padding=dil, dilation=dil).permute(0, 2, 3, 1).numpy()
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)


def test_network_gradients_match_autograd():
    rng = np.random.default_rng(1)
    chans = [4, 6, 6, 6, 6, 6, 1]
    dils = [1, 2, 3, 1, 2, 1]
    params = rand_params(rng, chans)
    x = rng.standard_normal((2, 9, 8, 4))
    y = rng.standard_normal((2, 9, 8, 1))
    loss, grads = conv_ref.loss_and_grads(params, x, y, dils)
    tp = [(torch.tensor(w, requires_grad=True), torch.tensor(b, requires_grad=True)) for w, b in params]
    a = torch.from_numpy(x).permute(0, 3, 1, 2)
    for k, (w, b) in enumerate(tp):
        a = torch.nn.functional.conv2d(a, w.permute(0, 3, 1, 2), b, padding=dils[k], dilation=dils[k])
        if k < len(tp) - 1:
            a = torch.relu(a)
    tl = ((a.permute(0, 2, 3, 1) - torch.from_numpy(y)) ** 2).mean()
    tl.backward()
    assert abs(loss - tl.item()) < 1e-12 * max(1.0, abs(loss))
    for (gw, gb), (w, b) in zip(grads, tp):
        np.testing.assert_allclose(gw, w.grad.numpy(), rtol=1e-10, atol=1e-12)
        np.testing.assert_allclose(gb, b.grad.numpy(), rtol=1e-10, atol=1e-12)


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(2)
    params = rand_params(rng, [2, 3, 1])
    x = rng.standard_normal((1, 4, 4, 2))
    y = rng.standard_normal((1, 4, 4, 1))
    _, grads = conv_ref.loss_and_grads(params, x, y)
    eps = 1e-6
    for k in range(len(params)):
        w, b = params[k]
        for idx in [(0, 0, 0, 0), (w.shape[0] - 1, 2, 1, w.shape[3] - 1), (0, 1, 2, 0)]:
            wp = w.copy(); wp[idx] += eps
            wm = w.copy(); wm[idx] -= eps
            pp = list(params); pp[k] = (wp, b)
            pm = list(params); pm[k] = (wm, b)
            fd = (conv_ref.loss_and_grads(pp, x, y)[0] - conv_ref.loss_and_grads(pm, x, y)[0]) / (2 * eps)
            assert abs(fd - grads[k][0][idx]) < 1e-6 * max(1.0, abs(fd))
