"""Surrogate network kernels (dd_sur_*) against the FP64 reference of oracle/conv_ref.py,
plus training and the exact fallback.  Inputs are rounded to BF16 first and fed to both
sides, so the differences come only from FP32 accumulation and the BF16 rounding of
the GPU's BF16 outputs (relative 2^-8)."""
import math

import numpy as np
import pytest

from oracle import conv_ref
from paper_2507_00294_gb300 import binding as b

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def bf(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(torch.bfloat16)


def r64(t):
    return t.to(torch.float64).cpu().numpy()


def flip(w):  # [co][9][ci] -> [ci][8 - tap][co]
    return np.ascontiguousarray(w[:, ::-1, :].transpose(2, 1, 0))


@pytest.mark.parametrize("ci,co,dil", [(16, 32, 1), (32, 32, 1), (32, 16, 1), (16, 16, 1), (32, 32, 4),
                                         (16, 32, 32), (32, 16, 9)])
def test_conv_forward(cuda, ci, co, dil):
    rng = np.random.default_rng(ci * 100 + co + dil)
    x = bf(rng.standard_normal((2, 40, 128, ci))).to(cuda)
    wt = bf(rng.standard_normal((co, 9, ci)) * 0.2).to(cuda)
    bias = torch.from_numpy(rng.standard_normal(co).astype(np.float32)).to(cuda)
    ref = conv_ref.conv3x3(r64(x), r64(wt).reshape(co, 3, 3, ci), bias.double().cpu().numpy(), dil)
    out = torch.empty((2, 40, 128, co), dtype=torch.bfloat16, device=cuda)
    b.dd_sur_conv3x3(x, wt, bias, None, out, 0, dil)
    relu = np.maximum(ref, 0)
    np.testing.assert_allclose(r64(out), relu, rtol=8e-3, atol=1e-3 * np.abs(ref).max())
    lin = torch.empty((2, 40, 128), dtype=torch.float32, device=cuda)
    b.dd_sur_conv3x3(x, wt, bias, None, lin, 1, dil)
    b.dd_sur_check()                 # no tensor-memory convolution gave up waiting
    np.testing.assert_allclose(r64(lin), ref[..., 0], rtol=1e-4, atol=1e-5 * np.abs(ref).max())


@pytest.mark.parametrize("ci,co,dil", [(32, 32, 1), (32, 16, 1), (32, 32, 8), (32, 16, 32)])
def test_conv_data_gradient(cuda, ci, co, dil):
    rng = np.random.default_rng(7 + ci + co + dil)
    wt = rng.standard_normal((co, 9, ci)) * 0.2
    dz = bf(rng.standard_normal((2, 36, 128, co))).to(cuda)
    a = bf(rng.standard_normal((2, 36, 128, ci))).to(cuda)    # layer input, ReLU mask = a > 0
    wfl = bf(flip(r64(bf(wt)))).to(cuda)
    out = torch.empty((2, 36, 128, ci), dtype=torch.bfloat16, device=cuda)
    b.dd_sur_conv3x3(dz, wfl, None, a, out, 2, dil)
    b.dd_sur_check()
    ref = conv_ref.conv3x3_dgrad(r64(dz), r64(bf(wt)).reshape(co, 3, 3, ci), dil) * (r64(a) > 0)
    np.testing.assert_allclose(r64(out), ref, rtol=8e-3, atol=1e-3 * np.abs(ref).max())


def test_tensor_core_wait_timeout_is_reported(cuda, monkeypatch):
    """Failure detection without a GPU fault: with DD_FAULT=tc_wait no MMA is issued, the
    tensor-memory convolution's completion wait runs out (bounded), the CTA releases its
    TMEM and returns, and dd_sur_check reports DD_ETIMEOUT; the next call runs normally."""
    rng = np.random.default_rng(77)
    x = bf(rng.standard_normal((1, 8, 128, 32))).to(cuda)
    wt = bf(rng.standard_normal((32, 9, 32)) * 0.2).to(cuda)
    bias = torch.from_numpy(rng.standard_normal(32).astype(np.float32)).to(cuda)
    out = torch.empty((1, 8, 128, 32), dtype=torch.bfloat16, device=cuda)
    monkeypatch.setenv("DD_FAULT", "tc_wait")
    b.dd_sur_conv3x3(x, wt, bias, None, out, 0, 1)
    with pytest.raises(b.DDError) as e:
        b.dd_sur_check()
    assert e.value.status == b.DD_ETIMEOUT
    monkeypatch.delenv("DD_FAULT")
    b.dd_sur_conv3x3(x, wt, bias, None, out, 0, 1)
    b.dd_sur_check()
    ref = conv_ref.conv3x3(r64(x), r64(wt).reshape(32, 3, 3, 32), bias.double().cpu().numpy(), 1)
    np.testing.assert_allclose(r64(out), np.maximum(ref, 0), rtol=8e-3, atol=1e-3 * np.abs(ref).max())


@pytest.mark.parametrize("ci,co,dil", [(32, 32, 2), (16, 16, 32)])
def test_conv_forward_64_pixel_tiles(cuda, ci, co, dil):
    """Rows that are not a multiple of 128 pixels (W = 192) take the 64-pixel mma.sync
    tiles instead of the 128-pixel tensor-memory tile: same results."""
    rng = np.random.default_rng(31 + ci + co + dil)
    x = bf(rng.standard_normal((1, 24, 192, ci))).to(cuda)
    wt = bf(rng.standard_normal((co, 9, ci)) * 0.2).to(cuda)
    bias = torch.from_numpy(rng.standard_normal(co).astype(np.float32)).to(cuda)
    ref = conv_ref.conv3x3(r64(x), r64(wt).reshape(co, 3, 3, ci), bias.double().cpu().numpy(), dil)
    out = torch.empty((1, 24, 192, co), dtype=torch.bfloat16, device=cuda)
    b.dd_sur_conv3x3(x, wt, bias, None, out, 0, dil)
    np.testing.assert_allclose(r64(out), np.maximum(ref, 0), rtol=8e-3, atol=1e-3 * np.abs(ref).max())


@pytest.mark.parametrize("ci,co,dil", [(16, 32, 1), (32, 32, 1), (32, 16, 1), (32, 32, 16), (16, 32, 32)])
def test_conv_weight_gradient(cuda, ci, co, dil):
    rng = np.random.default_rng(11 + ci + co + dil)
    x = bf(rng.standard_normal((3, 40, 128, ci))).to(cuda)
    dz = bf(rng.standard_normal((3, 40, 128, co))).to(cuda)
    part = torch.zeros(608 * (co * 9 * ci + co), dtype=torch.float32, device=cuda)
    grad = torch.empty(co * 9 * ci + co, dtype=torch.float32, device=cuda)
    b.dd_sur_wgrad(x, dz, part, grad, dil)
    dw, db = conv_ref.conv3x3_wgrad(r64(x), r64(dz), dil)
    g = grad.double().cpu().numpy()
    np.testing.assert_allclose(g[: co * 9 * ci], dw.reshape(-1), rtol=1e-4, atol=1e-5 * np.abs(dw).max())
    np.testing.assert_allclose(g[co * 9 * ci:], db, rtol=1e-4, atol=1e-5 * np.abs(db).max())


def test_network_gradients_match_reference(cuda):
    from paper_2507_00294_gb300 import surrogate as sur
    net = sur.Net(cuda, seed=3)
    B = 2
    net.buffers(B)
    rng = np.random.default_rng(5)
    x = np.zeros((B, 128, 128, 16))
    x[..., :4] = rng.standard_normal((B, 128, 128, 4))
    net.x.copy_(bf(x).to(cuda))
    target = torch.from_numpy(rng.standard_normal((B, 128, 128)).astype(np.float32)).to(cuda)
    net.forward()
    loss = float(net.backward(target).item()) / (B * 128 * 128)
    params = []
    for k, (ci, co) in enumerate(sur.LAYERS):
        wt = r64(net.wb[k]).reshape(co, 3, 3, ci)
        bias = net.params[k][co * 9 * ci:].double().cpu().numpy()
        if k == len(sur.LAYERS) - 1:          # the last layer's real output is channel 0
            wt, bias = wt[:1], bias[:1]
        params.append((wt, bias))
    ref_loss, ref_grads = conv_ref.loss_and_grads(params, r64(net.x), target.double().cpu().numpy()[..., None],
                                                  list(net.dil))
    assert abs(loss / ref_loss - 1) < 2e-2
    for k, (ci, co) in enumerate(sur.LAYERS):
        g = net.grads[k].double().cpu().numpy()
        if k == len(sur.LAYERS) - 1:
            g = np.concatenate([g[: co * 9 * ci].reshape(co, 9 * ci)[:1].reshape(-1), g[co * 9 * ci:][:1]])
        ref = np.concatenate([ref_grads[k][0].reshape(-1), ref_grads[k][1]])
        cos = g @ ref / (np.linalg.norm(g) * np.linalg.norm(ref) + 1e-300)
        assert cos > 0.995, (k, cos)
        assert np.linalg.norm(g - ref) <= 0.06 * np.linalg.norm(ref), k


def test_target_field_and_spot_error_kernels(cuda):
    from paper_2507_00294_gb300 import surrogate as sur
    rng = np.random.default_rng(4)
    n_maps, hw = 3, 128 * 128
    psi = 10.0 ** rng.uniform(-40, 12, (n_maps, hw))
    scale = np.array([1e-12, 3e-13, 2e-12])
    t = torch.empty((n_maps, hw), dtype=torch.float32, device=cuda)
    b.dd_sur_targets(torch.from_numpy(psi).to(cuda), torch.from_numpy(scale).to(cuda), n_maps, hw,
                     sur.FLOOR_REL, sur.MU, sur.SIGMA, t)
    f = psi * scale[:, None]
    lo = f.max(axis=1, keepdims=True) * 10.0 ** sur.FLOOR_REL
    expect = (np.log10(np.maximum(f, lo)) - sur.MU) / sur.SIGMA
    np.testing.assert_allclose(t.double().cpu().numpy(), expect, rtol=1e-6, atol=1e-6)
    back = torch.empty((n_maps, hw), dtype=torch.float64, device=cuda)
    b.dd_sur_fields(t, torch.from_numpy(scale).to(cuda), n_maps, hw, sur.MU, sur.SIGMA, back)
    keep = f > lo
    np.testing.assert_allclose(back.cpu().numpy()[keep], psi[keep], rtol=5e-5)
    idx = rng.choice(hw, (n_maps, 64)).astype(np.int32)
    exact = np.take_along_axis(psi, idx, 1) * (1 + 0.01 * rng.standard_normal((n_maps, 64)))
    err = torch.empty(n_maps, dtype=torch.float64, device=cuda)
    b.dd_sur_spot_error(t, torch.from_numpy(idx).to(cuda), torch.from_numpy(exact).to(cuda),
                        torch.from_numpy(scale).to(cuda), n_maps, hw, 64, sur.MU, sur.SIGMA, err)
    pred_v = back.cpu().numpy()
    ref = [np.linalg.norm(np.take_along_axis(pred_v, idx, 1)[m] - exact[m]) / np.linalg.norm(exact[m])
           for m in range(n_maps)]
    np.testing.assert_allclose(err.cpu().numpy(), ref, rtol=1e-9)


def test_adam_and_input_planes(cuda):
    rng = np.random.default_rng(9)
    n = 32 * 9 * 16
    p0 = rng.standard_normal(n).astype(np.float32)
    g = rng.standard_normal(n).astype(np.float32)
    p = torch.from_numpy(p0.copy()).to(cuda)
    m = torch.zeros(n, device=cuda)
    v = torch.zeros(n, device=cuda)
    wb = torch.empty(n, dtype=torch.bfloat16, device=cuda)
    wf = torch.empty(n, dtype=torch.bfloat16, device=cuda)
    b.dd_sur_adam(p, torch.from_numpy(g).to(cuda), m, v, 1e-2, 1, w_bf16=wb, w_flip=wf, cin=16, cout=32)
    # first Adam step with zero moments moves every weight by lr * g / (|g| + eps')
    mh, vh = g, g * g
    expect = p0 - 1e-2 * mh / (np.sqrt(vh) + 1e-8)
    np.testing.assert_allclose(p.cpu().numpy(), expect, rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(r64(wb), expect, rtol=8e-3)
    np.testing.assert_array_equal(r64(wf).reshape(16, 9, 32), flip(r64(wb).reshape(32, 9, 16)))
    tmap = np.full((2, 128, 128), -1.0, np.float32)
    tmap[0, 3, 5] = 0.25
    tmap[1, 0, 0] = 0.0
    scal = np.array([[0.5, -1.0], [1.5, 2.0]], np.float32)
    x = torch.empty((2, 128, 128, 16), dtype=torch.bfloat16, device=cuda)
    b.dd_sur_planes(torch.from_numpy(tmap).to(cuda), torch.from_numpy(scal).to(cuda), x)
    xh = r64(x)
    assert xh[0, 3, 5, 0] == 0.25 and xh[0, 3, 5, 1] == 1.0 and xh[0, 3, 4, 1] == 0.0
    assert xh[1, 0, 0, 0] == 0.0 and xh[1, 0, 0, 1] == 1.0
    assert np.all(xh[0, ..., 2] == 0.5) and np.all(xh[1, ..., 3] == 2.0) and np.all(xh[..., 4:] == 0)


def test_background_planes(cuda):
    """dd_sur_planes_bg: the first four planes as dd_sur_planes, then each background
    visit's own term ln(w1/w0) (Eq. 3/4 at rho = 0) in the target's normalised log10 units
    and the background mask, against the same numbers formed in FP64."""
    import torch
    from paper_2507_00294_gb300 import surrogate as sur
    rng = np.random.default_rng(12)
    B = 3
    tmap = np.full((B, 128, 128), -1.0, np.float32)
    ages = rng.integers(1, 5000, (B, 400))
    for m in range(B):
        idx = rng.choice(128 * 128, 400, replace=False)
        tmap[m].reshape(-1)[idx] = (1.0 / ages[m]).astype(np.float32)
    kap = np.array([4e-4, 0.24, 40.0], np.float32)
    scal = np.stack([rng.normal(size=B), rng.normal(size=B), kap], axis=1).astype(np.float32)
    x = torch.empty((B, 128, 128, 16), dtype=torch.bfloat16, device=cuda)
    s_dim, k_exact = 0.04, 64
    b.dd_sur_planes_bg(torch.from_numpy(tmap).to(cuda), torch.from_numpy(scal).to(cuda), s_dim, k_exact,
                       sur.MU, sur.SIGMA, x)
    xh = r64(x)
    x4 = torch.empty_like(x)
    b.dd_sur_planes(torch.from_numpy(tmap).to(cuda), torch.from_numpy(np.ascontiguousarray(scal[:, :2])).to(cuda), x4)
    np.testing.assert_array_equal(xh[..., :4], r64(x4)[..., :4])
    age = np.where(tmap > 0, 1.0 / np.maximum(tmap.astype(np.float64), 1e-30), 0.0)
    bg = (tmap > 0) & (age > k_exact + 0.5)
    k = np.broadcast_to(kap.astype(np.float64)[:, None, None], tmap.shape)
    ref = np.zeros(tmap.shape)
    own = np.log1p(4 * k[bg] / (2 * s_dim + 4 * k[bg] * (age[bg] - 1)))
    ref[bg] = (np.log10(own) - sur.MU) / sur.SIGMA
    assert np.all(xh[..., 5] == bg.astype(np.float64))
    np.testing.assert_allclose(xh[..., 4], ref, rtol=8e-3, atol=1e-6)
    assert np.all(xh[..., 6:] == 0)


def test_training_reduces_loss_and_fallback_is_exact(cuda):
    from paper_2507_00294_gb300 import surrogate as sur
    specs, tmap, scal, target = sur.build_dataset(96, seed=123, device=cuda)
    net = sur.Net(cuda, seed=1)
    losses = sur.train(net, tmap, scal, target, epochs=6, batch=16, lr=3e-3)
    assert losses[-1] < 0.5 * losses[0], losses
    exact = sur.exact_fields(specs[:32], cuda).view(32, -1)
    fields, fell_back, est, secs = sur.infer_with_fallback(net, specs[:32], tmap[:32], scal[:32], cuda,
                                                           threshold=1e-2)
    fb = np.nonzero(fell_back)[0]
    kept = np.nonzero(~fell_back)[0]
    if len(fb):
        assert torch.equal(fields[torch.from_numpy(fb).to(cuda)], exact[torch.from_numpy(fb).to(cuda)])
    assert np.all(est[kept] <= 1e-2)
    # a network that has not been trained is always caught by the spot check
    fresh = sur.Net(cuda, seed=2)
    _, fell, _, _ = sur.infer_with_fallback(fresh, specs[:8], tmap[:8], scal[:8], cuda)
    assert fell.all()


def test_checkpoint_resume_continues_identically(cuda, tmp_path):
    from paper_2507_00294_gb300 import surrogate as sur
    specs, tmap, scal, target = sur.build_dataset(32, seed=77, device=cuda)
    a = sur.Net(cuda, seed=4)
    sur.train(a, tmap, scal, target, epochs=1, batch=16, seed=1)
    path = str(tmp_path / "ckpt.npz")
    a.save(path)
    c = sur.Net.load(path, cuda)
    assert c.step_count == a.step_count
    la = sur.train(a, tmap, scal, target, epochs=1, batch=16, seed=2)
    lc = sur.train(c, tmap, scal, target, epochs=1, batch=16, seed=2)
    assert la == lc
    for pa, pc in zip(a.state(), c.state()):
        np.testing.assert_array_equal(pa, pc)


def test_weighted_loss_kernels(cuda):
    """dd_sur_weights and dd_sur_wmse against their definitions in numpy."""
    import torch
    rng = np.random.default_rng(3)
    n_maps, hw = 3, 128 * 128
    t = rng.uniform(-1.0, 1.2, (n_maps, hw)).astype(np.float32)
    mu, sg, alpha = -3.0, 3.0, 0.9
    wt = torch.empty((n_maps, hw), dtype=torch.float32, device=cuda)
    b.dd_sur_weights(torch.from_numpy(t).to(cuda), n_maps, hw, mu, sg, alpha, wt)
    f = 10.0 ** (t.astype(np.float64) * sg + mu)
    want = alpha * hw * f ** 2 / np.sum(f ** 2, axis=1, keepdims=True) + (1 - alpha)
    np.testing.assert_allclose(wt.cpu().numpy(), want, rtol=1e-5)
    assert np.allclose(wt.cpu().numpy().mean(axis=1), 1.0, rtol=1e-4)     # mean weight 1 per map
    pred = (t + rng.normal(0, 0.01, t.shape)).astype(np.float32)
    n = pred.size
    dz = torch.zeros((n, 16), dtype=torch.bfloat16, device=cuda)
    bs = torch.zeros((n + 255) // 256, dtype=torch.float64, device=cuda)
    ls = torch.zeros(1, dtype=torch.float64, device=cuda)
    b.dd_sur_wmse(torch.from_numpy(pred).to(cuda), torch.from_numpy(t).to(cuda), wt, dz, bs, ls)
    d = pred.astype(np.float64) - t
    w64 = wt.cpu().numpy().astype(np.float64)
    assert float(ls.item()) == pytest.approx(np.sum(w64 * d * d), rel=1e-6)
    g = dz.float().cpu().numpy()
    np.testing.assert_allclose(g[:, 0], (2 * w64 * d / n).reshape(-1), rtol=1e-2, atol=1e-12)
    assert np.all(g[:, 1:] == 0)


def test_background_plus_last_visits_is_the_whole_field(cuda):
    """The surrogate's split of a scan: the exact field of its first n - K visits at the
    scan's end plus that of its last K visits, each seen in its own clock, equals the whole
    scan's field (FP64, to its tolerance), on the canvas."""
    from paper_2507_00294_gb300 import surrogate as sur
    specs = sur.draw_scans(6, seed=31)
    parts = [sur.split_scan(s) for s in specs]
    whole = sur.exact_fields(specs, cuda, prec="fp64").view(6, -1).cpu().numpy()
    bg = sur.exact_fields([p[0] for p in parts], cuda, prec="fp64", times=[p[1] for p in parts]).view(6, -1)
    near = sur.exact_fields([p[2] for p in parts], cuda, prec="fp64", times=[p[3] for p in parts]).view(6, -1)
    total = (bg + near).cpu().numpy()
    m = whole > 1e-12 * whole.max(axis=1, keepdims=True)
    assert np.max(np.abs(total[m] / whole[m] - 1.0)) <= 1e-12
    for s, (b_, _, n_, _) in zip(specs, parts):
        assert b.Scan(b_).visits()[0].size + b.Scan(n_).visits()[0].size == b.Scan(s).visits()[0].size
