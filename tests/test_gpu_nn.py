"""Warm-start network kernels vs the FP64 reference (oracle/nn_ref.py), and the
learned warm start end to end.

Inputs and weights are rounded to bfloat16 once and both sides use the same
rounded values.  Results accumulated in FP32 (FP32 copies of the convolution
output, weight gradients, AdamW) are compared at 1e-4 of the largest
magnitude: a sum of at most a few hundred FP32 terms.  Results stored as
bfloat16 (8 significant bits) are compared at 1e-2 of the largest magnitude.
Whole-network gradients are compared by cosine similarity >= 0.999.
"""
import numpy as np
import pytest

import oracle as O
from oracle import nn_ref as R
from paper_1609_09685_gb300 import build, lbm

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    lbm.load()
    O.build()


def _bf(a):
    """bf16-rounded numpy array and the matching CUDA tensor."""
    r = R.bf16_round(a)
    return r, torch.tensor(r, dtype=torch.float32, device="cuda").to(torch.bfloat16).contiguous()


def _np(t):
    return t.float().cpu().numpy().astype(np.float64)


def _close(a, b, rel):
    scale = max(np.abs(b).max(), 1e-30)
    assert np.abs(a - b).max() <= rel * scale, (np.abs(a - b).max(), scale)


@pytest.mark.parametrize("taps,cin,cout,shape", [(9, 16, 16, (2, 5, 9)), (9, 32, 48, (1, 7, 130)),
                                                 (1, 16, 16, (2, 4, 6)), (9, 48, 32, (3, 2, 4))])
def test_conv_forward_backward(taps, cin, cout, shape):
    n, h, w = shape
    rng = np.random.default_rng(taps * 100 + cin)
    x, xt = _bf(rng.standard_normal((n, h, w, cin)))
    wt_, wtt = _bf(rng.standard_normal((taps, cout, cin)) * 0.2)
    b = rng.standard_normal(cout).astype(np.float32)
    bt = torch.tensor(b, device="cuda")
    y = torch.empty((n, h, w, cout), dtype=torch.bfloat16, device="cuda")
    y32 = torch.empty((n, h, w, cout), dtype=torch.float32, device="cuda")
    lbm.lbm_nn_conv_fwd(xt, n, h, w, cin, wtt, bt, taps, cout, 1, y, y32)
    ref = R.conv(x, wt_, b.astype(np.float64), relu=True)
    _close(_np(y32), ref, 1e-4)
    _close(_np(y), ref, 1e-2)
    # data and weight gradients
    gy, gyt = _bf(rng.standard_normal((n, h, w, cout)))
    gx = torch.empty((n, h, w, cin), dtype=torch.bfloat16, device="cuda")
    flip = torch.empty((taps, cin, cout), dtype=torch.bfloat16, device="cuda")
    lbm.lbm_nn_conv_bwd_data(gyt, n, h, w, cout, wtt, taps, cin, flip, gx)
    _close(_np(gx), R.conv_dx(gy, wt_), 1e-2)
    dw = torch.empty((taps, cout, cin), dtype=torch.float32, device="cuda")
    db = torch.empty(cout, dtype=torch.float32, device="cuda")
    scratch = torch.empty(1 << 20, dtype=torch.float32, device="cuda")
    lbm.lbm_nn_conv_bwd_weight(xt, gyt, n, h, w, cin, cout, taps, dw, db, 0, scratch, scratch.numel())
    _close(_np(dw), R.conv_dw(x, gy, taps), 1e-4)
    _close(_np(db), R.conv_db(gy), 1e-4)


def test_pool_upsample_copy_relu_add():
    rng = np.random.default_rng(3)
    n, h, w, c = 2, 6, 10, 16
    x, xt = _bf(rng.standard_normal((n, h, w, c)))
    p = torch.empty((n, h // 2, w // 2, c), dtype=torch.bfloat16, device="cuda")
    lbm.lbm_nn_pool2_fwd(xt, n, h, w, c, p)
    _close(_np(p), R.pool2(x), 1e-2)
    gp, gpt = _bf(rng.standard_normal((n, h // 2, w // 2, c)))
    gi = torch.empty_like(xt)
    lbm.lbm_nn_pool2_bwd(gpt, n, h, w, c, gi)
    _close(_np(gi), R.pool2_bwd(gp), 1e-2)
    u = torch.empty((n, 2 * h, 2 * w, c), dtype=torch.bfloat16, device="cuda")
    lbm.lbm_nn_up2_fwd(xt, n, h, w, c, u)
    assert np.array_equal(_np(u), R.up2(x))
    gu, gut = _bf(rng.standard_normal((n, 2 * h, 2 * w, c)))
    gx = torch.empty_like(xt)
    lbm.lbm_nn_up2_bwd(gut, n, h, w, c, gx)
    _close(_np(gx), R.up2_bwd(gu), 1e-2)
    cat = torch.zeros((n, h, w, 2 * c), dtype=torch.bfloat16, device="cuda")
    lbm.lbm_nn_copy_channels(xt, c, 0, cat, 2 * c, c, c, n * h * w)
    assert np.array_equal(_np(cat)[..., c:], x) and np.all(_np(cat)[..., :c] == 0)
    g = torch.empty_like(xt)
    lbm.lbm_nn_relu_bwd(xt, gut[:, :h, :w].contiguous(), g, g.numel())
    assert np.array_equal(_np(g), R.relu_bwd(x, gu[:, :h, :w]))
    s = torch.empty_like(xt)
    lbm.lbm_nn_add(xt, xt, s, s.numel())
    assert np.array_equal(_np(s), 2 * x)


def test_mse_adamw_input():
    rng = np.random.default_rng(4)
    npix = 300
    pred, predt = _bf(rng.standard_normal((npix, 16)))
    tgt = rng.standard_normal((npix, 3)).astype(np.float32)
    solid = (rng.random(npix) < 0.3).astype(np.uint8)
    inv = 1.0 / (3 * int((solid == 0).sum()))
    grad = torch.empty_like(predt)
    part = torch.empty(256, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    lbm.lbm_nn_mse(predt, 16, torch.tensor(tgt, device="cuda"), torch.tensor(solid, device="cuda"), npix, 3,
                   inv, grad, part, loss, weights=[4.0, 1.0, 0.5])
    lref, gref = R.mse(pred, tgt.astype(np.float64), solid.astype(bool), inv, weights=[4.0, 1.0, 0.5])
    assert float(loss.item()) == pytest.approx(lref, rel=1e-5)
    _close(_np(grad), gref, 1e-2)
    p = rng.standard_normal(1000).astype(np.float32)
    g = rng.standard_normal(1000).astype(np.float32)
    pt, gt = torch.tensor(p, device="cuda"), torch.tensor(g, device="cuda")
    m, v = torch.zeros_like(pt), torch.zeros_like(pt)
    pr, mr, vr = p.astype(np.float64), np.zeros(1000), np.zeros(1000)
    for step in (1, 2, 3):
        lbm.lbm_nn_adamw(pt, gt, m, v, 1000, 1e-2, 0.9, 0.999, 1e-8, 0.01, step)
        pr, mr, vr = R.adamw(pr, g.astype(np.float64), mr, vr, step, 1e-2, wd=0.01)
    _close(pt.cpu().numpy().astype(np.float64), pr, 1e-5)
    solid2 = (rng.random((5, 9)) < 0.4).astype(np.uint8)
    xin = torch.empty((5, 9, 16), dtype=torch.bfloat16, device="cuda")
    lbm.lbm_nn_make_input(torch.tensor(solid2, device="cuda"), 5, 9, 0.37, xin)
    assert np.array_equal(_np(xin), R.bf16_round(R.make_input(solid2, 0.37)))


def test_targets_and_warm_start_match_oracle():
    mask, _ = lbm.lbm_qsgs(5, (32, 64), 0.02, 0.72)
    tau, drho = 0.9, 8e-4
    with lbm.lbm_create_domain(mask, tau, drho) as s:
        lbm.lbm_step(s, 400)
        rho, ux, uy = lbm.lbm_get_fields(s, 0)
        out = torch.empty((32, 64, 3), dtype=torch.float32, device="cuda")
        lbm.lbm_nn_targets(s, 0, out)
        torch.cuda.synchronize()
        ref = R.targets(mask, rho, ux, uy, tau, drho)
        _close(out.cpu().numpy().astype(np.float64), ref, 1e-5)
        # warm start from a bf16 prediction: populations = f_eq of the de-normalised fields
        pred, predt = _bf(np.concatenate([ref, np.zeros((32, 64, 13))], axis=-1) * 1.1)
        lbm.lbm_warm_start(s, 0, predt, 16)
        f = lbm.lbm_get_populations(s, 0)
    scale = (tau - 0.5) / 3.0 * 63 / (drho / 3.0)
    ramp = 1.0 - np.arange(64)[None, :] / 63.0
    r0 = 1.0 + (pred[..., 0] + ramp) * drho
    feq = O.equilibrium(mask, r0, pred[..., 1] / scale, pred[..., 2] / scale)
    fluid = ~mask.astype(bool)
    w = O.lattice(9)[1]
    a, b = (f - w)[fluid], (feq - w)[fluid]
    assert np.abs(a - b).max() <= 2e-6 * np.abs(b).max()


def _ref_unet_forward(chans, x, params):
    """FP64 forward of the same U-Net composition with nn_ref layers."""
    L = len(chans)
    enc_p, dec_p, head_p = params
    cur, skips = x, []
    for l in range(L):
        a1 = R.conv(R.conv(cur, *enc_p[l][0], relu=True), *enc_p[l][1], relu=True)
        skips.append(a1)
        cur = R.pool2(a1) if l < L - 1 else a1
    for l in range(L - 2, -1, -1):
        cat = np.concatenate([R.up2(cur), skips[l]], axis=-1)
        cur = R.conv(R.conv(cat, *dec_p[l][0], relu=True), *dec_p[l][1], relu=True)
    return R.conv(cur, *head_p)


def _ref_unet_backward(net, gout):
    """FP64 backward of the U-Net composition, with nn_ref layer adjoints, from
    the GPU's own saved forward tensors (each layer's input x and output y), so
    the ReLU masks are the same on both sides; returns the weight gradients in
    UNet.layers() order."""
    X = lambda c: _np(c.x)  # noqa: E731
    Y = lambda c: _np(c.y)  # noqa: E731
    W = lambda c: c.w32.cpu().numpy().astype(np.float64)  # noqa: E731
    L, C = net.L, net.chans
    grads = {}

    def conv_bwd(c, g):
        if c.relu:
            g = R.relu_bwd(Y(c), g)
        grads[id(c)] = R.conv_dw(X(c), g, c.taps)
        return R.conv_dx(g, W(c))

    g = conv_bwd(net.head, gout)
    gskip = {}
    for l in range(0, L - 1):
        gcat = conv_bwd(net.dec[l][0], conv_bwd(net.dec[l][1], g))
        gskip[l] = gcat[..., C[l + 1]:]
        g = R.up2_bwd(gcat[..., :C[l + 1]])
    for l in range(L - 1, -1, -1):
        if l < L - 1:
            g = R.pool2_bwd(g) + gskip[l]
        g = conv_bwd(net.enc[l][0], conv_bwd(net.enc[l][1], g))
    return [grads[id(c)] for c in net.layers()]


def test_unet_gradients_match_fp64_composition():
    from paper_1609_09685_gb300.warmstart import UNet
    chans = (16, 32, 32)
    net = UNet(chans, seed=3)
    n, h, w = 2, 8, 16
    rng = np.random.default_rng(8)
    x, xt = _bf(np.concatenate([rng.standard_normal((n, h, w, 3)), np.zeros((n, h, w, 13))], -1))
    for c in net.layers():  # give the biases some value and round the masters to bf16
        c.b32.copy_(torch.tensor(rng.standard_normal(c.cout) * 0.1, dtype=torch.float32))
        c.w32.copy_(torch.tensor(R.bf16_round(c.w32.cpu().numpy()), dtype=torch.float32))
        lbm.lbm_nn_f32_to_bf16(c.w32, c.wbf, c.w32.numel())
    L = len(chans)
    P = lambda c: (c.w32.cpu().numpy().astype(np.float64), c.b32.cpu().numpy().astype(np.float64))  # noqa: E731
    params = ([[P(net.enc[l][0]), P(net.enc[l][1])] for l in range(L)],
              [[P(net.dec[l][0]), P(net.dec[l][1])] if l < L - 1 else None for l in range(L)],
              P(net.head))
    y = net.forward(xt, n, h, w)
    g, gt = _bf(rng.standard_normal((n, h, w, 16)) * 0.1)
    net.backward(gt, n)
    torch.cuda.synchronize()
    ref_out = _ref_unet_forward(chans, x, params)
    assert np.abs(_np(y) - ref_out).max() <= 3e-2 * np.abs(ref_out).max()
    for c, rg in zip(net.layers(), _ref_unet_backward(net, g)):
        dg = c.dw.cpu().numpy().astype(np.float64).ravel()
        cos = dg @ rg.ravel() / (np.linalg.norm(dg) * np.linalg.norm(rg) + 1e-300)
        assert cos >= 0.999, cos


def test_trained_warm_start_beats_equilibrium_start():
    """A small U-Net trained on solver-generated solutions must reach the
    permeability (within 1e-4 of the converged k) in fewer steps than the
    equilibrium start on held-out masks, without changing the converged k."""
    from paper_1609_09685_gb300 import warmstart as WS
    shape = (64, 128)
    train_doms = WS.make_domains(192, shape, seed0=100, master_seed=1)
    eval_doms = WS.make_domains(8, shape, seed0=100000, master_seed=2)
    ds = WS.generate(train_doms, shape)
    ev = WS.generate(eval_doms, shape)
    net = WS.UNet((16, 32, 32, 64), seed=0)
    hist = WS.train(net, ds, epochs=60, batch=16, lr=2e-3)
    assert hist[-1] < 0.2 * hist[0]
    res = WS.evaluate(net, ev)
    assert res["k_rel_diff_max"] < 1e-4
    assert res["steps_to_k_warm"] < res["steps_to_k_equilibrium"]
