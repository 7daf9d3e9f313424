"""Pins of the FP64 network-layer reference against independent facts:
scipy's correlate, finite differences, adjointness identities, the closed form
of AdamW's first step, and bfloat16 rounding of exactly representable ties."""
import numpy as np
import pytest

from oracle import nn_ref as R

scipy_signal = pytest.importorskip("scipy.signal")


def _rand(shape, seed):
    return np.random.default_rng(seed).standard_normal(shape)


def test_conv_matches_scipy_correlate():
    x = _rand((1, 7, 9, 3), 1)
    w = _rand((9, 2, 3), 2)
    y = R.conv(x, w)
    for co in range(2):
        ref = np.zeros((7, 9))
        for ci in range(3):
            k = w[:, co, ci].reshape(3, 3)
            ref += scipy_signal.correlate(x[0, :, :, ci], k, mode="same")
        assert np.allclose(y[0, :, :, co], ref, atol=1e-12)


@pytest.mark.parametrize("taps", [9, 1])
def test_conv_gradients_by_finite_differences(taps):
    x = _rand((2, 5, 6, 3), 3)
    w = _rand((taps, 4, 3), 4)
    b = _rand(4, 5)
    gy = _rand((2, 5, 6, 4), 6)
    L = lambda x_, w_, b_: float((gy * R.conv(x_, w_, b_)).sum())  # noqa: E731
    gx, gw, gb = R.conv_dx(gy, w), R.conv_dw(x, gy, taps), R.conv_db(gy)
    eps = 1e-6
    rng = np.random.default_rng(7)
    for _ in range(6):
        i = tuple(rng.integers(0, s) for s in x.shape)
        d = np.zeros_like(x)
        d[i] = eps
        assert gx[i] == pytest.approx((L(x + d, w, b) - L(x - d, w, b)) / (2 * eps), rel=1e-6, abs=1e-8)
        j = tuple(rng.integers(0, s) for s in w.shape)
        d = np.zeros_like(w)
        d[j] = eps
        assert gw[j] == pytest.approx((L(x, w + d, b) - L(x, w - d, b)) / (2 * eps), rel=1e-6, abs=1e-8)
    d = np.zeros_like(b)
    d[1] = eps
    assert gb[1] == pytest.approx((L(x, w, b + d) - L(x, w, b - d)) / (2 * eps), rel=1e-6)


def test_adjoint_identities():
    x = _rand((2, 6, 8, 3), 8)
    w = _rand((9, 5, 3), 9)
    y = _rand((2, 6, 8, 5), 10)
    assert (R.conv(x, w) * y).sum() == pytest.approx((x * R.conv_dx(y, w)).sum(), rel=1e-12)
    p = _rand((2, 3, 4, 3), 11)
    assert (R.pool2(x) * p).sum() == pytest.approx((x * R.pool2_bwd(p)).sum(), rel=1e-12)
    u = _rand((2, 12, 16, 3), 12)
    assert (R.up2(x) * u).sum() == pytest.approx((x * R.up2_bwd(u)).sum(), rel=1e-12)
    # pooling an upsampled field gives the field back
    assert np.allclose(R.pool2(R.up2(x)), x)


def test_mse_gradient_by_finite_differences():
    pred = _rand((4, 5, 16), 13)
    tgt = _rand((4, 5, 3), 14)
    solid = np.random.default_rng(15).random((4, 5)) < 0.3
    inv = 1.0 / (3 * (~solid).sum())
    loss, g = R.mse(pred, tgt, solid, inv)
    assert np.all(g[..., 3:] == 0) and np.all(g[solid] == 0)
    eps = 1e-6
    for i in [(1, 2, 0), (3, 4, 2), (0, 0, 1)]:
        d = np.zeros_like(pred)
        d[i] = eps
        fd = (R.mse(pred + d, tgt, solid, inv)[0] - R.mse(pred - d, tgt, solid, inv)[0]) / (2 * eps)
        assert g[i] == pytest.approx(fd, rel=1e-6, abs=1e-10)


def test_adamw_first_step_closed_form():
    # after one step with m = v = 0, the bias-corrected update is g/(|g| + eps)
    p = np.array([0.5, -2.0, 3.0])
    g = np.array([0.1, -4.0, 0.0])
    lr, wd, eps = 0.01, 0.1, 1e-8
    p1, _, _ = R.adamw(p, g, np.zeros(3), np.zeros(3), 1, lr, eps=eps, wd=wd)
    want = p - lr * (g / (np.abs(g) + eps) + wd * p)
    assert np.allclose(p1, want, rtol=1e-12, atol=1e-15)


def test_bf16_rounding():
    assert R.bf16_round(1.0) == 1.0
    assert R.bf16_round(1.0 + 2.0 ** -8) == 1.0            # tie, even neighbour kept
    assert R.bf16_round(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6  # tie, rounds to even (up)
    assert R.bf16_round(1.0 + 2.0 ** -8 + 2.0 ** -12) == 1.0 + 2.0 ** -7
