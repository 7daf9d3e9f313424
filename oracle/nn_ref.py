"""FP64 numpy reference of the warm-start network layers -- TEST INFRASTRUCTURE ONLY.

Plain definitions, written for checking the CUDA kernels: NHWC tensors,
weights [taps][cout][cin] with taps = 9 (3x3, zero padding) or 1 (1x1).
    conv:        y[p, co] = b[co] + sum_{t, ci} x[p + off_t, ci] w[t, co, ci]
    conv_dx:     the adjoint of conv in x (gradient wrt the input)
    conv_dw/db:  the gradients wrt weights and bias
    pool2/up2:   2x2 average pooling and nearest-neighbour 2x upsampling, with adjoints
    mse:         masked mean squared error and its gradient
    adamw:       one AdamW step (Loshchilov & Hutter 2019)
    targets:     the normalised steady fields the network learns
Shares no code with the CUDA library.
"""
from __future__ import annotations

import numpy as np

OFFSETS9 = [(dy, dx) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def _offsets(taps):
    return OFFSETS9 if taps == 9 else [(0, 0)]


def _shift(x, dy, dx):
    """s[n, y, x, c] = x[n, y + dy, x + dx, c], zero outside."""
    N, H, W, C = x.shape
    out = np.zeros_like(x)
    ys, ye = max(0, -dy), min(H, H - dy)
    xs, xe = max(0, -dx), min(W, W - dx)
    out[:, ys:ye, xs:xe] = x[:, ys + dy:ye + dy, xs + dx:xe + dx]
    return out


def conv(x, w, b=None, relu=False):
    taps = w.shape[0]
    y = np.zeros(x.shape[:3] + (w.shape[1],))
    for t, (dy, dx) in enumerate(_offsets(taps)):
        y += np.einsum("nhwc,oc->nhwo", _shift(x, dy, dx), w[t])
    if b is not None:
        y = y + b
    return np.maximum(y, 0.0) if relu else y


def conv_dx(gy, w):
    """sum over taps of g shifted back by the tap offset, times w[t]."""
    taps = w.shape[0]
    gx = np.zeros(gy.shape[:3] + (w.shape[2],))
    for t, (dy, dx) in enumerate(_offsets(taps)):
        gx += _shift(np.einsum("nhwo,oc->nhwc", gy, w[t]), -dy, -dx)
    return gx


def conv_dw(x, gy, taps):
    dw = np.zeros((taps, gy.shape[3], x.shape[3]))
    for t, (dy, dx) in enumerate(_offsets(taps)):
        dw[t] = np.einsum("nhwo,nhwc->oc", gy, _shift(x, dy, dx))
    return dw


def conv_db(gy):
    return gy.sum(axis=(0, 1, 2))


def relu_bwd(y, gy):
    return np.where(y > 0, gy, 0.0)


def pool2(x):
    N, H, W, C = x.shape
    return x.reshape(N, H // 2, 2, W // 2, 2, C).mean(axis=(2, 4))


def pool2_bwd(gy):
    return np.repeat(np.repeat(gy, 2, axis=1), 2, axis=2) / 4.0


def up2(x):
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def up2_bwd(gy):
    N, H, W, C = gy.shape
    return gy.reshape(N, H // 2, 2, W // 2, 2, C).sum(axis=(2, 4))


def mse(pred, target, solid, inv_count, weights=None):
    """pred [..., >=nout], target [..., nout], solid bool [...], per-channel
    weights (default 1); returns (loss, grad)."""
    nout = target.shape[-1]
    wc = np.ones(nout) if weights is None else np.asarray(weights, float)
    d = pred[..., :nout] - target
    fl = (~solid)[..., None]
    loss = float((wc * d * d * fl).sum() * inv_count)
    g = np.zeros_like(pred)
    g[..., :nout] = 2.0 * wc * d * fl * inv_count
    return loss, g


def adamw(p, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8, wd=0.0):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    p = p - lr * (mh / (np.sqrt(vh) + eps) + wd * p)
    return p, m, v


def make_input(solid, tau_feat):
    H, W = solid.shape
    x = np.zeros((H, W, 16))
    x[..., 0] = solid.astype(float)
    x[..., 1] = np.arange(W)[None, :] / max(W - 1, 1)
    x[..., 2] = tau_feat
    return x


def targets(solid, rho, ux, uy, tau, drho, rho_out=1.0):
    """((rho - rho_out)/drho - (1 - x/(nx - 1)), u nu (nx - 1)/(c_s^2 drho)) on
    fluid nodes (the density as its deviation from the linear ramp), 0 on solids."""
    nx = solid.shape[1]
    s = (tau - 0.5) / 3.0 * (nx - 1) / (drho / 3.0)
    ramp = 1.0 - np.arange(nx)[None, :] / (nx - 1)
    t = np.stack([(rho - rho_out) / drho - ramp, ux * s, uy * s], axis=-1)
    t[solid.astype(bool)] = 0.0
    return t


def bf16_round(a):
    """Round FP32/FP64 values to the nearest bfloat16 (ties to even)."""
    f = np.asarray(a, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = ((u + 0x7FFF + lsb) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)
