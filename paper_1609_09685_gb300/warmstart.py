"""Learned warm start: a U-Net assembled from the library's kernels.

The network maps (solid mask, x / (nx - 1), tau - 1/2) to the normalised steady
fields of a 2D domain: the density's deviation from the linear inlet-to-outlet
ramp, (rho - rho_out)/drho - (1 - x/(nx - 1)), and u nu (nx - 1)/(c_s^2 drho).
A zero prediction therefore reproduces the equilibrium start's pressure ramp.  Its
prediction only initialises the populations (lbm_warm_start); the lattice
Boltzmann iteration of the paper then converges from there, so a poor
prediction costs time, never accuracy.

This module orders the C-ABI calls of one forward / backward / AdamW step and
owns the buffers (PyTorch CUDA tensors, used only as device memory).  Every
arithmetic step -- convolutions on the tensor cores, pooling, upsampling,
concatenation, loss, optimiser, target extraction and the warm start itself --
runs in the library's kernels.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

from . import lbm

C_IN = 16     # input channels (3 used, padded to the kernels' multiple of 16)
C_OUT = 16    # head channels (3 used)
N_TARGET = 3


def _torch():
    import torch
    return torch


class Conv:
    """One convolution layer (3x3 or 1x1) with optional ReLU."""

    def __init__(self, cin: int, cout: int, taps: int, relu: bool, rng: np.random.Generator, ctx: "Ctx"):
        torch = _torch()
        self.cin, self.cout, self.taps, self.relu, self.ctx = cin, cout, taps, relu, ctx
        bound = math.sqrt(6.0 / (taps * cin)) if relu else math.sqrt(3.0 / (taps * cin))
        w = rng.uniform(-bound, bound, (taps, cout, cin)).astype(np.float32)
        dev = ctx.device
        self.w32 = torch.from_numpy(w).to(dev)
        self.b32 = torch.zeros(cout, dtype=torch.float32, device=dev)
        self.wbf = torch.empty((taps, cout, cin), dtype=torch.bfloat16, device=dev)
        self.dw = torch.zeros_like(self.w32)
        self.db = torch.zeros_like(self.b32)
        self.mw, self.vw = torch.zeros_like(self.w32), torch.zeros_like(self.w32)
        self.mb, self.vb = torch.zeros_like(self.b32), torch.zeros_like(self.b32)
        self.wflip = torch.empty((taps, cin, cout), dtype=torch.bfloat16, device=dev)
        lbm.lbm_nn_f32_to_bf16(self.w32, self.wbf, self.w32.numel(), ctx.stream)
        self.x = self.y = None
        self.shape = None

    @property
    def nparams(self):
        return self.w32.numel() + self.b32.numel()

    def forward(self, x, n, h, w):
        torch = _torch()
        y = torch.empty((n, h, w, self.cout), dtype=torch.bfloat16, device=self.ctx.device)
        lbm.lbm_nn_conv_fwd(x, n, h, w, self.cin, self.wbf, self.b32, self.taps, self.cout, self.relu, y,
                            None, self.ctx.stream)
        self.x, self.y, self.shape = x, y, (n, h, w)
        return y

    def backward(self, gy, need_gx: bool = True):
        torch = _torch()
        n, h, w = self.shape
        g = gy
        if self.relu:
            g = torch.empty_like(gy)
            lbm.lbm_nn_relu_bwd(self.y, gy, g, gy.numel(), self.ctx.stream)
        lbm.lbm_nn_conv_bwd_weight(self.x, g, n, h, w, self.cin, self.cout, self.taps, self.dw, self.db, 0,
                                   self.ctx.scratch, self.ctx.scratch.numel(), self.ctx.stream)
        if not need_gx:
            return None
        gx = torch.empty((n, h, w, self.cin), dtype=torch.bfloat16, device=self.ctx.device)
        lbm.lbm_nn_conv_bwd_data(g, n, h, w, self.cout, self.wbf, self.taps, self.cin, self.wflip, gx,
                                 self.ctx.stream)
        return gx

    def step(self, t: int, lr: float, wd: float):
        s = self.ctx.stream
        lbm.lbm_nn_adamw(self.w32, self.dw, self.mw, self.vw, self.w32.numel(), lr, 0.9, 0.999, 1e-8, wd, t,
                         self.wbf, s)
        lbm.lbm_nn_adamw(self.b32, self.db, self.mb, self.vb, self.b32.numel(), lr, 0.9, 0.999, 1e-8, 0.0, t,
                         None, s)

    def state(self):
        return {"w": self.w32.detach().cpu().numpy(), "b": self.b32.detach().cpu().numpy()}

    def load(self, st):
        torch = _torch()
        self.w32.copy_(torch.from_numpy(st["w"]))
        self.b32.copy_(torch.from_numpy(st["b"]))
        lbm.lbm_nn_f32_to_bf16(self.w32, self.wbf, self.w32.numel(), self.ctx.stream)


@dataclass
class Ctx:
    device: object
    stream: Optional[int]
    scratch: object = None  # FP32 wgrad partial sums


class UNet:
    """L-level U-Net: per level two 3x3 ReLU convolutions, 2x2 average pooling
    down, nearest 2x upsampling + skip concatenation + two 3x3 ReLU convolutions
    up, and a 1x1 head."""

    def __init__(self, chans=(16, 32, 32, 64, 64, 128, 128, 128), seed: int = 0, stream=None,
                 scratch_floats: int = 1 << 24):
        torch = _torch()
        self.chans = list(chans)
        self.L = len(self.chans)
        self.ctx = Ctx(device=torch.device("cuda"), stream=stream)
        self.ctx.scratch = torch.empty(scratch_floats, dtype=torch.float32, device="cuda")
        rng = np.random.default_rng(seed)
        C = self.chans
        self.enc = []
        for l in range(self.L):
            cin = C_IN if l == 0 else C[l - 1]
            self.enc.append([Conv(cin, C[l], 9, True, rng, self.ctx), Conv(C[l], C[l], 9, True, rng, self.ctx)])
        self.dec = [None] * (self.L - 1)
        for l in range(self.L - 2, -1, -1):
            self.dec[l] = [Conv(C[l + 1] + C[l], C[l], 9, True, rng, self.ctx), Conv(C[l], C[l], 9, True, rng, self.ctx)]
        self.head = Conv(C[0], C_OUT, 1, False, rng, self.ctx)
        self.t = 0

    def layers(self) -> List[Conv]:
        out = [c for pair in self.enc for c in pair]
        out += [c for pair in self.dec if pair for c in pair]
        return out + [self.head]

    @property
    def nparams(self):
        return sum(c.nparams for c in self.layers())

    def forward(self, x, n, h, w):
        torch = _torch()
        s = self.ctx.stream
        C = self.chans
        self._skips = []
        self._dims = []
        cur, H, W = x, h, w
        for l in range(self.L):
            cur = self.enc[l][0].forward(cur, n, H, W)
            cur = self.enc[l][1].forward(cur, n, H, W)
            self._skips.append(cur)
            self._dims.append((H, W))
            if l < self.L - 1:
                p = torch.empty((n, H // 2, W // 2, C[l]), dtype=torch.bfloat16, device="cuda")
                lbm.lbm_nn_pool2_fwd(cur, n, H, W, C[l], p, s)
                cur, H, W = p, H // 2, W // 2
        for l in range(self.L - 2, -1, -1):
            Hs, Ws = self._dims[l]
            up = torch.empty((n, Hs, Ws, C[l + 1]), dtype=torch.bfloat16, device="cuda")
            lbm.lbm_nn_up2_fwd(cur, n, Hs // 2, Ws // 2, C[l + 1], up, s)
            cat = torch.empty((n, Hs, Ws, C[l + 1] + C[l]), dtype=torch.bfloat16, device="cuda")
            npix = n * Hs * Ws
            lbm.lbm_nn_copy_channels(up, C[l + 1], 0, cat, C[l + 1] + C[l], 0, C[l + 1], npix, s)
            lbm.lbm_nn_copy_channels(self._skips[l], C[l], 0, cat, C[l + 1] + C[l], C[l + 1], C[l], npix, s)
            cur = self.dec[l][0].forward(cat, n, Hs, Ws)
            cur = self.dec[l][1].forward(cur, n, Hs, Ws)
        return self.head.forward(cur, n, h, w)

    def backward(self, gout, n):
        torch = _torch()
        s = self.ctx.stream
        C = self.chans
        g = self.head.backward(gout)
        gskip = [None] * self.L
        for l in range(0, self.L - 1):
            Hs, Ws = self._dims[l]
            g = self.dec[l][1].backward(g)
            gcat = self.dec[l][0].backward(g)
            npix = n * Hs * Ws
            gup = torch.empty((n, Hs, Ws, C[l + 1]), dtype=torch.bfloat16, device="cuda")
            gs = torch.empty((n, Hs, Ws, C[l]), dtype=torch.bfloat16, device="cuda")
            lbm.lbm_nn_copy_channels(gcat, C[l + 1] + C[l], 0, gup, C[l + 1], 0, C[l + 1], npix, s)
            lbm.lbm_nn_copy_channels(gcat, C[l + 1] + C[l], C[l + 1], gs, C[l], 0, C[l], npix, s)
            gskip[l] = gs
            g2 = torch.empty((n, Hs // 2, Ws // 2, C[l + 1]), dtype=torch.bfloat16, device="cuda")
            lbm.lbm_nn_up2_bwd(gup, n, Hs // 2, Ws // 2, C[l + 1], g2, s)
            g = g2
        # g is now the gradient at the bottom level's output
        for l in range(self.L - 1, -1, -1):
            H, W = self._dims[l]
            if l < self.L - 1:
                gp = torch.empty((n, H, W, C[l]), dtype=torch.bfloat16, device="cuda")
                lbm.lbm_nn_pool2_bwd(g, n, H, W, C[l], gp, s)
                tot = torch.empty_like(gp)
                lbm.lbm_nn_add(gp, gskip[l], tot, tot.numel(), s)
                g = tot
            g = self.enc[l][1].backward(g)
            g = self.enc[l][0].backward(g, need_gx=l > 0)

    def step(self, lr: float, wd: float = 1e-4):
        self.t += 1
        for c in self.layers():
            c.step(self.t, lr, wd)

    def state(self):
        return [c.state() for c in self.layers()]

    def load(self, st):
        for c, s in zip(self.layers(), st):
            c.load(s)


# ---------------------------------------------------------------------------
# data, training and evaluation
# ---------------------------------------------------------------------------
@dataclass
class Dataset:
    h: int
    w: int
    taus: List[float] = field(default_factory=list)
    drhos: List[float] = field(default_factory=list)
    masks_host: List[np.ndarray] = field(default_factory=list)
    solid: object = None    # uint8 [N, h, w] on the device
    inputs: object = None   # bf16 [N, h, w, 16]
    targets: object = None  # fp32 [N, h, w, 3]
    seconds: float = 0.0
    steps: List[int] = field(default_factory=list)

    def __len__(self):
        return len(self.taus)


def make_domains(n: int, shape, seed0: int, porosity=(0.6, 0.8), tau=(0.51, 1.5), master_seed: int = 0):
    """Seeded draws of (mask seed, porosity, tau) for n domains of `shape`."""
    rng = np.random.default_rng(master_seed)
    out = []
    for i in range(n):
        phi = float(rng.uniform(*porosity))
        t = float(rng.uniform(*tau))
        out.append((seed0 + i, phi, t))
    return out


def generate(domains, shape, stream=None, max_steps: int = 400_000, tol: float = 1e-9, core_p: float = 0.02,
             chunk: int = 2048):
    """Solve every domain to steady state with the batched solver (in
    batches of at most `chunk` domains: a batch's Q x nodes must stay below
    2^32) and keep masks, network inputs and normalised targets on the
    device."""
    torch = _torch()
    h, w = shape
    ds = Dataset(h, w)
    masks = []
    for seed, phi, tau in domains:
        m, _ = lbm.lbm_qsgs(seed, shape, core_p, phi, stream=stream)
        masks.append(m)
        ds.taus.append(tau)
        ds.drhos.append(min(1e-3, 1e-4 * (tau - 0.5) / 3.0 * (w - 1)))
    ds.masks_host = masks
    n = len(masks)
    t0 = time.perf_counter()
    ds.targets = torch.empty((n, h, w, N_TARGET), dtype=torch.float32, device="cuda")
    for c0 in range(0, n, chunk):
        c1 = min(n, c0 + chunk)
        s = lbm.lbm_batch_create(masks[c0:c1], ds.taus[c0:c1], ds.drhos[c0:c1], lbm.make_options(stream=stream))
        _, st, steps, _ = lbm.lbm_run_to_steady(s, tol, max_steps)
        ds.steps += [int(v) for v in steps]
        for d in range(c1 - c0):
            lbm.lbm_nn_targets(s, d, ds.targets[c0 + d])
        torch.cuda.synchronize()
        s.close()
    ds.seconds = time.perf_counter() - t0
    ds.solid = torch.from_numpy(np.stack(masks)).to("cuda")
    ds.inputs = torch.empty((n, h, w, C_IN), dtype=torch.bfloat16, device="cuda")
    for d in range(n):
        lbm.lbm_nn_make_input(ds.solid[d], h, w, ds.taus[d] - 0.5, ds.inputs[d], stream)
    torch.cuda.synchronize()
    return ds


# Loss weights of (density deviation, u_x, u_y).  The density deviation from
# the ramp is ~5x smaller than the normalised velocity but it is what sets the
# slow pressure-diffusion mode the iteration has to relax; the velocity
# relaxes to the local pressure gradient on the fast pore-viscous time scale.
LOSS_WEIGHTS = (25.0, 1.0, 1.0)


def train(net: UNet, ds: Dataset, epochs: int = 20, batch: int = 8, lr: float = 2e-3, seed: int = 0,
          log=None, weights=LOSS_WEIGHTS):
    """AdamW on the masked, channel-weighted MSE of the normalised fields;
    returns per-epoch mean losses."""
    torch = _torch()
    s = net.ctx.stream
    n = len(ds)
    nb = n // batch
    rng = np.random.default_rng(seed)
    grad = torch.empty((batch, ds.h, ds.w, C_OUT), dtype=torch.bfloat16, device="cuda")
    part = torch.empty(256, dtype=torch.float32, device="cuda")
    lossd = torch.empty(1, dtype=torch.float32, device="cuda")
    hist = []
    total_steps = epochs * nb
    nfluid = [int((m == 0).sum()) for m in ds.masks_host]
    for ep in range(epochs):
        order = rng.permutation(nb)
        acc = 0.0
        for bi in order:
            i0 = int(bi) * batch
            x = ds.inputs[i0:i0 + batch]
            y = net.forward(x, batch, ds.h, ds.w)
            nfl = sum(nfluid[i0:i0 + batch])
            lbm.lbm_nn_mse(y, C_OUT, ds.targets[i0:i0 + batch], ds.solid[i0:i0 + batch],
                           batch * ds.h * ds.w, N_TARGET, 1.0 / (N_TARGET * nfl), grad, part, lossd, s,
                           weights=weights)
            net.backward(grad, batch)
            # cosine learning-rate decay
            frac = net.t / max(total_steps, 1)
            net.step(lr * 0.5 * (1 + math.cos(math.pi * frac)))
            acc += float(lossd.item())
        hist.append(acc / max(nb, 1))
        if log:
            log(f"epoch {ep}: loss {hist[-1]:.4e}")
    return hist


def predict(net: UNet, ds: Dataset, i0: int, n: int):
    return net.forward(ds.inputs[i0:i0 + n], n, ds.h, ds.w)


def time_to_k(t, k, tol, k_ref=None):
    """(time, index) of the first check interval after which k(t) stays within
    tol (relative) of k_ref for every later interval; k_ref is the oracle's
    converged k where one is known, else the run's own last k.  (None, None)
    when the history is empty or its last k is not within tol of k_ref."""
    k = np.asarray(k, np.float64)
    if len(k) == 0:
        return None, None
    kf = k[-1] if k_ref is None else float(k_ref)
    bad = np.where(~(np.abs(k - kf) <= tol * abs(kf)))[0]
    i = int(bad[-1]) + 1 if len(bad) else 0
    if i >= len(k):
        return None, None
    return float(t[i]), i


# Ablations of the warm start: the converged fields' channels put in place of
# the network's (0 = density deviation, 1, 2 = velocity), to see which part of
# the prediction limits the gain.
ABLATIONS = {"warm_true_density": (0,), "warm_true_velocity": (1, 2), "warm_true_fields": (0, 1, 2)}


def _with_true_channels(y, ds: Dataset, i0: int, nb: int, chans, stream=None):
    """Copy the stored targets' channels `chans` of domains i0 .. i0 + nb - 1
    into the prediction y (bf16 [nb, h, w, C_OUT]), with the library's kernels."""
    torch = _torch()
    tb = torch.empty((nb, ds.h, ds.w, N_TARGET), dtype=torch.bfloat16, device="cuda")
    lbm.lbm_nn_f32_to_bf16(ds.targets[i0:i0 + nb], tb, tb.numel(), stream)
    for c in chans:
        lbm.lbm_nn_copy_channels(tb, N_TARGET, c, y, C_OUT, c, 1, nb * ds.h * ds.w, stream)
    return y


def evaluate(net: UNet, ds: Dataset, stream=None, tol_k: float = 1e-4, max_steps: int = 400_000,
             tol: float = 1e-9, batch: int = 8, ablations: bool = False):
    """Equilibrium start vs warm start on the same domains (one batched solver
    each); returns per-domain steps and times to k within tol_k of each run's
    converged k, and the converged k of both.  With ablations, also warm
    starts whose density, velocity or both come from the converged solution
    (the targets) instead of the network."""
    torch = _torch()
    n = len(ds)
    res = {}
    modes = ["equilibrium", "warm"] + (list(ABLATIONS) if ablations else [])
    for mode in modes:
        s = lbm.lbm_batch_create(ds.masks_host, ds.taus, ds.drhos, lbm.make_options(stream=stream))
        t0 = time.perf_counter()
        if mode != "equilibrium":
            for i0 in range(0, n, batch):
                nb = min(batch, n - i0)
                y = predict(net, ds, i0, nb)
                if mode in ABLATIONS:
                    y = _with_true_channels(y, ds, i0, nb, ABLATIONS[mode], stream)
                for d in range(nb):
                    lbm.lbm_warm_start(s, i0 + d, y[d], C_OUT)
            torch.cuda.synchronize()
        t_pred = time.perf_counter() - t0
        _, st, steps, _ = lbm.lbm_run_to_steady(s, tol, max_steps)
        t_run = time.perf_counter() - t0
        k, _ = lbm.lbm_permeability(s)
        per = []
        for d in range(n):
            stp, kk, rr, tt = lbm.lbm_get_history(s, d)
            tk, ik = time_to_k(tt + t_pred, kk, tol_k)
            per.append({"steps_to_k": int(stp[ik]) if ik is not None else None, "time_to_k": tk,
                        "steps_total": int(steps[d]), "status": int(st[d])})
        s.close()
        res[mode] = {"k": [float(v) for v in k], "per_domain": per, "wall_s": t_run, "predict_s": t_pred}
    eq, wm = res["equilibrium"], res["warm"]
    # compare on the domains that converged in both runs (a domain with almost
    # no through-path can need more than max_steps from any start)
    both = [d for d in range(n) if eq["per_domain"][d]["status"] == 0 and wm["per_domain"][d]["status"] == 0]
    res["domains_converged_both"] = len(both)
    res["domains_not_converged"] = n - len(both)
    keq = np.array([eq["k"][d] for d in both])
    kwm = np.array([wm["k"][d] for d in both])
    res["k_rel_diff_max"] = float(np.max(np.abs(kwm - keq) / np.abs(keq))) if both else None
    res["k_rel_diff"] = [float(v) for v in (kwm - keq) / np.abs(keq)] if both else []
    res["steps_to_k_equilibrium"] = int(np.sum([eq["per_domain"][d]["steps_to_k"] for d in both]))
    res["steps_to_k_warm"] = int(np.sum([wm["per_domain"][d]["steps_to_k"] for d in both]))
    res["time_to_all_k_equilibrium_s"] = max([eq["per_domain"][d]["time_to_k"] for d in both], default=None)
    res["time_to_all_k_warm_s"] = max([wm["per_domain"][d]["time_to_k"] for d in both], default=None)
    for mode in ABLATIONS:
        if mode in res:
            ok = [d for d in both if res[mode]["per_domain"][d]["steps_to_k"] is not None]
            res["steps_to_k_" + mode] = int(np.sum([res[mode]["per_domain"][d]["steps_to_k"] for d in ok]))
            res["steps_to_k_equilibrium_on_" + mode] = int(np.sum([eq["per_domain"][d]["steps_to_k"] for d in ok]))
            res["domains_" + mode] = len(ok)
    return res
