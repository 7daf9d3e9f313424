#!/usr/bin/env python3
"""Throughput benchmark of the fused D2Q9/D3Q19 stream-collide hot path.

One benchmark step is one convergence-check interval of the steady-state
iteration over the whole workload: N-1 fused stream + boundary + collide
steps, one more that also reduces the FP64 observables, the per-domain
reduction, and the host readback that the steady-state control needs.  The
default workload is the batch of 128 independent uneven D2Q9 domains (N_x
uniform in [200, 1200], N_y = N_x/2, porosity U[0.6, 0.8], tau U[0.51, 1.5]; 23
M fluid nodes, 1.7 GB of populations per step, 13x the L2), the largest 2D
configuration of the paper's sweeps run as one batch.  The metric is MLUPS
counted over fluid nodes (million fluid-node lattice updates per second),
whole job over all ranks.  The same line carries the per-kernel rooflines of
four 256x128x128 D3Q19 domains (`roofline_d3q19`) and the time to
permeability of the 400x200 tau sweep, batched against one domain at a time,
measured against the FP64 oracle's converged k where one is stored.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_1609_09685_gb300 import workloads  # noqa: E402

METRIC = "MLUPS"
UNIT = "MLUPS (fluid-node lattice updates/s)"
FALLBACK_HBM_GBS = 6800.0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=30)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["native", "reference"], default="native")
    p.add_argument("--workload", choices=["sweep", "batch128", "d3q19", "d3q19_one", "small"], default="batch128")
    p.add_argument("--no-d3q19", action="store_true",
                   help="skip the per-kernel rooflines of the D3Q19 256x128x128 workload")
    p.add_argument("--no-ttp", action="store_true", help="skip the time-to-permeability measurement")
    p.add_argument("--interval", type=int, default=100)
    p.add_argument("--kn-sweep", action="store_true",
                   help="also solve the 24 tau-sweep domains to steady state (BGK and TRT) and report k/k_int vs Kn")
    p.add_argument("--forced3d", action="store_true",
                   help="also run the paper's force-driven periodic 3D experiment (100^3, phi 0.748587)")
    p.add_argument("--local-kn", action="store_true",
                   help="also time the local pore-size / local-Kn pass over every domain")
    p.add_argument("--conv-bench", action="store_true",
                   help="only time the warm-start network's convolution shapes on both tensor-core paths "
                        "(mma.sync and tcgen05) and print that line")
    p.add_argument("--conv-reps", type=int, default=20)
    p.add_argument("--no-autotune", action="store_true",
                   help="keep the default launch configuration instead of running the library's autotuner")
    p.add_argument("--tile-rows", type=int, default=0,
                   help="gather step: rows per staged tile (1..4), -1 = direct loads, 0 = library default")
    p.add_argument("--band-rows", type=int, default=0,
                   help="band gather step rows per band (D2Q9; 0 = the library's default, -1 = not used)")
    p.add_argument("--pair-block-mb", type=int, default=0,
                   help="L2-blocked pairs, MB of populations per block (0 = the library's default, -1 = whole batch)")
    p.add_argument("--collision", choices=["bgk", "trt"], default="bgk",
                   help="BGK (the paper's model) or TRT with Lambda = 3/16")
    p.add_argument("--e2e-steps", type=int, default=3)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    p.add_argument("--ttp-sizes", default="400x200",
                   help="resolutions of the tau sweep used for --ttp, e.g. 400x200,800x400")
    p.add_argument("--ttp-tol", type=float, default=1e-4)
    p.add_argument("--warmstart", action="store_true",
                   help="also train the U-Net warm start and compare time-to-permeability on held-out domains")
    p.add_argument("--ws-train", type=int, default=256, help="training solutions (512x256 domains)")
    p.add_argument("--ws-eval", type=int, default=16, help="held-out evaluation domains")
    p.add_argument("--ws-epochs", type=int, default=30)
    p.add_argument("--ws-shape", default="256x512", help="ny x nx of the warm-start domains")
    p.add_argument("--ws-weights", default="",
                   help="extra loss weights (density, u_x, u_y) to train and evaluate as well, ';'-separated")
    p.add_argument("--ws-ablations", action="store_true",
                   help="also warm-start from the converged density, velocity or both (diagnosis)")
    p.add_argument("--ws-plain", type=int, default=32, help="held-out domains also solved one at a time")
    return p.parse_args()


def get_workload(name: str, rank: int) -> workloads.Workload:
    if name == "sweep":
        return workloads.tau_sweep(seed=1 + rank)
    if name == "batch128":
        return workloads.batch128(master_seed=2026 + rank)
    if name == "d3q19":
        return workloads.d3q19_256(seed=1 + rank)
    if name == "d3q19_one":
        return workloads.d3q19_256(taus=(0.6,), seed=1 + rank)
    return workloads.small_2d(seed=1 + rank)


def lattice_q(wl):
    return 19 if wl.domains[0].nz > 1 else 9


def combine_ranks(dist, device, maxima, sums):
    """Whole-job figures of a weak-scaling run: each rank solves its own
    independent domains (no data-path collective); timing takes the slowest
    rank (MAX) and work adds up over ranks (SUM).  Returns (maxima, sums)."""
    if dist is None:
        return list(maxima), list(sums)
    import torch
    a = torch.tensor(list(maxima), dtype=torch.float64, device=device)
    b = torch.tensor(list(sums), dtype=torch.float64, device=device)
    dist.all_reduce(a, op=dist.ReduceOp.MAX)
    dist.all_reduce(b, op=dist.ReduceOp.SUM)
    return a.tolist(), b.tolist()


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            parts = [x.strip() for x in l.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
                power.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def measured_hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            v = float(json.load(fh)["hbm_gbs"])
            return v, "measured (MEASURED_PEAKS.json hbm_gbs, STREAM-style copy)"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback 6.8 TB/s (no MEASURED_PEAKS.json)"


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("lbm_kernels.cu", "aa_kernels.cu", "lbm_stencil.cuh", "lbm_device.cuh"):
        with open(os.path.join(ROOT, "paper_1609_09685_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(workload: str, q: int, kind: str):
    """DRAM bytes per launch of one kernel kind from the committed ncu summary,
    if it was taken on the current kernel source."""
    p = os.path.join(ROOT, "profiles", "stream_collide_traffic.json")
    try:
        with open(p) as fh:
            d = json.load(fh)
        e = d[f"{workload}_q{q}_{kind}"]
        if e.get("kernel_hash") != kernel_source_hash():
            return None
        return float(e["dram_bytes_per_launch"])
    except Exception:
        return None


# ---------------------------------------------------------------------------
# CPU oracle baseline (a bounded sample of the same workload)
# ---------------------------------------------------------------------------
def oracle_sample(wl, seconds: float):
    import oracle as O
    dom = min(wl.domains, key=lambda d: (d.cells, abs(d.tau - 0.6)))
    mask, _ = O.qsgs(dom.shape, dom.seed, dom.core_p, dom.porosity, dom.d_face)
    f = O.init(mask, 1 + dom.drho, 1.0)
    fluid = int((mask == 0).sum())
    t0 = time.perf_counter()
    f = O.run(mask, f, dom.tau, 1 + dom.drho, 1.0, 2)
    t_probe = (time.perf_counter() - t0) / 2
    nsteps = max(2, int(seconds / max(t_probe, 1e-6)))
    t0 = time.perf_counter()
    O.run(mask, f, dom.tau, 1 + dom.drho, 1.0, nsteps)
    dt = time.perf_counter() - t0
    return {"value": fluid * nsteps / dt / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"FP64 oracle, {nsteps} steps of the {dom.nx}x{dom.ny} domain "
                      f"(tau={dom.tau:.2f}, {fluid} fluid nodes) of the workload, {dt:.1f} s, "
                      f"single thread"}


# ---------------------------------------------------------------------------
# time-to-permeability
# ---------------------------------------------------------------------------
GOLDEN_K = os.path.join(ROOT, "tests", "golden", "converged_k.txt")


ORACLE_RESIDUAL_MAX = 1e-13


def oracle_k_table():
    """Converged FP64 oracle permeabilities stored by
    tests/golden/make_converged_k.py: {(nx, ny, nz, seed, tau): (k, bound)}."""
    out = {}
    if not os.path.exists(GOLDEN_K):
        return out
    with open(GOLDEN_K) as fh:
        for line in fh:
            if not line.strip() or line.startswith("#"):
                continue
            t = line.split()
            key = (int(t[1]), int(t[2]), int(t[3]), int(t[4]), round(float(t[6]), 12))
            out[key] = (float(t[8]), float(t[9]))
    return out


def measure_ttp(args, lbm, sp):
    from paper_1609_09685_gb300.warmstart import time_to_k
    sizes = []
    for tok in args.ttp_sizes.split(","):
        nx, ny = (int(v) for v in tok.lower().split("x"))
        phi = {400: 0.7394, 800: 0.7532, 1200: 0.7578}.get(nx, 0.75)
        sizes.append((nx, ny, phi))
    wl = workloads.tau_sweep(sizes=sizes)
    cache, masks = {}, []
    for d in wl.domains:
        key = (d.shape, d.seed, d.porosity)
        if key not in cache:
            cache[key], _ = lbm.lbm_qsgs(d.seed, d.shape, d.core_p, d.porosity, d.d_face, stream=sp)
        masks.append(cache[key])
    taus = [d.tau for d in wl.domains]
    drhos = [d.drho for d in wl.domains]
    table = oracle_k_table()
    # the oracle's k where its stored state is the fixed point to the FP64
    # step's rounding level (residual <= 1e-13, as in the converged-k tests)
    k_ref = []
    for d in wl.domains:
        k, r = table.get((d.nx, d.ny, d.nz, d.seed, round(d.tau, 12)), (None, None))
        k_ref.append(k if (k is not None and r <= ORACLE_RESIDUAL_MAX) else None)
    n_ref = sum(v is not None for v in k_ref)
    have_ref = n_ref == len(k_ref)
    opts = lbm.make_options(stream=sp)
    out = {"workload": wl.name, "sizes": args.ttp_sizes, "domains": len(wl.domains), "tol_rel": args.ttp_tol,
           "residual_tol": wl.tol,
           "k_reference": (f"FP64 oracle's converged k (tests/golden/converged_k.txt, residual <= "
                           f"{ORACLE_RESIDUAL_MAX:g}) for {n_ref} of {len(k_ref)} domains"
                           + ("" if have_ref else ", each run's own converged k for the others"))}
    ref = k_ref
    # batched: all domains in one solver, converged ones retire
    s = lbm.lbm_batch_create(masks, taus, drhos, opts)
    t0 = time.perf_counter()
    rc, st, steps, res = lbm.lbm_run_to_steady(s, wl.tol, wl.max_steps)
    t_batch = time.perf_counter() - t0
    kb, _ = lbm.lbm_permeability(s)
    ttp_b = []
    for d in range(len(masks)):
        _, kk, _, tt = lbm.lbm_get_history(s, d)
        ttp_b.append(time_to_k(tt, kk, args.ttp_tol, ref[d])[0])
    s.close()
    # plain: one domain at a time
    ttp_p, t_plain, kp = [], 0.0, []
    for d in range(len(masks)):
        s1 = lbm.lbm_create_domain(masks[d], taus[d], drhos[d], opts)
        t0 = time.perf_counter()
        lbm.lbm_run_to_steady(s1, wl.tol, wl.max_steps)
        t_plain += time.perf_counter() - t0
        _, kk, _, tt = lbm.lbm_get_history(s1, 0)
        ttp_p.append(time_to_k(tt, kk, args.ttp_tol, ref[d])[0])
        kp.append(float(lbm.lbm_permeability(s1)[0][0]))
        s1.close()
    reached = all(v is not None for v in ttp_b + ttp_p)
    out.update({
        "all_reached_tol": reached,
        "batched_time_to_k_s": max(ttp_b) if reached else None,
        "plain_time_to_k_s": float(sum(ttp_p)) if reached else None,
        "batched_stop_s": t_batch, "plain_stop_s": t_plain,
        "speedup_time_to_k": float(sum(ttp_p)) / max(ttp_b) if reached else None,
        "max_rel_k_diff_batched_vs_plain": float(np.max(np.abs(np.array(kb) - np.array(kp)) / np.abs(kp))),
        "max_rel_k_diff_vs_oracle": (max(abs(kb[d] - k_ref[d]) / abs(k_ref[d]) for d in range(len(masks))
                                         if k_ref[d] is not None) if n_ref else None),
        "per_domain": [{"tau": taus[d], "nx": wl.domains[d].nx, "steps": int(steps[d]),
                        "status": int(st[d]), "k": float(kb[d]), "k_oracle": k_ref[d],
                        "ttp_batched_s": ttp_b[d], "ttp_plain_s": ttp_p[d]} for d in range(len(masks))],
    })
    return out


def measure_warmstart(args, lbm, sp):
    """Time-to-permeability on held-out domains: plain (one domain at a time,
    equilibrium start), batched (equilibrium start), batched + learned warm start."""
    from paper_1609_09685_gb300 import warmstart as WS
    ny, nx = (int(v) for v in args.ws_shape.lower().split("x"))
    shape = (ny, nx)
    t0 = time.perf_counter()
    ds = WS.generate(WS.make_domains(args.ws_train, shape, seed0=0, master_seed=11), shape)
    t_gen = time.perf_counter() - t0
    ev = WS.generate(WS.make_domains(args.ws_eval, shape, seed0=1_000_000, master_seed=12), shape)
    levels = 8 if min(ny, nx) % 128 == 0 else 4
    chans = (16, 32, 32, 64, 64, 128, 128, 128)[:levels]
    net = WS.UNet(chans, seed=0)
    t0 = time.perf_counter()
    hist = WS.train(net, ds, epochs=args.ws_epochs, batch=8, lr=2e-3)
    t_train = time.perf_counter() - t0
    res = WS.evaluate(net, ev, ablations=args.ws_ablations)
    # plain: one domain at a time from the equilibrium start, on (a sample of
    # at most --ws-plain of) the domains that converged in both batched runs
    eq, wm = res["equilibrium"], res["warm"]
    both = [d for d in range(len(ev)) if eq["per_domain"][d]["status"] == 0 and wm["per_domain"][d]["status"] == 0]
    plain_t, plain_steps = [], []
    for d in both[:args.ws_plain]:
        s1 = lbm.lbm_create_domain(ev.masks_host[d], ev.taus[d], ev.drhos[d], lbm.make_options())
        lbm.lbm_run_to_steady(s1, 1e-9, 400_000)
        stp, kk, rr, tt = lbm.lbm_get_history(s1, 0)
        s1.close()
        tk, ik = WS.time_to_k(tt, kk, args.ttp_tol)
        if tk is None:
            continue
        plain_t.append(tk)
        plain_steps.append(int(stp[ik]))
    extra = []
    for wspec in [w for w in args.ws_weights.split(";") if w.strip()]:
        wts = tuple(float(v) for v in wspec.split(","))
        net2 = WS.UNet(chans, seed=0)
        t0 = time.perf_counter()
        h2 = WS.train(net2, ds, epochs=args.ws_epochs, batch=8, lr=2e-3, weights=wts)
        t2 = time.perf_counter() - t0
        r2 = WS.evaluate(net2, ev)
        extra.append({"loss_weights": list(wts), "train_s": t2, "loss_first_last": [h2[0], h2[-1]],
                      "domains_compared": r2["domains_converged_both"],
                      "batched_steps_to_k": r2["steps_to_k_equilibrium"],
                      "batched_warm_steps_to_k": r2["steps_to_k_warm"],
                      "batched_time_to_k_s": r2["time_to_all_k_equilibrium_s"],
                      "batched_warm_time_to_k_s": r2["time_to_all_k_warm_s"]})
    return {
        "shape": [ny, nx], "domains_compared": len(both), "loss_weights": list(WS.LOSS_WEIGHTS),
        "other_loss_weights": extra, "domains_not_converged": res["domains_not_converged"], "train_solutions": len(ds), "eval_domains": len(ev), "unet_levels": levels,
        "unet_params": int(net.nparams), "epochs": args.ws_epochs, "loss_first_last": [hist[0], hist[-1]],
        "datagen_s": t_gen, "train_s": t_train, "tol_rel": args.ttp_tol,
        "plain_time_to_k_s": float(sum(plain_t)), "plain_steps_to_k": int(sum(plain_steps)),
        "batched_time_to_k_s": res["time_to_all_k_equilibrium_s"],
        "batched_warm_time_to_k_s": res["time_to_all_k_warm_s"],
        "batched_steps_to_k": res["steps_to_k_equilibrium"], "batched_warm_steps_to_k": res["steps_to_k_warm"],
        "warm_predict_s": wm["predict_s"], "k_rel_diff_warm_vs_equilibrium_max": res["k_rel_diff_max"],
        "k_rel_diff_warm_vs_equilibrium": res["k_rel_diff"],
        "plain_domains": min(len(both), args.ws_plain),
        "per_domain_steps_to_k": {"equilibrium": [eq["per_domain"][d]["steps_to_k"] for d in both],
                                  "warm": [wm["per_domain"][d]["steps_to_k"] for d in both]},
        "ablations": {k: v for k, v in res.items() if k.startswith(("steps_to_k_warm_true", "steps_to_k_equilibrium_on",
                                                                    "domains_warm_true"))},
    }


def measure_kn_sweep(lbm, sp):
    """Sec. 2's Figs. 2-3: k / k_int against Kn on the tau sweep at the three
    resolutions.  Two normalisers are reported: TRT's permeability with
    Lambda = 3/16, which does not depend on tau, and BGK's k extrapolated to
    tau -> 1/2 by a least-squares line in (tau - 1/2)^2 (the form of the exact
    channel solution)."""
    import torch
    wl = get_workload("sweep", 0)
    cache, masks = {}, []
    for d in wl.domains:
        key = (d.shape, d.seed, d.porosity)
        if key not in cache:
            cache[key], _ = lbm.lbm_qsgs(d.seed, d.shape, d.core_p, d.porosity, d.d_face, stream=sp)
        masks.append(cache[key])
    taus = [d.tau for d in wl.domains]
    drhos = [d.drho for d in wl.domains]
    out = {"workload": wl.name, "tol": 1e-9}
    for name, coll in (("bgk", lbm.LBM_COLL_BGK), ("trt", lbm.LBM_COLL_TRT)):
        s = lbm.lbm_batch_create(masks, taus, drhos, lbm.make_options(stream=sp, collision=coll))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, st, steps, _ = lbm.lbm_run_to_steady(s, 1e-9, 3_000_000)
        torch.cuda.synchronize()
        k, kn = lbm.lbm_permeability(s)
        out[name] = {"seconds": time.perf_counter() - t0, "k": [float(v) for v in k], "kn": [float(v) for v in kn],
                     "status": [int(v) for v in st], "steps": [int(v) for v in steps]}
        s.close()
    res = {}
    for nx in sorted({d.nx for d in wl.domains}):
        idx = [i for i, d in enumerate(wl.domains) if d.nx == nx]
        t2 = np.array([(taus[i] - 0.5) ** 2 for i in idx])
        kb = np.array([out["bgk"]["k"][i] for i in idx])
        A = np.vstack([np.ones_like(t2), t2]).T
        use = t2 <= 0.25  # the small-Kn end, where the (tau - 1/2)^2 form holds best
        coef, *_ = np.linalg.lstsq(A[use], kb[use], rcond=None)
        k_int = float(coef[0])
        k_trt = float(np.mean([out["trt"]["k"][i] for i in idx]))
        res[f"{nx}x{nx // 2}"] = {
            "k_int_bgk_extrapolated": k_int,
            "k_trt_mean": k_trt,
            "k_over_k_trt_bgk": [float(v / k_trt) for v in kb],
            "k_trt_spread": float(np.ptp([out["trt"]["k"][i] for i in idx]) / np.mean([out["trt"]["k"][i] for i in idx])),
            "kn": [out["bgk"]["kn"][i] for i in idx],
            "k_over_k_int_bgk": [float(v / k_int) for v in kb],
        }
    out["per_resolution"] = res
    return out


def measure_forced3d(lbm, sp):
    """Sec. 2's 3D experiment: a 100^3 QSGS medium at porosity 0.748587, driven
    by three body accelerations with every face periodic; k = nu <u>/g (Eq. 2)
    with the quadratic and with the linear (Stokes) equilibrium."""
    import torch
    mask, _ = lbm.lbm_qsgs(1, (100, 100, 100), 0.02, 0.748587, stream=sp)
    tau, gs = 1.0, [1e-5, 1e-3, 1e-2]
    out = {"mask": "3D QSGS 100^3, seed 1, core 0.02, porosity 0.748587", "tau": tau, "g": gs}
    for name, eq in (("quadratic", lbm.LBM_EQ_QUADRATIC), ("linear", lbm.LBM_EQ_LINEAR)):
        s = lbm.lbm_batch_create_forced([mask] * 3, [tau] * 3, gs, lbm.make_options(stream=sp, equilibrium=eq))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, st, steps, _ = lbm.lbm_run_to_steady(s, 1e-9, 400_000)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        k, _ = lbm.lbm_permeability(s)
        out[name] = {"k": [float(v) for v in k], "k_over_k_smallest_g": [float(v / k[0]) for v in k],
                     "status": [int(v) for v in st], "steps": [int(v) for v in steps], "seconds": dt,
                     "mlups": float(sum(int(v) for v in steps) * int((mask == 0).sum()) / dt / 1e6)}
        if name == "quadratic":
            # per-kernel device time of the plain steps (forced gather and local
            # steps of the in-place pairs, one pull step), CUDA events per launch
            s2 = lbm.lbm_batch_create_forced([mask] * 3, [tau] * 3, gs, lbm.make_options(stream=sp, equilibrium=eq))
            lbm.lbm_step(s2, 100)
            prof = lbm.lbm_profile_steps(s2, 101)
            s2.close()
            fluid = 3 * int((mask == 0).sum())
            bpl = 2 * 4 * 19 * fluid
            peak, peak_src = measured_hbm_peak()
            kern = {}
            for kind in ("gather", "local", "pull"):
                t_us, n = prof[kind]
                if n:
                    us = t_us / n
                    kern[kind] = {"avg_launch_us": us, "launches": n, "achieved": bpl / us / 1e3,
                                  "frac": bpl / us / 1e3 / peak}
            out["kernels"] = {"domains": 3, "fluid_nodes": fluid, "bytes_per_launch": bpl,
                              "algorithmic_bytes": "152 B per fluid-node update (one step)", "peak": peak,
                              "peak_source": peak_src, "per_kind": kern}
        s.close()
    return out


# ---------------------------------------------------------------------------
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle as O
    wl = get_workload(args.workload, 0)
    dom = min(wl.domains, key=lambda d: (d.cells, abs(d.tau - 0.6)))
    mask, _ = O.qsgs(dom.shape, dom.seed, dom.core_p, dom.porosity, dom.d_face)
    fluid = int((mask == 0).sum())
    f = O.init(mask, 1 + dom.drho, 1.0)
    per_step = 4  # oracle time steps per benchmark step (bounded sample)
    for _ in range(args.warmup):
        f = O.run(mask, f, dom.tau, 1 + dom.drho, 1.0, per_step)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        f = O.run(mask, f, dom.tau, 1 + dom.drho, 1.0, per_step)
    dt = time.perf_counter() - t0
    v = fluid * per_step * args.steps / dt / 1e6
    sample = (f"each step = {per_step} FP64 oracle time steps of the {dom.nx}x{dom.ny} domain "
              f"(tau={dom.tau:.2f}) of workload {wl.name}")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": wl.name, "sample": sample},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


KERNEL_NAMES = {"gather": "k_aa_gather (gather step of the in-place pair)",
                "local": "k_aa_local (local step of the in-place pair)",
                "pull": "k_stream_collide (pull step)"}


def masks_of(lbm, wl, sp):
    cache, masks = {}, []
    for d in wl.domains:
        key = (d.shape, d.seed, d.porosity)
        if key not in cache:
            cache[key], _ = lbm.lbm_qsgs(d.seed, d.shape, d.core_p, d.porosity, d.d_face, stream=sp)
        masks.append(cache[key])
    return masks


def time_intervals(lbm, s, stream, N, steps, warmup, barrier, sampler=None):
    """W warm-up intervals, then K timed intervals (graph-launched), then the
    same K intervals once more with every plain-step kernel bracketed by CUDA
    events (lbm_profile_steps).  Returns (seconds of the timed region, seconds
    per graph-launched plain step, seconds of the per-kernel pass,
    {kind: [us, launches]}, clocks)."""
    import torch
    clocks = None
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            lbm.lbm_step(s, N - 1)
            lbm.lbm_step_observe(s, 1)
        barrier()
        if sampler is not None:
            sampler.start()
            time.sleep(0.4)
        ka = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        kb = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for k in range(steps):
            ka[k].record(stream)
            lbm.lbm_step(s, N - 1)
            kb[k].record(stream)
            lbm.lbm_step_observe(s, 1)
        e1.record(stream)
        barrier()
        if sampler is not None:
            clocks = sampler.stop()
    t = e0.elapsed_time(e1) / 1e3
    t_kern = sum(a.elapsed_time(b) for a, b in zip(ka, kb)) / 1e3 / (steps * (N - 1))
    with torch.cuda.stream(stream):
        barrier()
        kt = {k: [0.0, 0] for k in lbm.KERNEL_KINDS}
        p0 = torch.cuda.Event(enable_timing=True)
        p1 = torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        for k in range(steps):
            prof = lbm.lbm_profile_steps(s, N - 1)
            for kind, (us, cnt) in prof.items():
                kt[kind][0] += us
                kt[kind][1] += cnt
            lbm.lbm_step_observe(s, 1)
        p1.record(stream)
        barrier()
    t_prof = p0.elapsed_time(p1) / 1e3
    return t, t_kern, t_prof, kt, clocks


def kernel_table(kt, steps, bytes_per_launch, peak, workload, q):
    """Per-kernel rooflines: algorithmic bytes per launch over the average
    event-timed launch duration, and each kernel's share of plain-step time."""
    kernels = {}
    for kind in [k for k in kt if kt[k][1] > 0]:
        us = kt[kind][0] / kt[kind][1]
        a = bytes_per_launch / (us * 1e-6) / 1e9
        kernels[kind] = {"kernel": KERNEL_NAMES.get(kind, kind), "launches_per_interval": kt[kind][1] // steps,
                         "avg_launch_us": us, "achieved": a, "frac": a / peak,
                         "traffic": profiled_traffic(workload, q, kind)}
    total_us = sum(v["avg_launch_us"] * v["launches_per_interval"] for v in kernels.values())
    for v in kernels.values():
        v["share_of_plain_steps"] = v["avg_launch_us"] * v["launches_per_interval"] / total_us
    return kernels


def roofline_of(lbm, wl_name, sp, stream, N, steps, warmup, coll, barrier, peak, peak_src, tile_rows=0,
                autotune=True):
    """Per-kernel rooflines of a second workload, timed like the headline one
    (used for the D3Q19 256x128x128 configuration)."""
    wl = get_workload(wl_name, 0)
    q = lattice_q(wl)
    masks = masks_of(lbm, wl, sp)
    opts = lbm.make_options(stream=sp, check_interval=N, collision=coll, tile_rows=tile_rows)
    s = lbm.lbm_batch_create(masks, [d.tau for d in wl.domains], [d.drho for d in wl.domains], opts)
    fluid = s.fluid_nodes
    bpl = 2 * 4 * q * fluid
    tune = lbm.lbm_autotune(s) if autotune else None
    t, t_kern, _, kt, _ = time_intervals(lbm, s, stream, N, steps, warmup, barrier)
    s.close()
    kernels = kernel_table(kt, steps, bpl, peak, wl_name, q)
    dom_kind = max(kernels, key=lambda k: kernels[k]["share_of_plain_steps"])
    dk = kernels[dom_kind]
    ach = bpl / t_kern / 1e9
    return {"workload": wl.name, "domains": len(wl.domains), "lattice": "D3Q19" if q == 19 else "D2Q9",
            "fluid_nodes": fluid, "nodes": wl.cells, "mlups": steps * N * fluid / t / 1e6,
            "bound": "hbm", "achieved": dk["achieved"], "peak": peak, "unit": "GB/s", "frac": dk["frac"],
            "traffic": dk["traffic"], "kernel": dk["kernel"], "bytes_per_launch": bpl,
            "algorithmic_bytes": f"{2 * 4 * q} B per fluid-node update (one step)",
            "avg_launch_us": dk["avg_launch_us"], "peak_source": peak_src, "kernels": kernels,
            "plain_step_average": {"avg_step_us": t_kern * 1e6, "achieved": ach, "frac": ach / peak,
                                   "timing": "CUDA events around the graph-launched plain steps"},
            "autotune": tune}


def run_conv_bench(args):
    """The 3x3 convolutions of the 8-level warm-start U-Net (batch 8, 256x512
    input, channels 16, 32, 32, 64, 64, 128, 128, 128) on the mma.sync and
    tcgen05 paths: CUDA-event time per launch and TFLOP/s (2 x 9 x Cin x Cout
    per output pixel)."""
    import torch

    from paper_1609_09685_gb300 import build as B
    from paper_1609_09685_gb300 import lbm
    B.build()
    lbm.load()
    batch, chans = 8, (16, 32, 32, 64, 64, 128, 128, 128)
    rows = []
    old = lbm.lbm_nn_get_conv_impl()
    try:
        for lvl, c in enumerate(chans):
            h, w = 256 >> lvl, 512 >> lvl
            for cin in ((chans[lvl - 1] if lvl else 16), c):
                x = torch.randn(batch, h, w, cin, device="cuda").to(torch.bfloat16)
                wt = (torch.randn(9, c, cin, device="cuda") * 0.1).to(torch.bfloat16)
                b = torch.zeros(c, device="cuda")
                y = torch.empty(batch, h, w, c, device="cuda", dtype=torch.bfloat16)
                row = {"n": batch, "h": h, "w": w, "cin": cin, "cout": c}
                for name, impl in (("mma_sync", lbm.LBM_NN_CONV_MMA_SYNC), ("tcgen05", lbm.LBM_NN_CONV_TCGEN05)):
                    lbm.lbm_nn_set_conv_impl(impl)
                    for _ in range(3):
                        lbm.lbm_nn_conv_fwd(x, batch, h, w, cin, wt, b, 9, c, 1, y)
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record()
                    for _ in range(args.conv_reps):
                        lbm.lbm_nn_conv_fwd(x, batch, h, w, cin, wt, b, 9, c, 1, y)
                    e1.record()
                    torch.cuda.synchronize()
                    us = e0.elapsed_time(e1) * 1e3 / args.conv_reps
                    row[name] = {"us": us, "tflops": 2.0 * 9 * cin * c * batch * h * w / us / 1e6}
                lbm.lbm_nn_sync_status()
                rows.append(row)
    finally:
        lbm.lbm_nn_set_conv_impl(old)
    tot = {k: sum(r[k]["us"] for r in rows) for k in ("mma_sync", "tcgen05")}
    print(json.dumps({"metric": "warm-start U-Net 3x3 convolutions, us per forward pass (batch 8)",
                      "value": tot, "unit": "us", "layers": rows}), flush=True)
    return 0


def run_native(args):
    import torch

    from paper_1609_09685_gb300 import build as B
    from paper_1609_09685_gb300 import lbm

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    B.build()
    lbm.load()

    wl = get_workload(args.workload, rank)
    q = lattice_q(wl)
    N = args.interval
    stream = torch.cuda.Stream()
    sp = stream.cuda_stream
    masks = masks_of(lbm, wl, sp)
    taus = [d.tau for d in wl.domains]
    drhos = [d.drho for d in wl.domains]
    coll = lbm.LBM_COLL_TRT if args.collision == "trt" else lbm.LBM_COLL_BGK
    opts = lbm.make_options(stream=sp, check_interval=N, collision=coll, tile_rows=args.tile_rows,
                            band_rows=args.band_rows, pair_block_mb=args.pair_block_mb)
    s = lbm.lbm_batch_create(masks, taus, drhos, opts)
    fluid = s.fluid_nodes
    bytes_per_launch = 2 * 4 * q * fluid
    tune = None
    if not args.no_autotune and args.tile_rows == 0 and args.band_rows == 0 and args.pair_block_mb == 0:
        tune = lbm.lbm_autotune(s)  # CUDA-event timing of every candidate on this solver's stream
    lbm_launch_of_run = lbm.lbm_get_launch(s)  # the configuration the timed region runs

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    t, t_kern, t_prof, kt, clocks = time_intervals(lbm, s, stream, N, args.steps, args.warmup, barrier,
                                                    sampler=ClockSampler(local))
    kinds = [k for k in lbm.KERNEL_KINDS if kt[k][1] > 0]
    avg_us = [kt[k][0] / kt[k][1] for k in kinds]
    (t, t_kern, t_prof, *avg_us), (updates,) = combine_ranks(
        dist, "cuda", [t, t_kern, t_prof] + avg_us, [float(args.steps * N * fluid)])
    for k, us in zip(kinds, avg_us):  # the slowest rank's kernel times
        kt[k][0] = us * kt[k][1]
    value = updates / t / 1e6

    # end to end through the C ABI: host masks (pinned) -> create -> one interval
    # -> permeability back on the host, per step
    pinned = []
    for m in masks:
        pm = torch.empty(m.shape, dtype=torch.uint8, pin_memory=True).numpy()
        pm[...] = m
        pinned.append(pm)
    h2d = sum(m.nbytes for m in pinned) + 48 * len(pinned) + 4 * (len(pinned) + 1)
    nseg = sum(((d.nx + 31) // 32) * d.ny * d.nz for d in wl.domains)
    d2h = 4 * nseg + 4 + 8 * lbm.NUM_OBS * len(pinned)
    if tune is not None:  # the end-to-end solvers take the tuned configuration through their options
        c = tune["chosen"]
        opts = lbm.make_options(stream=sp, check_interval=N, collision=coll, block_threads=c["block_threads"],
                                strip_rows=c["strip_rows"], gather_batch=c["gather_batch"],
                                tile_rows=c["tile_rows"], band_rows=c["band_rows"] if c["band_rows"] else -1,
                                pair_block_mb=c["pair_block_mb"] if c["pair_block_mb"] else -1)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        s2 = lbm.lbm_batch_create(pinned, taus, drhos, opts)
        lbm.lbm_step(s2, N - 1)
        lbm.lbm_step_observe(s2, 1)
        k, kn = lbm.lbm_permeability(s2)
        s2.close()
    torch.cuda.synchronize()
    t_e2e = time.perf_counter() - t0
    (t_e2e,), (e2e_updates,) = combine_ranks(dist, "cuda", [t_e2e], [float(args.e2e_steps * N * fluid)])
    lkn = None
    if args.local_kn and rank == 0:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        kmax, kmean = [], []
        for d in range(len(wl.domains)):
            _, hh, kn = lbm.lbm_local_knudsen(s, d)
            fl = kn > 0
            kmax.append(float(kn[fl].max()) if fl.any() else 0.0)
            kmean.append(float(kn[fl].mean()) if fl.any() else 0.0)
        t_lkn = time.perf_counter() - t0
        lkn = {"seconds_all_domains": t_lkn, "nodes": wl.cells,
               "note": "lbm_local_knudsen per domain, host copies of d2, h and Kn included",
               "max_local_kn_over_domain_kn": max(
                   km / (np.sqrt(np.pi / 6) * (d.tau - 0.5) / d.nx) for km, d in zip(kmax, wl.domains))}
    s.close()
    peak, peak_src = measured_hbm_peak()
    roof3 = None
    if rank == 0 and not args.no_d3q19 and q == 9:
        roof3 = roofline_of(lbm, "d3q19", sp, stream, N, args.steps, args.warmup, coll, torch.cuda.synchronize,
                            peak, peak_src, args.tile_rows, not args.no_autotune)
    ttp = measure_ttp(args, lbm, sp) if (not args.no_ttp and rank == 0) else None
    f3d = measure_forced3d(lbm, sp) if (args.forced3d and rank == 0) else None
    kns = measure_kn_sweep(lbm, sp) if (args.kn_sweep and rank == 0) else None
    ws = measure_warmstart(args, lbm, sp) if (args.warmstart and rank == 0) else None

    if rank == 0:
        achieved_step = bytes_per_launch / t_kern / 1e9
        kernels = kernel_table(kt, args.steps, bytes_per_launch, peak, args.workload, q)
        dom_kind = max(kernels, key=lambda k: kernels[k]["share_of_plain_steps"])
        dk = kernels[dom_kind]
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            cpu = oracle_sample(wl, args.cpu_seconds)
        total_nodes = wl.cells
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded QSGS masks at the paper's sizes and porosities)",
            "config": {
                "workload": wl.name, "domains": len(wl.domains), "lattice": f"D2Q9" if q == 9 else "D3Q19",
                "collision": "TRT (Lambda = 3/16)" if args.collision == "trt" else "BGK",
                "gather_tile_rows": args.tile_rows,
                "gather_launch": lbm_launch_of_run,
                "nodes": total_nodes, "fluid_nodes": fluid, "check_interval": N,
                "step": f"{N - 1} fused stream-collide steps + 1 observing step + FP64 reduction + "
                        "host readback (one convergence-check interval)",
                "all_node_mlups": value * total_nodes / fluid,
                "l2": f"inputs larger than L2: {2 * 4 * q * fluid / 1e9:.2f} GB of populations per step",
                "parallelism": f"independent domains, one replica per GPU ({world})",
            },
            "roofline": {"bound": "hbm", "achieved": dk["achieved"], "peak": peak, "unit": "GB/s",
                         "frac": dk["frac"], "traffic": dk["traffic"],
                         "kernel": dk["kernel"], "bytes_per_launch": bytes_per_launch,
                         "algorithmic_bytes": f"{2 * 4 * q} B per fluid-node update (one step)",
                         "avg_launch_us": dk["avg_launch_us"], "peak_source": peak_src,
                         "timing": "CUDA events around every kernel on the solver's stream over the "
                                   f"{args.steps} intervals of the per-kernel pass (lbm_profile_steps)",
                         "kernels": kernels,
                         "plain_step_average": {"avg_step_us": t_kern * 1e6, "achieved": achieved_step,
                                                "frac": achieved_step / peak,
                                                "timing": "CUDA events around the graph-launched plain "
                                                          "steps of the timed region"}},
            "e2e": {"value": e2e_updates / t_e2e / 1e6, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h,
                    "step": "create from pinned host masks + one interval + permeability readback"},
            "autotune": tune,
            "gpu_launches": args.steps * (sum(kt[k][1] for k in kinds) // args.steps + 2),
            "ms_per_step_per_kernel_pass": t_prof / args.steps * 1e3,
            "clocks": clocks,
        }
        if roof3 is not None:
            line["roofline_d3q19"] = roof3
        if cpu is not None:
            line["cpu_baseline"] = cpu
        if ttp is not None:
            line["time_to_permeability"] = ttp
        if lkn is not None:
            line["local_knudsen"] = lkn
        if f3d is not None:
            line["forced_3d"] = f3d
        if kns is not None:
            line["kn_sweep"] = kns
        if ws is not None:
            line["warm_start"] = ws
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.conv_bench:
        return run_conv_bench(args)
    return run_native(args)


if __name__ == "__main__":
    sys.exit(main())
