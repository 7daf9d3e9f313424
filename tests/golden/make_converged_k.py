"""Write tests/golden/converged_k.txt and converged_u_samples.npz: the FP64
oracle's converged permeability (and velocities at sampled fluid nodes) on the
benchmark configurations.  Calls only oracle/ and the input recipes of
paper_1609_09685_gb300/workloads.py; nothing here comes from the CUDA path.

Each domain's steady state is the fixed point of the oracle's FP64 step
(oracle/steady.py: Newton-Krylov on S(f) - f, every evaluation one oracle
step), from the solver's own initial state (rest equilibrium with the linear
inlet-to-outlet density ramp).  The permeability is the oracle's Darcy law
with the link mass flow rate (Sec. 2, Eq. 1 viscosity).

Sets (names as in the tests):
  C1  100x50, tau 0.8, rho_in/rho_out = 1.0005/1, QSGS seeds 1-10
  C2  the Sec. 2 tau sweep: 400x200 / 800x400 / 1200x600 at porosities 0.7394 /
      0.7532 / 0.7578, tau - 1/2 in {0.01 ... 1.5}, Stokes pressure difference
  C3  16 of the 128 uneven domains (indices drawn with numpy's generator from
      seed 2026), master seed 2026
  C4  256x128x128 D3Q19, porosity 0.70, tau 0.52 and 0.6

    python tests/golden/make_converged_k.py [--sets C1,C2,C3] [--procs N] [--names A,B] [--maxiter M] [--inner I]
    python tests/golden/make_converged_k.py --merge-only

Runs one process per job (spawned), longest first.  Each result is saved as
it finishes (a line in converged_k.partial.txt and tests/golden/partial/
NAME.npz with the sampled velocities); when every job of the chosen sets is
done the final files are rewritten from what they already hold plus every
saved result, so separate runs (e.g. the 3D set alone) merge instead of
overwriting each other.  --merge-only does just that merge.  Runtime on 8
x86 cores: hours (the 1200x600 and D3Q19 domains dominate).
"""
from __future__ import annotations

import argparse
import multiprocessing as mp
import os
import sys
import time

# one BLAS thread per worker process: the pool already uses every core
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

OUT_K = os.path.join(HERE, "converged_k.txt")
OUT_U = os.path.join(HERE, "converged_u_samples.npz")
PARTIAL = os.path.join(HERE, "converged_k.partial.txt")
PARTS = os.path.join(HERE, "partial")
NSAMPLE = 256


def jobs(sets):
    from paper_1609_09685_gb300 import workloads as W
    out = []
    if "C1" in sets:
        for seed in range(1, 11):
            d = W.small_2d(seed).domains[0]
            out.append(("C1", f"C1_seed{seed}", d))
    if "C2" in sets:
        for d in W.tau_sweep().domains:
            out.append(("C2", f"C2_{d.nx}x{d.ny}_tau{d.tau:.2f}", d))
    if "C3" in sets:
        wl = W.batch128()
        pick = sorted(int(i) for i in np.random.default_rng(2026).choice(len(wl.domains), 16, replace=False))
        for i in pick:
            out.append(("C3", f"C3_domain{i:03d}", wl.domains[i]))
    if "C4" in sets:
        for d in W.d3q19_256(taus=(0.52, 0.6)).domains:
            out.append(("C4", f"C4_tau{d.tau:.2f}", d))
    return out


def cost(d):
    """Rough relative cost (cells x N_x x viscosity-scaled relaxation)."""
    return d.cells * d.nx * (0.2 + (d.tau - 0.5)) * (19.0 / 9.0 if d.nz > 1 else 1.0)


MAXITER = 400
INNER = 30


def solve(job):
    import oracle as O
    from oracle import steady
    set_name, name, d = job[:3]
    maxiter = job[3] if len(job) > 3 else MAXITER
    inner = job[4] if len(job) > 4 else INNER
    t0 = time.time()
    mask, _ = O.qsgs(d.shape, d.seed, d.core_p, d.porosity, d.d_face)
    perc = O.percolates(mask)
    f, info = steady.steady_state(mask, d.tau, 1.0 + d.drho, 1.0, maxiter=maxiter, inner_maxiter=inner)
    k = O.permeability(mask, f, d.tau, 1.0 + d.drho, 1.0)
    fields = O.fields(mask, f)
    fl = np.flatnonzero(mask.ravel() == 0)
    rng = np.random.default_rng(d.seed % (2 ** 32))
    idx = np.sort(rng.choice(fl, size=min(NSAMPLE, len(fl)), replace=False))
    u = np.stack([fields[1 + a].ravel()[idx] for a in range(3 if d.nz > 1 else 2)], axis=1)
    return {"set": set_name, "name": name, "nx": d.nx, "ny": d.ny, "nz": d.nz, "seed": d.seed, "porosity": d.porosity,
            "tau": d.tau, "drho": d.drho, "k": k, "residual": info["residual_max"], "evals": info["evaluations"],
            "converged": info["converged"], "percolates": perc, "seconds": time.time() - t0, "idx": idx, "u": u}


HEADER = """# FP64 oracle: converged Darcy permeability of the benchmark configurations
# (Sec. 2: lattice Boltzmann iterated to steady state, permeability from the
# mass flow rate by Darcy's law, nu = (tau - 1/2)/3 from Eq. 1), written by
# tests/golden/make_converged_k.py from oracle/ only.  The steady state is the
# fixed point of the oracle's FP64 step (oracle/steady.py); `residual` is the
# max-norm of S(f) - f at the stored state; converged: the root finder met
# its tolerance (4e-16).  Columns:
# name nx ny nz seed porosity tau drho k residual evals percolates converged
"""


def line(r):
    return (f"{r['name']} {r['nx']} {r['ny']} {r['nz']} {r['seed']} {r['porosity']!r} {r['tau']!r} {r['drho']!r} "
            f"{r['k']!r} {r['residual']:.3e} {r['evals']} {int(r['percolates'])} {int(r['converged'])}")


def read_existing():
    rows, samples = {}, {}
    if os.path.exists(OUT_K):
        for ln in open(OUT_K):
            if ln.strip() and not ln.startswith("#"):
                rows[ln.split()[0]] = ln.rstrip("\n")
    if os.path.exists(OUT_U):
        z = np.load(OUT_U)
        for key in z.files:
            samples[key] = z[key]
    return rows, samples


def save_part(r):
    os.makedirs(PARTS, exist_ok=True)
    np.savez_compressed(os.path.join(PARTS, r["name"] + ".npz"), line=np.array(line(r)), idx=r["idx"], u=r["u"])


def merge():
    rows, samples = read_existing()
    if os.path.isdir(PARTS):
        for fn in sorted(os.listdir(PARTS)):
            if not fn.endswith(".npz"):
                continue
            z = np.load(os.path.join(PARTS, fn))
            ln = str(z["line"])
            name = ln.split()[0]
            rows[name] = ln
            samples[name + "/idx"] = z["idx"]
            samples[name + "/u"] = z["u"]
    with open(OUT_K, "w") as fh:
        fh.write(HEADER)
        for name in sorted(rows):
            fh.write(rows[name] + "\n")
    np.savez_compressed(OUT_U, **samples)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--sets", default="C1,C2,C3")
    ap.add_argument("--procs", type=int, default=max(1, (os.cpu_count() or 2) - 1))
    ap.add_argument("--names", default="", help="only these domains (comma list), e.g. to re-solve one")
    ap.add_argument("--maxiter", type=int, default=MAXITER, help="Newton iterations of the root finder")
    ap.add_argument("--inner", type=int, default=INNER, help="inner (LGMRES) iterations per Newton step")
    ap.add_argument("--merge-only", action="store_true", help="only merge the saved results into the final files")
    a = ap.parse_args()
    if a.merge_only:
        merge()
        return
    todo = sorted(jobs(set(a.sets.split(","))), key=lambda j: -cost(j[2]))
    if a.names:
        keep = set(a.names.split(","))
        todo = [j for j in todo if j[1] in keep]
    todo = [j + (a.maxiter, a.inner) for j in todo]
    ctx = mp.get_context("spawn")
    with ctx.Pool(a.procs) as pool, open(PARTIAL, "a") as part:
        for r in pool.imap_unordered(solve, todo):
            save_part(r)
            part.write(line(r) + f"  # {r['seconds']:.0f} s converged={r['converged']}\n")
            part.flush()
            print(line(r), f"{r['seconds']:.0f} s", flush=True)
    merge()


if __name__ == "__main__":
    main()
