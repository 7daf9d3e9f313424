"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerances.  The device state is FP32 shifted populations g = f - w rho_0.
One step of stream + boundary + collide is a few dozen FP32 operations on
values of magnitude max|g|, so one step's rounding is a few ulp of max|g|
(2^-24 ~ 6e-8 relative); over up to 10 steps the errors add, not multiply
(the BGK update is a contraction for tau > 1/2).  The bound used is
    |g_gpu - g_oracle| <= 2e-6 max|g_oracle|,
i.e. ~30 ulp of the largest population.  Converged permeabilities must agree
to 1e-4 relative and velocity fields to 1e-3 relative L2.
QSGS masks, segment tables and statuses are integer work and must match
exactly.
"""
import numpy as np
import pytest

import oracle as O
from paper_1609_09685_gb300 import build, lbm, workloads

pytestmark = pytest.mark.gpu

REL = 2e-6


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    lbm.load()
    O.build()


def _w(q):
    return O.lattice(q)[1]


def _shifted(f, q, rho0=1.0):
    return f - _w(q) * rho0


def _assert_close(gpu_f, orc_f, q, mask, rel=REL):
    fluid = ~mask.astype(bool)
    a = _shifted(gpu_f, q)[fluid]
    b = _shifted(orc_f, q)[fluid]
    scale = max(np.abs(b).max(), 1e-300)
    err = np.abs(a - b).max()
    assert err <= rel * scale, f"max err {err:.3e} vs scale {scale:.3e}"
    # solids carry nothing
    assert np.all(gpu_f[~fluid] == 0.0)


def _masks_2d():
    rng = np.random.default_rng(5)
    out = {}
    out["4x4"] = np.zeros((4, 4), np.uint8)
    m = np.zeros((6, 8), np.uint8)
    m[2, 3] = m[0, 5] = m[5, 1] = 1
    out["8x6_corners"] = m
    ch = np.zeros((8, 16), np.uint8)
    ch[0] = ch[-1] = 1
    out["channel16x8"] = ch
    r = (rng.random((13, 70)) < 0.3).astype(np.uint8)  # two full segments + ragged tail
    r[:, 0] = 0
    out["ragged70x13"] = r
    r2 = (rng.random((9, 96)) < 0.25).astype(np.uint8)  # exact multiple of 32
    r2[3, 0] = 1  # a solid inlet node
    r2[4, 95] = 1  # a solid outlet node
    out["full96x9"] = r2
    out["row1"] = np.zeros((1, 40), np.uint8)  # ny = 1: both mirror planes on one row
    return out


# --------------------------------------------------------------------------
# QSGS: bit-exact with the oracle
# --------------------------------------------------------------------------

@pytest.mark.parametrize("shape,seed,phi", [
    ((50, 100), 1, 0.74), ((13, 70), 7, 0.6), ((200, 400), 1, 0.7394), ((16, 24, 40), 3, 0.7),
    ((8, 16), 5, 1.0), ((8, 16), 5, 0.0),
])
def test_qsgs_bit_exact(shape, seed, phi):
    g, it_g = lbm.lbm_qsgs(seed, shape, 0.02, phi)
    o, it_o = O.qsgs(shape, seed, 0.02, phi)
    assert it_g == it_o
    assert np.array_equal(g, o)


def test_qsgs_all_cores_tie_break():
    g, _ = lbm.lbm_qsgs(5, (8, 16), 1.0, 0.5)
    o, _ = O.qsgs((8, 16), 5, 1.0, 0.5)
    assert np.array_equal(g, o)


# --------------------------------------------------------------------------
# Steps from the initial state and from random states
# --------------------------------------------------------------------------

@pytest.mark.parametrize("name", list(_masks_2d().keys()))
@pytest.mark.parametrize("eq", [0, 1])
@pytest.mark.parametrize("pairs", [True, False])
def test_d2q9_steps_from_init(name, eq, pairs):
    mask = _masks_2d()[name]
    tau, drho = 0.8, 1e-3
    opts = lbm.make_options(equilibrium=eq, in_place_pairs=pairs)
    with lbm.lbm_create_domain(mask, tau, drho, opts) as s:
        f0 = lbm.lbm_get_populations(s, 0)
        _assert_close(f0, O.init(mask, 1 + drho, 1.0), 9, mask)
        ref = f0
        done = 0
        for n in (1, 1, 8):
            lbm.lbm_step(s, n)
            done += n
            ref = O.run(mask, ref, tau, 1 + drho, 1.0, n, eq)
            _assert_close(lbm.lbm_get_populations(s, 0), ref, 9, mask)


@pytest.mark.parametrize("name", ["8x6_corners", "ragged70x13", "full96x9", "row1"])
@pytest.mark.parametrize("eq", [0, 1])
def test_d2q9_one_step_from_random_state(name, eq):
    mask = _masks_2d()[name]
    tau, drho = 0.67, 2e-3
    rng = np.random.default_rng(9)
    w = _w(9)
    f = w * (1 + 0.05 * rng.standard_normal(mask.shape + (9,)))
    f[mask.astype(bool)] = 0
    with lbm.lbm_create_domain(mask, tau, drho, lbm.make_options(equilibrium=eq)) as s:
        lbm.lbm_set_populations(s, 0, f)
        start = lbm.lbm_get_populations(s, 0)  # FP32-rounded start
        lbm.lbm_step(s, 1)
        _assert_close(lbm.lbm_get_populations(s, 0), O.step(mask, start, tau, 1 + drho, 1.0, eq),
                      9, mask)


def _masks_3d():
    rng = np.random.default_rng(11)
    out = {}
    out["4x4x4"] = np.zeros((4, 4, 4), np.uint8)
    r = (rng.random((5, 7, 37)) < 0.3).astype(np.uint8)
    r[..., 0] = 0
    out["ragged37x7x5"] = r
    out["plates"] = np.zeros((3, 8, 12), np.uint8)
    out["plates"][:, 0] = out["plates"][:, -1] = 1
    out["slab1"] = np.zeros((1, 6, 20), np.uint8)  # nz = 1 through the 3D entry point
    return out


@pytest.mark.parametrize("name", list(_masks_3d().keys()))
@pytest.mark.parametrize("eq", [0, 1])
@pytest.mark.parametrize("pairs", [True, False])
def test_d3q19_steps_from_init_and_random(name, eq, pairs):
    mask = _masks_3d()[name]
    tau, drho = 0.9, 1e-3
    with lbm.lbm_create_domain_3d(mask, tau, drho, lbm.make_options(equilibrium=eq, in_place_pairs=pairs)) as s:
        f0 = lbm.lbm_get_populations(s, 0)
        _assert_close(f0, O.init(mask, 1 + drho, 1.0), 19, mask)
        lbm.lbm_step(s, 10)
        _assert_close(lbm.lbm_get_populations(s, 0), O.run(mask, f0, tau, 1 + drho, 1.0, 10, eq),
                      19, mask)
        rng = np.random.default_rng(2)
        f = _w(19) * (1 + 0.05 * rng.standard_normal(mask.shape + (19,)))
        f[mask.astype(bool)] = 0
        lbm.lbm_set_populations(s, 0, f)
        start = lbm.lbm_get_populations(s, 0)
        lbm.lbm_step(s, 1)
        _assert_close(lbm.lbm_get_populations(s, 0), O.step(mask, start, tau, 1 + drho, 1.0, eq),
                      19, mask)


@pytest.mark.parametrize("dim", [2, 3])
def test_in_place_pairs_match_pull_steps(dim):
    """Two steps in place (gather step + local step) perform the arithmetic of
    two pull steps: every boundary rule (bounce-back, mirror, Zou-He) reads and
    writes the same slots and every kernel relaxes a node with the same
    operations, so the two schemes agree bit for bit from a random state over
    many steps, and 1 + 2k steps mix both."""
    rng = np.random.default_rng(31 + dim)
    if dim == 2:
        mask = (rng.random((23, 75)) < 0.3).astype(np.uint8)
        q, create = 9, lbm.lbm_create_domain
    else:
        mask = (rng.random((6, 9, 40)) < 0.3).astype(np.uint8)
        q, create = 19, lbm.lbm_create_domain_3d
    f = _w(q) * (1 + 0.05 * rng.standard_normal(mask.shape + (q,)))
    f[mask.astype(bool)] = 0
    out = {}
    for pairs in (True, False):
        with create(mask, 0.7, 1e-3, lbm.make_options(in_place_pairs=pairs)) as s:
            lbm.lbm_set_populations(s, 0, f)
            res = []
            for n in (2, 1, 6, 11):
                lbm.lbm_step(s, n)
                res.append(lbm.lbm_get_populations(s, 0))
            out[pairs] = res
    for a, b in zip(out[True], out[False]):
        assert np.array_equal(a, b)


def test_staged_gather_matches_direct_gather_bitwise():
    """The staged gather step (bulk copies of whole source-row ranges into
    shared memory, any tile height) and the direct one (per-node loads) do the
    same arithmetic on the same values: after in-place pairs from the initial
    state and from a random state, populations are bit-identical, for a batch
    of ragged, 32-multiple, single-row and channel masks (faces, mirrors and
    bounce-back on tile edges), with both equilibria."""
    masks = list(_masks_2d().values())
    taus = [0.6 + 0.1 * i for i in range(len(masks))]
    drhos = [1e-3] * len(masks)
    for eq in (0, 1):
        runs = {}
        for rows in (-1, 1, 2, 3, 4):
            opts = lbm.make_options(equilibrium=eq, tile_rows=rows)
            with lbm.lbm_batch_create(masks, taus, drhos, opts) as s:
                lbm.lbm_step(s, 6)
                for d, m in enumerate(masks):
                    f = O.init(m, 1 + drhos[d], 1.0)
                    f[~m.astype(bool)] += 1e-3 * np.random.default_rng(d).standard_normal(
                        f[~m.astype(bool)].shape)
                    if d % 2:
                        lbm.lbm_set_populations(s, d, f)
                lbm.lbm_step(s, 8)
                obs = lbm.lbm_step_observe(s, 2)
                runs[rows] = ([lbm.lbm_get_populations(s, d) for d in range(len(masks))], obs)
        for rows in (1, 2, 3, 4):
            for a, b in zip(runs[-1][0], runs[rows][0]):
                assert np.array_equal(a, b), (eq, rows)
            assert np.array_equal(runs[-1][1], runs[rows][1])


def test_band_gather_matches_direct_gather_bitwise():
    """The band gather step (a block walks down a band of rows, staging each
    row's compact range of every plane in a shared-memory ring by bulk copies)
    and the direct one (per-node loads) do the same arithmetic on the same
    values: after in-place pairs from the initial state and from a random
    state, populations and observables are bit-identical.  Masks: the small
    ragged, 32-multiple, single-row and channel cases, plus domains wide enough
    to be cut into two and three pieces of the width (a solid block, a fluid
    column on a piece edge), for band heights from one row to the maximum."""
    rng = np.random.default_rng(11)
    masks = list(_masks_2d().values())
    w1 = (rng.random((21, 530)) < 0.3).astype(np.uint8)  # 17 segments: pieces of 9 and 8
    w1[:, 288] = 0  # fluid column on the piece edge (x = 32 * 9)
    w1[5:9, 100:200] = 1
    masks.append(w1)
    w2, _ = O.qsgs((37, 1100), 4, 0.02, 0.7)  # 35 segments: pieces of 12, 12, 11
    masks.append(w2)
    w3 = np.zeros((70, 65), np.uint8)  # 3 segments, 70 rows: several bands per column
    w3[10:20, 30:40] = 1
    masks.append(w3)
    taus = [0.6 + 0.07 * i for i in range(len(masks))]
    drhos = [1e-3] * len(masks)
    for eq in (0, 1):
        runs = {}
        for rows in (-1, 1, 2, 5, 32, 64):
            opts = lbm.make_options(equilibrium=eq, band_rows=rows, tile_rows=0)
            with lbm.lbm_batch_create(masks, taus, drhos, opts) as s:
                assert lbm.lbm_get_launch(s)["band_rows"] == max(rows, 0)
                lbm.lbm_step(s, 6)
                for d, m in enumerate(masks):
                    f = O.init(m, 1 + drhos[d], 1.0)
                    f[~m.astype(bool)] += 1e-3 * np.random.default_rng(d).standard_normal(
                        f[~m.astype(bool)].shape)
                    if d % 2:
                        lbm.lbm_set_populations(s, d, f)
                lbm.lbm_step(s, 8)
                obs = lbm.lbm_step_observe(s, 2)
                runs[rows] = ([lbm.lbm_get_populations(s, d) for d in range(len(masks))], obs)
        for rows in (1, 2, 5, 32, 64):
            for d, (a, b) in enumerate(zip(runs[-1][0], runs[rows][0])):
                assert np.array_equal(a, b), (eq, rows, d)
            assert np.array_equal(runs[-1][1], runs[rows][1])


def test_band_gather_steps_match_oracle():
    """Band gather pairs against the FP64 oracle directly (not only through the
    direct gather step): 10 steps from a random state on a two-piece domain
    and a channel, TRT and BGK, within the step tolerance of the other kernels."""
    rng = np.random.default_rng(3)
    m1 = (rng.random((24, 530)) < 0.3).astype(np.uint8)
    m2 = np.zeros((9, 40), np.uint8)
    m2[0] = m2[-1] = 1
    for coll in (0, 1):
        opts = lbm.make_options(band_rows=8, collision=coll)
        for m, tau in ((m1, 0.7), (m2, 1.3)):
            f0 = O.init(m, 1.001, 1.0)
            fl = ~m.astype(bool)
            f0[fl] += 1e-3 * rng.standard_normal(f0[fl].shape)
            with lbm.lbm_create_domain(m, tau, 1e-3, opts) as s:
                assert lbm.lbm_get_launch(s)["band_rows"] == 8
                lbm.lbm_set_populations(s, 0, f0)
                start = lbm.lbm_get_populations(s, 0)  # FP32-rounded start
                lbm.lbm_step(s, 10)
                g = lbm.lbm_get_populations(s, 0)
            tau_m = O.tau_minus(tau, 3.0 / 16.0) if coll else None
            _assert_close(g, O.run(m, start, tau, 1.001, 1.0, 10, tau_m=tau_m), 9, m)


@pytest.mark.parametrize("dim", [2, 3])
def test_pair_blocks_match_whole_batch_pairs_bitwise(dim):
    """L2-blocked pairs (the gather step of block k + 1, then the local step of
    block k, blocks of about pair_block_mb MB cut between row groups in 2D and
    between z planes in 3D) give the populations and observables of
    whole-batch pairs bit for bit, from a random state, for blocks from a few
    rows to a whole domain."""
    rng = np.random.default_rng(40 + dim)
    if dim == 2:
        shapes = [(300, 600), (97, 211), (150, 1000)]
        create, q = lbm.lbm_batch_create, 9
    else:
        shapes = [(40, 48, 64), (17, 23, 50)]
        create, q = lbm.lbm_batch_create, 19
    masks = [(rng.random(sh) < 0.3).astype(np.uint8) for sh in shapes]
    taus = [0.55 + 0.2 * i for i in range(len(masks))]
    drhos = [1e-3] * len(masks)
    runs = {}
    for mb in (-1, 1, 2, 5, 64):
        with create(masks, taus, drhos, lbm.make_options(pair_block_mb=mb, band_rows=-1)) as s:
            assert lbm.lbm_get_launch(s)["pair_block_mb"] == max(mb, 0)
            for d, m in enumerate(masks):
                f = O.init(m, 1 + drhos[d], 1.0)
                fl = ~m.astype(bool)
                f[fl] += 1e-3 * np.random.default_rng(d).standard_normal(f[fl].shape)
                lbm.lbm_set_populations(s, d, f)
            lbm.lbm_step(s, 9)
            obs = lbm.lbm_step_observe(s, 1)
            runs[mb] = ([lbm.lbm_get_populations(s, d) for d in range(len(masks))], obs)
    for mb in (1, 2, 5, 64):
        for d, (a, b) in enumerate(zip(runs[-1][0], runs[mb][0])):
            assert np.array_equal(a, b), (dim, mb, d)
        assert np.array_equal(runs[-1][1], runs[mb][1])


def test_profile_steps_runs_the_same_steps_with_per_kernel_times():
    """lbm_profile_steps advances the state exactly as lbm_step does (the same
    kernels, launched one by one with events around them) and reports one
    gather and one local launch per pair and a pull launch for the odd step."""
    mask, _ = O.qsgs((30, 90), 8, 0.02, 0.72)
    with lbm.lbm_create_domain(mask, 0.8, 1e-3) as a, lbm.lbm_create_domain(mask, 0.8, 1e-3) as b:
        lbm.lbm_step(a, 7)
        prof = lbm.lbm_profile_steps(b, 7)
        assert np.array_equal(lbm.lbm_get_populations(a, 0), lbm.lbm_get_populations(b, 0))
        assert lbm.lbm_get_step(b) == 7
    assert prof["gather"][1] == 3 and prof["local"][1] == 3 and prof["pull"][1] == 1
    assert prof["pull_observe"] == (0.0, 0)
    assert all(prof[k][0] > 0 for k in ("gather", "local", "pull"))


def test_rest_state_is_exactly_zero_on_device():
    mask, _ = O.qsgs((30, 70), 4, 0.02, 0.7)
    with lbm.lbm_create_domain(mask, 0.7, 0.0) as s:
        lbm.lbm_step(s, 50)
        f = lbm.lbm_get_populations(s, 0)
        fluid = ~mask.astype(bool)
        assert np.array_equal(f[fluid], np.broadcast_to(_w(9), f[fluid].shape))


def test_batch_of_uneven_domains_matches_separate_oracle_runs():
    masks = [O.qsgs((20, 50), 1, 0.02, 0.7)[0], O.qsgs((7, 33), 2, 0.02, 0.75)[0],
             O.qsgs((31, 64), 3, 0.02, 0.65)[0]]
    taus = [0.6, 1.1, 0.8]
    drhos = [1e-3, 5e-4, 2e-4]
    with lbm.lbm_batch_create(masks, taus, drhos) as s:
        assert s.n_domains == 3
        lbm.lbm_step(s, 7)
        for d, m in enumerate(masks):
            ref = O.run(m, O.init(m, 1 + drhos[d], 1.0), taus[d], 1 + drhos[d], 1.0, 7)
            _assert_close(lbm.lbm_get_populations(s, d), ref, 9, m)
            assert lbm.lbm_domain_fluid_nodes(s, d) == int((m == 0).sum())


def test_observables_match_oracle_moments():
    mask, _ = O.qsgs((24, 60), 6, 0.02, 0.72)
    tau, drho = 0.75, 1e-3
    with lbm.lbm_create_domain(mask, tau, drho) as s:
        lbm.lbm_step(s, 30)
        f_prev = lbm.lbm_get_populations(s, 0)
        obs0 = lbm.lbm_step_observe(s, 0)  # sets u_prev to the current u
        obs = lbm.lbm_step_observe(s, 20)[0]
        f = lbm.lbm_get_populations(s, 0)
    rho, ux, uy = O.fields(mask, f)
    rp, uxp, uyp = O.fields(mask, f_prev)
    fluid = ~mask.astype(bool)
    jx = (rho * ux)[fluid].sum()
    du2 = ((ux - uxp) ** 2 + (uy - uyp) ** 2)[fluid].sum()
    u2 = (ux ** 2 + uy ** 2)[fluid].sum()
    assert obs[0] == pytest.approx(O.link_flux(mask, f).sum(), rel=1e-5)
    assert obs[6] == pytest.approx(jx, rel=1e-5)
    assert obs[1] == pytest.approx(du2, rel=1e-3)
    assert obs[2] == pytest.approx(u2, rel=1e-5)
    assert obs[3] == pytest.approx(np.sqrt(ux ** 2 + uy ** 2)[fluid].max(), rel=1e-5)
    assert obs[4] == 0
    assert obs[5] == pytest.approx((rho - 1.0)[fluid].sum(), rel=1e-5)
    assert obs0.shape == (1, lbm.NUM_OBS)


# --------------------------------------------------------------------------
# Converged permeability and fields (1e-4 / 1e-3)
# --------------------------------------------------------------------------

def _converged_oracle(mask, tau, drho, eq=0, tol=1e-10, start=None):
    f = O.init(mask, 1 + drho, 1.0) if start is None else start
    g, rc, steps, res = O.run_to_steady(mask, f, tau, 1 + drho, 1.0, tol, 2_000_000, eq=eq)
    assert rc == 0, (rc, steps, res)
    return g


def test_small_2d_workload_permeability_and_fields():
    wl = workloads.small_2d()
    d = wl.domains[0]
    mask, _ = lbm.lbm_qsgs(d.seed, d.shape, d.core_p, d.porosity)
    with lbm.lbm_create_domain(mask, d.tau, d.drho) as s:
        rc, st, steps, res = lbm.lbm_run_to_steady(s, wl.tol, wl.max_steps)
        assert st[0] in (lbm.LBM_OK, lbm.LBM_STALLED)
        k, kn = lbm.lbm_permeability(s)
        rho, ux, uy = lbm.lbm_get_fields(s, 0)
    g = _converged_oracle(mask, d.tau, d.drho)
    k_o = O.permeability(mask, g, d.tau, 1 + d.drho, 1.0)
    assert k[0] == pytest.approx(k_o, rel=1e-4)
    assert kn[0] == pytest.approx(O.knudsen(d.tau, d.nx), rel=1e-14)
    r_o, ux_o, uy_o = O.fields(mask, g)
    num = np.sqrt(((ux - ux_o) ** 2 + (uy - uy_o) ** 2).sum())
    den = np.sqrt((ux_o ** 2 + uy_o ** 2).sum())
    assert num / den < 1e-3


def test_channel_permeability_matches_exact_solution_on_device():
    h, tau = 16, 0.8
    mask = np.zeros((h + 2, 6 * h), np.uint8)
    mask[0] = mask[-1] = 1
    with lbm.lbm_create_domain(mask, tau, 1e-3, lbm.make_options(equilibrium=1)) as s:
        lbm.lbm_run_to_steady(s, 1e-9, 200000)
        k, _ = lbm.lbm_permeability(s)
        f = lbm.lbm_get_populations(s, 0)
    g = _converged_oracle(mask, tau, 1e-3, eq=1, tol=1e-12)
    assert k[0] == pytest.approx(O.permeability(mask, g, tau, 1.001, 1.0), rel=1e-4)


def test_checkpoint_round_trip_is_bitwise(tmp_path):
    mask, _ = O.qsgs((20, 45), 8, 0.02, 0.72)
    p = str(tmp_path / "c.ckpt")
    with lbm.lbm_create_domain(mask, 0.9, 1e-3) as a:
        lbm.lbm_step(a, 37)
        lbm.lbm_save(a, p)
        lbm.lbm_step(a, 25)
        fa = lbm.lbm_get_populations(a, 0)
    with lbm.lbm_load(p, masks=[mask]) as b:
        assert lbm.lbm_get_step(b) == 37
        lbm.lbm_step(b, 25)
        fb = lbm.lbm_get_populations(b, 0)
    assert np.array_equal(fa, fb)


def test_divergence_is_reported():
    mask = np.zeros((8, 20), np.uint8)
    with lbm.lbm_create_domain(mask, 0.8, 1e-3) as s:
        f = lbm.lbm_get_populations(s, 0)
        f[3, 5, 2] = np.nan
        lbm.lbm_set_populations(s, 0, f)
        with pytest.raises(lbm.LBMError) as e:
            lbm.lbm_run_to_steady(s, 1e-9, 1000)
        assert e.value.status == lbm.LBM_DIVERGED


def test_cancel_flag_stops_the_run_between_intervals():
    import ctypes as C
    mask, _ = O.qsgs((20, 40), 3, 0.02, 0.75)
    flag = C.c_int32(1)
    opts = lbm.make_options(cancel_flag=C.addressof(flag))
    with lbm.lbm_create_domain(mask, 0.8, 1e-3, opts) as s:
        with pytest.raises(lbm.LBMError) as e:
            lbm.lbm_run_to_steady(s, 1e-9, 100000)
        assert e.value.status == lbm.LBM_CANCELLED
        assert lbm.lbm_get_step(s) == 0  # cancelled before the first interval
        flag.value = 0
        rc, st, steps, _ = lbm.lbm_run_to_steady(s, 1e-9, 100000)
        assert st[0] == lbm.LBM_OK


# --------------------------------------------------------------------------
# TRT collision
# --------------------------------------------------------------------------

@pytest.mark.parametrize("lam", [3.0 / 16.0, 0.4])
@pytest.mark.parametrize("pairs", [True, False])
def test_trt_steps_match_oracle_2d_and_3d(lam, pairs):
    """TRT on the GPU against the oracle's TRT: from the ramp start and from a
    random state, 2D (all boundary kinds) and 3D, with in-place pairs and with
    pull steps."""
    rng = np.random.default_rng(41)
    cases = [(9, _masks_2d()["8x6_corners"], lbm.lbm_create_domain),
             (9, _masks_2d()["ragged70x13"], lbm.lbm_create_domain),
             (19, _masks_3d()["ragged37x7x5"], lbm.lbm_create_domain_3d)]
    tau, drho = 0.7, 1e-3
    tm = O.tau_minus(tau, lam)
    for q, mask, create in cases:
        opts = lbm.make_options(collision=lbm.LBM_COLL_TRT, trt_lambda=lam, in_place_pairs=pairs)
        with create(mask, tau, drho, opts) as s:
            f0 = lbm.lbm_get_populations(s, 0)
            lbm.lbm_step(s, 6)
            _assert_close(lbm.lbm_get_populations(s, 0), O.run(mask, f0, tau, 1 + drho, 1.0, 6, tau_m=tm),
                          q, mask)
            f = _w(q) * (1 + 0.05 * rng.standard_normal(mask.shape + (q,)))
            f[mask.astype(bool)] = 0
            lbm.lbm_set_populations(s, 0, f)
            start = lbm.lbm_get_populations(s, 0)
            lbm.lbm_step(s, 3)
            _assert_close(lbm.lbm_get_populations(s, 0), O.run(mask, start, tau, 1 + drho, 1.0, 3, tau_m=tm),
                          q, mask)


def test_trt_channel_on_device_gives_lambda_permeability():
    """Pressure-driven channel, linear equilibrium, TRT with Lambda = 3/16:
    the mid-channel permeability is (h^2 - 1 + 8 Lambda)/12 for every tau."""
    h, lam = 10, 3.0 / 16.0
    ny, nx = h + 2, 6 * h
    mask = np.zeros((ny, nx), np.uint8)
    mask[0] = mask[-1] = 1
    for tau in (0.6, 1.2):
        opts = lbm.make_options(equilibrium=lbm.LBM_EQ_LINEAR, collision=lbm.LBM_COLL_TRT, trt_lambda=lam)
        with lbm.lbm_create_domain(mask, tau, 1e-3, opts) as s:
            lbm.lbm_run_to_steady(s, 1e-9, 400000)
            rho, ux, _ = lbm.lbm_get_fields(s, 0)
        xm = nx // 2
        j = (rho * ux)[1:-1, xm]
        beta = (rho[1:-1, xm + h // 2] - rho[1:-1, xm - h // 2]).mean() / (2 * (h // 2))
        k_local = (tau - 0.5) / 3.0 * j.mean() / (-beta / 3.0)
        assert k_local == pytest.approx((h * h - 1 + 8 * lam) / 12.0, rel=2e-4)


def test_trt_converged_permeability_matches_oracle():
    mask, _ = O.qsgs((40, 80), 9, 0.02, 0.72)
    tau, drho, lam = 1.2, 1e-3, 3.0 / 16.0
    opts = lbm.make_options(collision=lbm.LBM_COLL_TRT, trt_lambda=lam)
    with lbm.lbm_create_domain(mask, tau, drho, opts) as s:
        lbm.lbm_run_to_steady(s, 1e-9, 2_000_000)
        k, _ = lbm.lbm_permeability(s)
    f0 = O.init(mask, 1 + drho, 1.0)
    g, rc, _, _ = O.run_to_steady(mask, f0, tau, 1 + drho, 1.0, 1e-10, 3_000_000, tau_m=O.tau_minus(tau, lam))
    assert rc == 0
    assert k[0] == pytest.approx(O.permeability(mask, g, tau, 1 + drho, 1.0), rel=1e-4)


# --------------------------------------------------------------------------
# Local pore size and local Knudsen number
# --------------------------------------------------------------------------

def test_local_knudsen_matches_oracle_bit_exact():
    """Integer squared distances bit-exact with the oracle's brute force, on 2D
    and 3D masks spanning many blocks, a channel and a mask without solids."""
    rng = np.random.default_rng(51)
    cases = [(O.qsgs((70, 150), 3, 0.02, 0.7)[0], 0.8, lbm.lbm_create_domain),
             ((rng.random((7, 13, 33)) < 0.2).astype(np.uint8), 0.9, lbm.lbm_create_domain_3d)]
    ch = np.zeros((9, 40), np.uint8)
    ch[0] = ch[-1] = 1
    cases.append((ch, 0.7, lbm.lbm_create_domain))
    cases.append((np.zeros((5, 12), np.uint8), 0.7, lbm.lbm_create_domain))
    for mask, tau, create in cases:
        with create(mask, tau, 1e-3) as s:
            d2, h, kn = lbm.lbm_local_knudsen(s, 0)
        assert np.array_equal(d2, O.pore_d2(mask))
        h_o, kn_o = O.local_knudsen(mask, tau)
        assert np.array_equal(np.isinf(h), np.isinf(h_o))
        fin = np.isfinite(h_o)
        assert np.allclose(h[fin], h_o[fin], rtol=0, atol=1e-12)
        assert np.allclose(kn, kn_o, rtol=1e-14, atol=0)


# --------------------------------------------------------------------------
# Force-driven flow with every face periodic (Sec. 2's 3D experiment)
# --------------------------------------------------------------------------

def _forced_masks():
    rng = np.random.default_rng(61)
    m2 = (rng.random((13, 70)) < 0.25).astype(np.uint8)   # solids on every face: x- and y-wrap cases
    m3 = (rng.random((5, 9, 37)) < 0.25).astype(np.uint8)
    return [(9, m2), (19, m3)]


@pytest.mark.parametrize("pairs", [True, False])
@pytest.mark.parametrize("eq", [0, 1])
def test_forced_periodic_steps_match_oracle(eq, pairs):
    """Steps with periodic wrap in x, y (and z), halfway bounce-back and Guo
    forcing -- in-place pairs of the forced gather and local steps, or pull
    steps -- against the oracle from the rest start and a random state."""
    rng = np.random.default_rng(7)
    tau, g = 0.8, 2e-4
    for q, mask in _forced_masks():
        with lbm.lbm_batch_create_forced([mask], [tau], [g], lbm.make_options(equilibrium=eq,
                                                                               in_place_pairs=pairs)) as s:
            f0 = lbm.lbm_get_populations(s, 0)
            lbm.lbm_step(s, 8)
            _assert_close(lbm.lbm_get_populations(s, 0), O.run_forced(mask, f0, tau, g, 8, eq), q, mask)
            f = _w(q) * (1 + 0.05 * rng.standard_normal(mask.shape + (q,)))
            f[mask.astype(bool)] = 0
            lbm.lbm_set_populations(s, 0, f)
            start = lbm.lbm_get_populations(s, 0)
            lbm.lbm_step(s, 1)
            _assert_close(lbm.lbm_get_populations(s, 0), O.step_forced(mask, start, tau, g, eq), q, mask)


@pytest.mark.parametrize("coll", [0, 1])
def test_forced_pairs_match_forced_pull_steps_bitwise(coll):
    """The forced in-place pair (gather step writing each result back to the
    slot it read -- periodic streaming and bounce-back keep the pairing exact
    -- then the local step) relaxes every node with the same written-out
    operations as the forced pull step: bit-identical populations and
    observables from a random state, BGK and TRT, both equilibria, 2D and 3D,
    for even and odd step counts."""
    rng = np.random.default_rng(71 + coll)
    for eq in (0, 1):
        for q, mask in _forced_masks():
            f = _w(q) * (1 + 0.05 * rng.standard_normal(mask.shape + (q,)))
            f[mask.astype(bool)] = 0
            out = {}
            for pairs in (True, False):
                opts = lbm.make_options(equilibrium=eq, in_place_pairs=pairs, collision=coll)
                with lbm.lbm_batch_create_forced([mask, mask[..., ::-1].copy()], [0.7, 1.1], [3e-4, 1e-4],
                                                 opts) as s:
                    lbm.lbm_set_populations(s, 0, f)
                    res = []
                    for n in (2, 1, 6):
                        lbm.lbm_step(s, n)
                        res.append([lbm.lbm_get_populations(s, d) for d in range(2)])
                    res.append(lbm.lbm_step_observe(s, 4))
                    res.append([lbm.lbm_get_populations(s, d) for d in range(2)])
                    out[pairs] = res
            for a, b in zip(out[True], out[False]):
                if isinstance(a, list):
                    for x, y in zip(a, b):
                        assert np.array_equal(x, y), (eq, q, coll)
                else:
                    assert np.array_equal(a, b), (eq, q, coll)


def test_forced_permeability_matches_oracle_and_translation():
    """Converged Eq. 2 permeability of a porous 3D domain within 1e-4 of the
    oracle's; the same domain shifted periodically in x and y gives the same
    k (exercises the wrap at both x ends and across rows)."""
    mask, _ = O.qsgs((8, 10, 12), 4, 0.05, 0.75)
    tau, g = 0.8, 1e-5
    f, rc, _, _ = O.run_forced_to_steady(mask, O.init(mask, 1.0, 1.0), tau, g, 1e-10, 100000)
    assert rc == 0
    k_o = O.permeability_forced(mask, f, tau, g)
    shifted = np.roll(np.roll(mask, 5, axis=2), 3, axis=1)
    with lbm.lbm_batch_create_forced([mask, shifted], [tau, tau], [g, g]) as s:
        lbm.lbm_run_to_steady(s, 1e-8, 200000)
        k, _ = lbm.lbm_permeability(s)
    assert k[0] == pytest.approx(k_o, rel=1e-4)
    assert k[1] == pytest.approx(k_o, rel=1e-4)


def test_forced_k_force_independent_with_stokes_equilibrium_on_device():
    mask, _ = O.qsgs((8, 10, 12), 4, 0.05, 0.75)
    opts = lbm.make_options(equilibrium=lbm.LBM_EQ_LINEAR)
    with lbm.lbm_batch_create_forced([mask, mask], [0.8, 0.8], [1e-6, 5e-4], opts) as s:
        lbm.lbm_run_to_steady(s, 1e-8, 200000)
        k, _ = lbm.lbm_permeability(s)
    assert k[0] == pytest.approx(k[1], rel=1e-5)


def test_forced_solver_rejects_pressure_only_calls(tmp_path):
    mask = np.zeros((6, 10), np.uint8)
    with lbm.lbm_batch_create_forced([mask], [0.8], [1e-5]) as s:
        with pytest.raises(lbm.LBMError):
            lbm.lbm_save(s, str(tmp_path / "x.ckpt"))


def test_degenerate_domains_in_a_batch():
    """An all-solid domain (no fluid node at all) and a domain whose fluid
    does not connect inlet to outlet, batched with a normal one: the normal
    domain matches its separate oracle run, the all-solid one holds nothing,
    and the blocked one converges to zero flux (k = 0)."""
    normal, _ = O.qsgs((20, 48), 2, 0.02, 0.7)
    solid = np.ones((8, 40), np.uint8)
    blocked = np.zeros((10, 40), np.uint8)
    blocked[:, 20] = 1  # a solid wall across the channel
    masks = [normal, solid, blocked]
    taus, drhos = [0.8, 0.9, 0.7], [1e-3, 1e-3, 1e-3]
    with lbm.lbm_batch_create(masks, taus, drhos) as s:
        assert lbm.lbm_domain_fluid_nodes(s, 1) == 0
        lbm.lbm_step(s, 9)
        ref = O.run(normal, O.init(normal, 1 + drhos[0], 1.0), taus[0], 1 + drhos[0], 1.0, 9)
        _assert_close(lbm.lbm_get_populations(s, 0), ref, 9, normal)
        assert np.all(lbm.lbm_get_populations(s, 1) == 0.0)
        rc, st, steps, res = lbm.lbm_run_to_steady(s, 1e-7, 400000)
        k, _ = lbm.lbm_permeability(s)
    assert st[1] == lbm.LBM_OK and st[2] in (lbm.LBM_OK, lbm.LBM_STALLED)
    assert k[1] == 0.0
    assert abs(k[2]) < 1e-6 * abs(k[0])


def test_forced_observation_without_stepping_gives_eq2_flux():
    """An observation taken without a step on a force-driven solver reports
    Eq. 2's flux, so lbm_permeability agrees with the oracle's Eq. 2 on the
    same (GPU) populations, before and after stepping."""
    mask, _ = O.qsgs((6, 8, 20), 3, 0.05, 0.75)
    tau, g = 0.9, 1e-4
    with lbm.lbm_batch_create_forced([mask], [tau], [g]) as s:
        lbm.lbm_step(s, 40)
        lbm.lbm_step_observe(s, 0)
        k, _ = lbm.lbm_permeability(s)
        f = lbm.lbm_get_populations(s, 0)
        assert k[0] == pytest.approx(O.permeability_forced(mask, f, tau, g), rel=1e-5)
        lbm.lbm_step_observe(s, 1)
        k, _ = lbm.lbm_permeability(s)
        f = lbm.lbm_get_populations(s, 0)
        assert k[0] == pytest.approx(O.permeability_forced(mask, f, tau, g), rel=1e-5)


def test_forced_permeability_of_states_no_forced_step_produced():
    """The F/2 of Eq. 2's Guo momentum belongs to post-collision states of a
    forced step only: a fresh force-driven solver (fluid at rest) reports
    k = 0, and populations set by the caller report their own momentum; after
    a forced step the oracle's Eq. 2 applies again."""
    mask, _ = O.qsgs((6, 8, 20), 3, 0.05, 0.75)
    tau, g = 0.9, 1e-4
    nu = (tau - 0.5) / 3.0
    c = O.lattice(19)[0]
    with lbm.lbm_batch_create_forced([mask], [tau], [g]) as s:
        k, _ = lbm.lbm_permeability(s)
        assert k[0] == 0.0
        lbm.lbm_step(s, 30)
        f = lbm.lbm_get_populations(s, 0)
        lbm.lbm_set_populations(s, 0, f)
        k, _ = lbm.lbm_permeability(s)
        jx = float((f * c[:, 0]).sum())
        assert k[0] == pytest.approx(nu * jx / (mask.size * g), rel=1e-6)
        lbm.lbm_step(s, 1)
        lbm.lbm_step_observe(s, 0)
        k, _ = lbm.lbm_permeability(s)
        f = lbm.lbm_get_populations(s, 0)
        assert k[0] == pytest.approx(O.permeability_forced(mask, f, tau, g), rel=1e-5)


def test_batch_entry_points_match_the_handle_calls():
    """lbm_batch_run_to_steady / lbm_batch_permeability / lbm_batch_destroy
    are the batch forms of the handle calls: same statuses, bit-identical k."""
    masks = [O.qsgs((20, 40), 1, 0.02, 0.7)[0], O.qsgs((16, 48), 2, 0.02, 0.72)[0]]
    taus, drhos = [0.8, 1.0], [1e-3, 1e-3]
    s1 = lbm.lbm_batch_create(masks, taus, drhos)
    rc1, st1 = lbm.lbm_batch_run_to_steady(s1, 1e-8, 200000)
    k1 = lbm.lbm_batch_permeability(s1)
    lbm.lbm_batch_destroy(s1)
    assert s1.handle is None
    with lbm.lbm_batch_create(masks, taus, drhos) as s2:
        rc2, st2, _, _ = lbm.lbm_run_to_steady(s2, 1e-8, 200000)
        k2, _ = lbm.lbm_permeability(s2)
    assert rc1 == rc2 and np.array_equal(st1, st2)
    assert np.array_equal(k1, k2)


def test_solve_sharded_without_a_process_group_runs_the_whole_list():
    from paper_1609_09685_gb300 import sharding
    masks = [O.qsgs((20, 40), 1, 0.02, 0.7)[0], O.qsgs((16, 48), 2, 0.02, 0.72)[0]]
    k, st = sharding.solve_sharded(masks, [0.8, 1.0], [1e-3, 1e-3], tol=1e-8, max_steps=200000)
    with lbm.lbm_batch_create(masks, [0.8, 1.0], [1e-3, 1e-3]) as s:
        lbm.lbm_run_to_steady(s, 1e-8, 200000)
        k2, _ = lbm.lbm_permeability(s)
    assert np.array_equal(k, k2) and np.all(st == 0)


@pytest.mark.parametrize("eq", [0, 1])
def test_forced_trt_steps_match_oracle(eq):
    rng = np.random.default_rng(8)
    tau, g, lam = 0.8, 2e-4, 3.0 / 16.0
    tm = O.tau_minus(tau, lam)
    opts = lbm.make_options(equilibrium=eq, collision=lbm.LBM_COLL_TRT, trt_lambda=lam)
    for q, mask in _forced_masks():
        with lbm.lbm_batch_create_forced([mask], [tau], [g], opts) as s:
            f0 = lbm.lbm_get_populations(s, 0)
            lbm.lbm_step(s, 5)
            _assert_close(lbm.lbm_get_populations(s, 0), O.run_forced(mask, f0, tau, g, 5, eq, tau_m=tm), q, mask)
            f = _w(q) * (1 + 0.05 * rng.standard_normal(mask.shape + (q,)))
            f[mask.astype(bool)] = 0
            lbm.lbm_set_populations(s, 0, f)
            start = lbm.lbm_get_populations(s, 0)
            lbm.lbm_step(s, 1)
            _assert_close(lbm.lbm_get_populations(s, 0), O.step_forced(mask, start, tau, g, eq, tau_m=tm), q, mask)


def test_forced_channel_closed_forms_on_device():
    """Force-driven channel on the GPU: BGK gives the pressure-driven exact
    k = (h^2 - 1 + 8 (tau - 1/2)^2)/12, TRT with Lambda = 3/16 gives
    (h^2 + 1/2)/12 for every tau."""
    h, g = 8, 1e-6
    m = np.zeros((h + 2, 6), np.uint8)
    m[0] = m[-1] = 1
    for tau in (0.7, 1.2):
        for coll, expect in ((lbm.LBM_COLL_BGK, (h * h - 1 + 8 * (tau - 0.5) ** 2) / 12.0),
                             (lbm.LBM_COLL_TRT, (h * h + 0.5) / 12.0)):
            opts = lbm.make_options(equilibrium=lbm.LBM_EQ_LINEAR, collision=coll)
            with lbm.lbm_batch_create_forced([m], [tau], [g], opts) as s:
                lbm.lbm_run_to_steady(s, 1e-9, 400000)
                k, _ = lbm.lbm_permeability(s)
            assert k[0] * (h + 2) / h == pytest.approx(expect, rel=2e-4)
