"""Pins for the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: the lattice
isotropy conditions, an exact discrete channel solution derived by hand, exact
conservation laws, mirror symmetries of the boundary rules, the defining
equations of the Zou-He condition, hand-stepped populations, the kinetic-theory
mean free path behind the paper's Kn, exact linearity of the Stokes
equilibrium, and published splitmix64 outputs.
"""
import math
import os

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_ints(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        return [int(l.split()[0]) for l in fh if l.strip() and not l.startswith("#")]


def _random_mask(shape, frac, seed, open_x_ends=True):
    rng = np.random.default_rng(seed)
    m = (rng.random(shape) < frac).astype(np.uint8)
    if open_x_ends:
        m[..., 0] = 0
        m[..., -1] = 0
    return m


def _random_state(mask, seed, amp=0.05):
    """Positive non-equilibrium populations near w (a valid LBM state)."""
    q = 9 if mask.ndim == 2 else 19
    _, w, _ = O.lattice(q)
    rng = np.random.default_rng(seed)
    f = w * (1.0 + amp * rng.standard_normal(mask.shape + (q,)))
    f[mask.astype(bool)] = 0.0
    return f


# --------------------------------------------------------------------------
# Lattices: Qian et al. (1992) isotropy conditions (Sec. 2 names D2Q9/D3Q19)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("q,d", [(9, 2), (19, 3)])
def test_lattice_isotropy(q, d):
    c, w, opp = O.lattice(q)
    c = c[:, :d].astype(float)
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.allclose(np.einsum("i,ia->a", w, c), 0.0, atol=1e-16)
    # second moment: c_s^2 delta_ab with c_s^2 = 1/3
    assert np.allclose(np.einsum("i,ia,ib->ab", w, c, c), np.eye(d) / 3.0, atol=1e-15)
    # third moment vanishes, fourth is c_s^4 (d_ab d_cd + d_ac d_bd + d_ad d_bc)
    assert np.allclose(np.einsum("i,ia,ib,ic->abc", w, c, c, c), 0.0, atol=1e-16)
    I = np.eye(d)
    iso4 = (np.einsum("ab,cd->abcd", I, I) + np.einsum("ac,bd->abcd", I, I)
            + np.einsum("ad,bc->abcd", I, I)) / 9.0
    assert np.allclose(np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c), iso4, atol=1e-15)
    for i in range(q):
        assert np.array_equal(c[opp[i]], -c[i])
    assert len({tuple(v) for v in c}) == q


# --------------------------------------------------------------------------
# Kn and Eq. (1)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("tau,nx", [(0.51, 400), (0.8, 100), (2.0, 1200), (1.0, 256)])
def test_knudsen_is_mean_free_path_over_length(tau, nx):
    # Kinetic theory: mu = rho nu, p = rho R T, lambda = (mu/p) sqrt(pi R T / 2).
    # Lattice units: R T = c_s^2 = 1/3 and nu = c_s^2 (tau - 1/2)  (Eq. 1).
    RT = 1.0 / 3.0
    nu = RT * (tau - 0.5)
    lam = nu / RT * math.sqrt(math.pi * RT / 2.0)
    assert O.knudsen(tau, nx) == pytest.approx(lam / nx, rel=1e-14)


# --------------------------------------------------------------------------
# Exact invariants of one step
# --------------------------------------------------------------------------

@pytest.mark.parametrize("shape", [(9, 17), (4, 6, 11)])
def test_rest_state_is_fixed_point(shape):
    mask = _random_mask(shape, 0.25, 3)
    f = O.init(mask, 1.0, 1.0)
    q = f.shape[-1]
    _, w, _ = O.lattice(q)
    g = O.run(mask, f, 0.73, 1.0, 1.0, 60)
    fluid = ~mask.astype(bool)
    assert np.abs(g[fluid] - w).max() < 1e-15


@pytest.mark.parametrize("shape", [(7, 13), (5, 6, 9)])
@pytest.mark.parametrize("eq", [O.EQ_QUADRATIC, O.EQ_LINEAR])
def test_closed_box_conserves_mass(shape, eq):
    # Solid end columns: no pressure boundary acts; bounce-back and the mirror
    # planes each send every population to exactly one slot, and BGK keeps rho.
    mask = _random_mask(shape, 0.2, 5, open_x_ends=False)
    mask[..., 0] = 1
    mask[..., -1] = 1
    f = _random_state(mask, 11)
    m0 = f.sum()
    g = f
    for _ in range(25):
        g = O.step(mask, g, 0.9, 1.0, 1.0, eq)
    assert abs(g.sum() - m0) / m0 < 1e-14


def _moments(f, c):
    rho = f.sum(-1)
    j = np.einsum("...i,ia->...a", f, c.astype(float))
    return rho, j


def _feq(rho, j, c, w):
    cj = np.einsum("...a,ia->...i", j, c.astype(float))
    u = j / rho[..., None]
    cu = cj / rho[..., None]
    uu = (u * u).sum(-1)[..., None]
    return w * rho[..., None] * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * uu)


@pytest.mark.parametrize("shape", [(6, 9), (4, 5, 8)])
def test_zou_he_defining_equations(shape):
    """At inlet/outlet fluid nodes: rho is imposed, transverse momentum is zero,
    and the non-equilibrium part bounces back along the normal (the closure that
    defines the Zou & He condition).  BGK keeps rho and j and scales the
    non-equilibrium part uniformly, so all three hold after collision too."""
    mask = _random_mask(shape, 0.0, 1)
    q = 9 if mask.ndim == 2 else 19
    c, w, opp = O.lattice(q)
    f = _random_state(mask, 21)
    rho_in, rho_out = 1.003, 0.998
    g = O.step(mask, f, 0.77, rho_in, rho_out)
    rho, j = _moments(g, c)
    feq = _feq(rho, j, c, w)
    ex = [i for i in range(q) if tuple(c[i]) == (1, 0, 0)][0]
    for x, r_imp in ((0, rho_in), (-1, rho_out)):
        assert np.allclose(rho[..., x], r_imp, rtol=0, atol=2e-15)
        assert np.abs(j[..., x, 1:]).max() < 2e-15
        neq = g[..., x, :] - feq[..., x, :]
        assert np.abs(neq[..., ex] - neq[..., opp[ex]]).max() < 2e-15


def test_hand_stepped_4x4_inlet():
    """All-fluid 4x4 at uniform rest, rho_in = 1 + eps: worked by hand."""
    eps, tau = 1e-3, 0.8
    mask = np.zeros((4, 4), np.uint8)
    _, w, _ = O.lattice(9)
    f = np.broadcast_to(w, (4, 4, 9)).copy()
    g = O.step(mask, f, tau, 1.0 + eps, 1.0)
    # interior columns and the outlet (rho_out = 1, inflow zero) stay at rest
    assert np.abs(g[:, 1:, :] - w).max() < 5e-16
    # inlet: rho u_x = eps; f1 = 1/9 + 2 eps/3; f5 = f8 = 1/36 + eps/6; others w
    pre = w.copy()
    pre[1] = 1 / 9 + 2 * eps / 3
    pre[5] = 1 / 36 + eps / 6
    pre[8] = 1 / 36 + eps / 6
    rho = 1.0 + eps
    u = eps / rho
    cx = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1], float)
    feq = w * rho * (1 + 3 * cx * u + 4.5 * cx * cx * u * u - 1.5 * u * u)
    post = pre - (pre - feq) / tau
    for y in range(4):
        assert np.abs(g[y, 0] - post).max() < 5e-16


def test_hand_stepped_streaming_slots():
    """Which slot each population comes from, enumerated by hand on a 4x4 grid
    with one interior solid and one wall-row solid.  With tau huge, collision is
    the identity to ~1e-15, so each value identifies its source slot."""
    mask = np.zeros((4, 4), np.uint8)
    mask[1, 2] = 1  # (x=2, y=1)
    mask[0, 3] = 1  # (x=3, y=0) on the bottom row
    f = np.zeros((4, 4, 9))
    for y in range(4):
        for x in range(4):
            for i in range(9):
                f[y, x, i] = 1.0 + 1e-3 * ((y * 4 + x) * 9 + i)
    f[mask.astype(bool)] = 0.0
    g = O.step(mask, f, 1e15, 1.0, 1.0)
    tag = lambda x, y, i: f[y, x, i]  # noqa: E731
    cases = [
        # (x, y, i) <- source slot, derived from the pull rule
        ((1, 1, 1), (0, 1, 1)),   # plain streaming
        ((1, 1, 3), (1, 1, 1)),   # from (2,1): solid -> bounce back f*_1 at d
        ((1, 1, 7), (2, 2, 7)),
        ((1, 1, 6), (2, 0, 6)),
        ((1, 0, 2), (1, 0, 4)),   # from (1,-1): mirror onto row 0, dir 2 -> 4
        ((1, 0, 5), (0, 0, 8)),   # from (0,-1): mirror, (1,1) -> (1,-1)
        ((1, 0, 6), (2, 0, 7)),   # from (2,-1): mirror, (-1,1) -> (-1,-1)
        ((2, 0, 4), (2, 0, 2)),   # from (2,1): solid -> bounce back
        ((2, 0, 6), (2, 0, 8)),   # from (3,-1): mirrored source (3,0) solid -> bounce back
        ((1, 2, 8), (0, 3, 8)),
        ((1, 2, 6), (1, 2, 8)),   # from (2,1): solid -> bounce back
        ((1, 2, 2), (1, 1, 2)),
        ((2, 3, 4), (2, 3, 2)),   # top wall mirror
        ((2, 3, 7), (3, 3, 6)),
        ((2, 3, 8), (1, 3, 5)),
        ((2, 2, 4), (2, 3, 4)),   # from (2,3): fluid
    ]
    for (x, y, i), (sx, sy, si) in cases:
        assert abs(g[y, x, i] - tag(sx, sy, si)) < 1e-9, ((x, y, i), (sx, sy, si))


# --------------------------------------------------------------------------
# Specular symmetry planes (Sec. 2, Fig. 1)
# --------------------------------------------------------------------------

def test_mirror_plane_equals_doubled_domain_2d():
    mask = _random_mask((6, 14), 0.25, 8)
    stacked = np.concatenate([mask, mask[::-1]], axis=0)
    args = (0.85, 1.002, 1.0)
    a = O.run(mask, O.init(mask, 1.002, 1.0), *args, 40)
    b = O.run(stacked, O.init(stacked, 1.002, 1.0), *args, 40)
    assert np.abs(b[:6] - a).max() < 1e-14


def test_mirror_planes_equal_doubled_domain_3d():
    mask = _random_mask((3, 4, 9), 0.2, 9)
    ys = np.concatenate([mask, mask[:, ::-1]], axis=1)
    zs = np.concatenate([mask, mask[::-1]], axis=0)
    args = (0.9, 1.002, 1.0)
    a = O.run(mask, O.init(mask, 1.002, 1.0), *args, 20)
    by = O.run(ys, O.init(ys, 1.002, 1.0), *args, 20)
    bz = O.run(zs, O.init(zs, 1.002, 1.0), *args, 20)
    assert np.abs(by[:, :4] - a).max() < 1e-14
    assert np.abs(bz[:3] - a).max() < 1e-14


def test_flipped_mask_flips_field():
    mask = _random_mask((9, 20), 0.3, 12)
    args = (0.7, 1.001, 1.0)
    a = O.run(mask, O.init(mask, 1.001, 1.0), *args, 60)
    fl = mask[::-1].copy()
    b = O.run(fl, O.init(fl, 1.001, 1.0), *args, 60)
    ra, uxa, uya = O.fields(mask, a)
    rb, uxb, uyb = O.fields(fl, b)
    # rounding of populations ~0.1 in FP64 sets the floor for velocities ~1e-5
    umax = np.abs(uxa).max()
    assert np.abs(rb[::-1] - ra).max() < 1e-14
    assert np.abs(uxb[::-1] - uxa).max() < 1e-9 * umax
    assert np.abs(uyb[::-1] + uya).max() < 1e-9 * umax


# --------------------------------------------------------------------------
# Bounce-back + Darcy: exact discrete channel solution
# --------------------------------------------------------------------------

def _channel_exact_k(h, tau):
    """Exact steady solution of pressure-driven BGK flow between halfway
    bounce-back walls with the linear equilibrium, derived by hand.  Away from
    the inlet/outlet the state is f_i = a_i(y) + beta w_i x (beta = d rho/dx);
    the streaming equations force non-equilibrium parts n_1 = -beta w_1 tau,
    n_5 = p + q s, n_7 = -p + q s (s = y - y_c), and the zero-momentum condition
    on them fixes p = beta tau / 18 and U'' = beta/(3 nu).  Bounce-back at
    y = 1/2 then fixes the wall value, giving the row-mean momentum
        <U> = alpha (h^2 - 1 + 8 (tau - 1/2)^2) / 12,  alpha = -beta/(3 nu),
    i.e. k = nu <U> / (-c_s^2 beta) = (h^2 - 1 + 8 (tau - 1/2)^2) / 12."""
    return (h * h - 1 + 8 * (tau - 0.5) ** 2) / 12.0


@pytest.mark.parametrize("h,tau", [(8, 0.8), (8, 1.0), (16, 0.8), (12, 1.3)])
def test_channel_matches_exact_discrete_solution(h, tau):
    ny, nx = h + 2, 6 * h
    mask = np.zeros((ny, nx), np.uint8)
    mask[0] = mask[-1] = 1
    drho = 1e-3
    f = O.init(mask, 1 + drho, 1.0)
    g, rc, steps, res = O.run_to_steady(mask, f, tau, 1 + drho, 1.0, 1e-12, 200000,
                                        eq=O.EQ_LINEAR)
    assert rc == 0
    rho, ux, _ = O.fields(mask, g)
    xm = nx // 2
    j = (rho * ux)[1:-1, xm]
    beta = (rho[1:-1, xm + h // 2] - rho[1:-1, xm - h // 2]).mean() / (2 * (h // 2))
    nu = (tau - 0.5) / 3.0
    k_local = nu * j.mean() / (-beta / 3.0)
    assert k_local == pytest.approx(_channel_exact_k(h, tau), rel=1e-9)
    # the profile across the channel is an exact parabola
    y = np.arange(1, h + 1) - (h + 1) / 2.0
    A = np.vstack([np.ones(h), y * y]).T
    coef, *_ = np.linalg.lstsq(A, j, rcond=None)
    assert np.abs(A @ coef - j).max() < 1e-9 * np.abs(j).max()
    assert coef[1] == pytest.approx(beta / (3 * nu) / 2.0, rel=1e-8)
    # the Darcy permeability of the whole domain (superficial average, L = N_x - 1)
    # equals the channel value up to the short inlet/outlet transition
    k_darcy = O.permeability(mask, g, tau, 1 + drho, 1.0)
    assert k_darcy * ny / h == pytest.approx(_channel_exact_k(h, tau), rel=2e-3)


def test_plates_3d_match_exact_discrete_solution():
    """D3Q19 between two bounce-back plates with specular z faces: the flow is
    z-invariant and D3Q19 projects onto D2Q9 weights, so the 2D closed form holds."""
    h, tau = 8, 0.9
    nz, ny, nx = 3, h + 2, 6 * h
    mask = np.zeros((nz, ny, nx), np.uint8)
    mask[:, 0] = mask[:, -1] = 1
    drho = 1e-3
    f = O.init(mask, 1 + drho, 1.0)
    g, rc, _, _ = O.run_to_steady(mask, f, tau, 1 + drho, 1.0, 1e-12, 200000, eq=O.EQ_LINEAR)
    assert rc == 0
    rho, ux, _, uz = O.fields(mask, g)
    assert np.abs(uz).max() < 1e-15
    xm = nx // 2
    j = (rho * ux)[1, 1:-1, xm]
    beta = (rho[1, 1:-1, xm + h // 2] - rho[1, 1:-1, xm - h // 2]).mean() / (2 * (h // 2))
    k_local = (tau - 0.5) / 3.0 * j.mean() / (-beta / 3.0)
    assert k_local == pytest.approx(_channel_exact_k(h, tau), rel=1e-9)


# --------------------------------------------------------------------------
# Steady state: linearity (Sec. 2, 3D discussion) and flux invariance
# --------------------------------------------------------------------------

def test_percolates_false_on_blocked_masks():
    """A full solid column (2D) or plane (3D) across the flow cuts every path,
    as does an all-solid interior; an open channel percolates."""
    m = np.zeros((6, 9), np.uint8)
    assert O.percolates(m)
    m[:, 4] = 1
    assert not O.percolates(m)
    m3 = np.zeros((3, 4, 7), np.uint8)
    assert O.percolates(m3)
    m3[:, :, 3] = 1
    assert not O.percolates(m3)
    m = np.ones((5, 8), np.uint8)
    m[:, 0] = 0  # fluid only in the inlet column
    assert not O.percolates(m)
    m[:, -1] = 0  # and in the outlet column, with solid between
    assert not O.percolates(m)


def test_percolates_follows_the_lattice_links():
    """Connectivity is along lattice links: a 2D path of diagonal steps only
    connects (D2Q9 has the diagonals); in 3D an edge contact connects (D3Q19
    has the 12 edge directions) but a corner-only contact does not."""
    m = np.array([[0, 1, 0, 1],
                  [1, 0, 1, 0]], np.uint8)
    assert O.percolates(m)
    m3 = np.ones((2, 2, 2), np.uint8)
    m3[0, 0, 0] = 0
    m3[1, 1, 1] = 0  # (x, y, z) -> (x+1, y+1, z+1): corner only
    assert not O.percolates(m3)
    m3 = np.ones((2, 2, 2), np.uint8)
    m3[0, 0, 0] = 0
    m3[0, 1, 1] = 0  # (x, y) -> (x+1, y+1) in one z plane: an edge link
    assert O.percolates(m3)


@pytest.mark.parametrize("dim", [2, 3])
def test_percolates_matches_connected_component_labelling(dim):
    """Brute force against scipy's connected-component labelling with the
    lattice's neighbourhood (8 in 2D; 18 in 3D: faces and edges, no corners)
    on random masks near the percolation threshold."""
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(40 + dim)
    if dim == 2:
        structure = np.ones((3, 3), bool)
        shape, ps = (7, 11), (0.4, 0.5, 0.6)
    else:
        structure = np.ones((3, 3, 3), bool)
        for c in ((0, 0, 0), (0, 0, 2), (0, 2, 0), (0, 2, 2), (2, 0, 0), (2, 0, 2), (2, 2, 0), (2, 2, 2)):
            structure[c] = False
        shape, ps = (4, 5, 8), (0.5, 0.6, 0.7)
    seen = set()
    for p in ps:
        for _ in range(30):
            m = (rng.random(shape) < p).astype(np.uint8)
            lab, _ = ndimage.label(m == 0, structure=structure)
            a, b = set(lab[..., 0].ravel()) - {0}, set(lab[..., -1].ravel()) - {0}
            want = bool(a & b)
            seen.add(want)
            assert O.percolates(m) == want
    assert seen == {True, False}


def _porous(shape, seed):
    m, _ = O.qsgs(shape, seed, 0.05, 0.75)
    assert O.percolates(m)
    return m


def test_linear_equilibrium_k_independent_of_driving():
    mask = _porous((14, 36), 4)
    ks = []
    for drho in (1e-3, 1e-2, 5e-2):
        f = O.init(mask, 1 + drho, 1.0)
        g, rc, _, _ = O.run_to_steady(mask, f, 0.8, 1 + drho, 1.0, 1e-11, 300000,
                                      eq=O.EQ_LINEAR)
        assert rc == 0
        ks.append(O.permeability(mask, g, 0.8, 1 + drho, 1.0))
    assert max(ks) / min(ks) - 1 < 1e-7


def test_steady_link_flux_is_x_independent():
    mask = _porous((16, 40), 7)
    f = O.init(mask, 1.0005, 1.0)
    g, rc, _, _ = O.run_to_steady(mask, f, 0.8, 1.0005, 1.0, 1e-11, 300000)
    assert rc == 0
    J = O.link_flux(mask, g)
    assert (J.max() - J.min()) / abs(J.mean()) < 1e-7
    # and the link flux equals the node-average flux times the cross-section
    assert J.mean() == pytest.approx(O.mean_jx(mask, g) * mask.size / mask.shape[1], rel=1e-3)


def test_rescaled_geometry_keeps_physical_permeability():
    """Eq. (3): the same geometry at twice the resolution has k_lattice about
    4x larger, i.e. the same physical k = k_lattice dx^2 (up to discretisation)."""
    mask = _porous((12, 30), 2)
    fine = np.repeat(np.repeat(mask, 2, 0), 2, 1)
    ks = []
    for m in (mask, fine):
        f = O.init(m, 1.0005, 1.0)
        g, rc, _, _ = O.run_to_steady(m, f, 0.8, 1.0005, 1.0, 1e-9, 300000, eq=O.EQ_LINEAR)
        ks.append(O.permeability(m, g, 0.8, 1.0005, 1.0))
    assert 0.75 < ks[1] / (4 * ks[0]) < 1.25


# --------------------------------------------------------------------------
# splitmix64 and QSGS (Sec. 2, "randomly generated quartet structure")
# --------------------------------------------------------------------------

def test_splitmix64_published_vector():
    want = _golden_ints("splitmix64_seed1234567.txt")
    got = [O.splitmix64(1234567, n) for n in range(1, 6)]
    assert got == want


def test_qsgs_hash_is_uniform():
    hs = np.array([O.qsgs_hash(99, 3, c, 5) for c in range(20000)], float) / 2**32
    assert abs(hs.mean() - 0.5) < 5 * math.sqrt(1 / 12 / 20000)
    assert abs((hs < 0.2).mean() - 0.2) < 5 * math.sqrt(0.16 / 20000)


def test_qsgs_paper_porosities_exact():
    with open(os.path.join(GOLDEN, "paper_porosities.txt")) as fh:
        rows = [l.split() for l in fh if l.strip() and not l.startswith("#")]
    for nx, ny, phi, fluid in rows:
        m, it = O.qsgs((int(ny), int(nx)), 1, 0.02, float(phi))
        assert int((m == 0).sum()) == int(fluid)
        assert it >= 1


@pytest.mark.parametrize("shape", [(50, 100), (24, 20, 16)])
def test_qsgs_growth_rule(shape):
    seed, core_p = 17, 0.02
    m, it = O.qsgs(shape, seed, core_p, 0.74)
    N = m.size
    assert int(m.sum()) == int(math.floor(0.26 * N + 0.5))
    assert np.array_equal(m, O.qsgs(shape, seed, core_p, 0.74)[0])
    assert not np.array_equal(m, O.qsgs(shape, seed + 1, core_p, 0.74)[0])
    thr = math.floor(core_p * 2**32)
    flat = m.reshape(-1)
    core = np.array([O.qsgs_hash(seed, 0, c, 0) < thr for c in range(N)])
    assert np.all(flat[core] == 1)  # cores stay solid (S exceeds the core count)
    ncore = core.sum()
    assert abs(ncore - core_p * N) < 5 * math.sqrt(N * core_p * (1 - core_p))
    # every grown cell touches another solid cell in the final mask
    pad = np.pad(m, 1)
    nb = np.zeros_like(m, dtype=int)
    d = m.ndim
    for off in np.ndindex(*(3,) * d):
        if all(o == 1 for o in off):
            continue
        sl = tuple(slice(o, o + s) for o, s in zip(off, m.shape))
        nb += pad[sl]
    grown = (flat == 1) & ~core
    assert np.all(nb.reshape(-1)[grown] > 0)


def test_qsgs_degenerate_cases():
    m, _ = O.qsgs((8, 16), 5, 0.02, 1.0)
    assert m.sum() == 0
    m, _ = O.qsgs((8, 16), 5, 0.5, 0.0)
    assert m.sum() == 128
    # every cell a core candidate: exactly the S smallest draws are kept
    m, it = O.qsgs((8, 16), 5, 1.0, 0.5)
    assert it == 0 and m.sum() == 64
    h = np.array([O.qsgs_hash(5, 0, c, 0) for c in range(128)])
    keep = np.argsort(h, kind="stable")[:64]
    want = np.zeros(128, np.uint8)
    want[keep] = 1
    assert np.array_equal(m.reshape(-1), want)


@pytest.mark.parametrize("shape", [(5, 7), (4, 5, 6)])
@pytest.mark.parametrize("eq", [O.EQ_QUADRATIC, O.EQ_LINEAR])
def test_equilibrium_moments(shape, eq):
    """With tau = 1 the post-collision state is exactly f_eq(rho, j).  Its
    moments define the equilibrium: sum f = rho, sum c f = j and the momentum
    flux sum c c f = rho c_s^2 I + j j / rho (quadratic) or rho c_s^2 I (linear)."""
    mask = _random_mask(shape, 0.0, 1)
    q = 9 if mask.ndim == 2 else 19
    c, w, _ = O.lattice(q)
    d = mask.ndim
    f = _random_state(mask, 4, amp=0.2)
    g = O.step(mask, f, 1.0, 1.0, 1.0, eq)
    cf = c[:, :d].astype(float)
    rho = g.sum(-1)
    j = np.einsum("...i,ia->...a", g, cf)
    pi = np.einsum("...i,ia,ib->...ab", g, cf, cf)
    want = rho[..., None, None] * np.eye(d) / 3.0
    if eq == O.EQ_QUADRATIC:
        want = want + np.einsum("...a,...b->...ab", j, j) / rho[..., None, None]
    # interior nodes only (x = 0 and N_x - 1 carry the pressure boundary)
    assert np.abs((pi - want)[..., 1:-1, :, :]).max() < 1e-15


@pytest.mark.parametrize("dim", [2, 3])
def test_qsgs_growth_probabilities(dim):
    """From isolated single solid cells, each neighbour becomes a candidate with
    the growth probability of its class: D_face, D_face/2 (3D edges),
    D_face/4 (2D diagonals, 3D corners)."""
    d_face = 0.2
    if dim == 2:
        shape, step = (120, 120), 4
    else:
        shape, step = (40, 40, 40), 4
    start = np.zeros(shape, np.uint8)
    centres = tuple(slice(1, s - 1, step) for s in shape)
    start[centres] = 1
    cand = O.qsgs_grow_once(start, 31, 1, d_face)
    idx = np.argwhere(start == 1)
    counts = {}
    for off in np.ndindex(*(3,) * dim):
        o = np.array(off) - 1
        k = int(np.abs(o).sum())
        if k == 0:
            continue
        nb = idx + o
        ok = np.all((nb >= 0) & (nb < np.array(shape)), axis=1)
        vals = cand[tuple(nb[ok].T)]
        n, s = counts.get(k, (0, 0))
        counts[k] = (n + len(vals), s + int(vals.sum()))
    want = {1: d_face, 2: d_face / 2 if dim == 3 else d_face / 4, 3: d_face / 4}
    for k, (n, s) in counts.items():
        p = want[k]
        assert abs(s / n - p) < 5 * math.sqrt(p * (1 - p) / n), (k, s / n, p)


def test_mass_flow_rate_is_unique_with_boxed_in_boundary_node():
    """A fluid node of the inlet column boxed in by solid keeps whatever momentum
    it starts with (the pressure condition alone fixes it, no flow reaches it),
    but it is on no through-path: the permeability from the mass flow rate
    through the cross-section planes must not depend on the initial state."""
    m = np.zeros((12, 30), np.uint8)
    m[0] = m[-1] = 1
    m[5, 0] = m[7, 0] = 1
    m[5:8, 1] = 1
    tau, dr = 0.8, 1e-3
    f0 = O.init(m, 1 + dr, 1.0)
    f1 = f0 * (1 + 0.01 * np.random.default_rng(5).standard_normal(f0.shape))
    f1[m.astype(bool)] = 0
    ks, jx6 = [], []
    for f in (f0, f1):
        g, rc, _, _ = O.run_to_steady(m, f, tau, 1 + dr, 1.0, 1e-12, 400000)
        assert rc == 0
        ks.append(O.permeability(m, g, tau, 1 + dr, 1.0))
        rho, ux, _ = O.fields(m, g)
        jx6.append(rho[6, 0] * ux[6, 0])
    assert abs(jx6[1] - jx6[0]) > 1e-5          # the boxed-in node remembers its start
    assert ks[1] == pytest.approx(ks[0], rel=1e-5)  # the mass flow rate does not


# ---------------------------------------------------------------------------
# Two-relaxation-time collision (the multi-relaxation direction of Sec. 2)
# ---------------------------------------------------------------------------

def test_trt_with_equal_times_is_bgk():
    """TRT relaxes the even and odd parts of f - f_eq separately; with
    tau_minus = tau it must reproduce BGK (the two are separate code paths)."""
    rng = np.random.default_rng(3)
    for q, shape in ((9, (9, 17)), (19, (4, 5, 11))):
        mask = (rng.random(shape) < 0.25).astype(np.uint8)
        w = O.lattice(q)[1]
        f = w * (1 + 0.05 * rng.standard_normal(mask.shape + (q,)))
        f[mask.astype(bool)] = 0
        for eq in (O.EQ_QUADRATIC, O.EQ_LINEAR):
            a = O.step(mask, f, 0.8, 1.001, 1.0, eq)
            b = O.step(mask, f, 0.8, 1.001, 1.0, eq, tau_m=0.8)
            assert np.abs(a - b).max() < 1e-15


def test_trt_conserves_mass_and_keeps_the_rest_state():
    """Collision invariants: in a closed box TRT conserves mass for any pair of
    times, and the rest equilibrium stays a fixed point."""
    rng = np.random.default_rng(5)
    mask = np.zeros((10, 14), np.uint8)
    mask[0] = mask[-1] = 1
    mask[:, 0] = mask[:, -1] = 1
    w = O.lattice(9)[1]
    f = w * (1 + 0.05 * rng.standard_normal(mask.shape + (9,)))
    f[mask.astype(bool)] = 0
    g = O.run(mask, f, 0.7, 1.0, 1.0, 25, tau_m=1.9)
    assert g.sum() == pytest.approx(f.sum(), rel=1e-13)
    m1 = np.zeros((3, 5), np.uint8)
    rest = O.init(m1, 1.0, 1.0)
    out = O.run(m1, rest, 0.9, 1.0, 1.0, 10, tau_m=0.6)
    assert np.abs(out - rest).max() < 1e-15


@pytest.mark.parametrize("h", [8, 12])
@pytest.mark.parametrize("tau", [0.6, 0.9, 1.5])
def test_trt_channel_k_depends_only_on_lambda(h, tau):
    """Pressure-driven channel with halfway bounce-back and the linear
    equilibrium.  The BGK solution k = (h^2 - 1 + 8 (tau - 1/2)^2)/12 depends
    on tau only through Lambda = (tau - 1/2)^2; TRT steady states depend on the
    two times only through Lambda = (tau - 1/2)(tau_minus - 1/2), so TRT gives
    k = (h^2 - 1 + 8 Lambda)/12 for every tau at fixed Lambda.  With the
    'magic' Lambda = 3/16 the wall sits at the half link independently of the
    viscosity."""
    lam = 3.0 / 16.0
    ny, nx = h + 2, 6 * h
    mask = np.zeros((ny, nx), np.uint8)
    mask[0] = mask[-1] = 1
    drho = 1e-3
    f = O.init(mask, 1 + drho, 1.0)
    g, rc, steps, res = O.run_to_steady(mask, f, tau, 1 + drho, 1.0, 1e-12, 400000,
                                        eq=O.EQ_LINEAR, tau_m=O.tau_minus(tau, lam))
    assert rc == 0
    rho, ux, _ = O.fields(mask, g)
    xm = nx // 2
    j = (rho * ux)[1:-1, xm]
    beta = (rho[1:-1, xm + h // 2] - rho[1:-1, xm - h // 2]).mean() / (2 * (h // 2))
    nu = (tau - 0.5) / 3.0
    k_local = nu * j.mean() / (-beta / 3.0)
    assert k_local == pytest.approx((h * h - 1 + 8 * lam) / 12.0, rel=1e-9)


def test_trt_porous_k_is_viscosity_independent_at_fixed_lambda():
    """On a porous QSGS domain the steady TRT permeability at fixed Lambda is
    the same for every tau (Stokes regime, linear equilibrium), while BGK's
    varies with tau."""
    mask, _ = O.qsgs((16, 32), 5, 0.02, 0.72)
    assert O.percolates(mask)
    drho = 1e-4
    ks, kb = [], []
    for tau in (0.7, 1.3):
        f = O.init(mask, 1 + drho, 1.0)
        g, rc, _, _ = O.run_to_steady(mask, f, tau, 1 + drho, 1.0, 1e-9, 600000, eq=O.EQ_LINEAR,
                                      tau_m=O.tau_minus(tau, 3.0 / 16.0))
        assert rc == 0
        ks.append(O.permeability(mask, g, tau, 1 + drho, 1.0))
        g, rc, _, _ = O.run_to_steady(mask, f, tau, 1 + drho, 1.0, 1e-9, 600000, eq=O.EQ_LINEAR)
        assert rc == 0
        kb.append(O.permeability(mask, g, tau, 1 + drho, 1.0))
    assert ks[0] == pytest.approx(ks[1], rel=1e-6)
    assert abs(kb[0] - kb[1]) > 1e-3 * abs(kb[0])


# ---------------------------------------------------------------------------
# Local pore size and local Knudsen number (Sec. 2)
# ---------------------------------------------------------------------------

def test_pore_distance_closed_forms():
    # 3-4-5: one solid node; the fluid node 3 along x and 4 along y is 5 away
    m = np.zeros((6, 8), np.uint8)
    m[0, 0] = 1
    d2 = O.pore_d2(m)
    assert d2[4, 3] == 25 and d2[0, 0] == 0 and d2[0, 1] == 1 and d2[1, 1] == 2
    assert d2[5, 7] == 5 * 5 + 7 * 7
    # no solid anywhere: infinite distance, zero local Kn
    e = np.zeros((3, 4), np.uint8)
    assert np.all(O.pore_d2(e) == np.uint32(2**32 - 1))
    h, kn = O.local_knudsen(e, 0.8)
    assert np.all(np.isinf(h)) and np.all(kn == 0)
    # 3D: the nearest solid of a corner node along the space diagonal
    c = np.zeros((4, 4, 4), np.uint8)
    c[3, 3, 3] = 1
    assert O.pore_d2(c)[0, 0, 0] == 27


@pytest.mark.parametrize("h", [1, 4, 7])
def test_channel_pore_size_and_local_kn(h):
    """Channel of h fluid rows between solid rows: the centre row's pore size
    is h (odd h) and its local Kn is sqrt(pi/6)(tau - 1/2)/h; every row's pore
    size is 2 (distance to the nearer wall) - 1."""
    tau = 0.9
    m = np.zeros((h + 2, 10), np.uint8)
    m[0] = m[-1] = 1
    hh, kn = O.local_knudsen(m, tau)
    for r in range(1, h + 1):
        dwall = min(r, h + 1 - r)
        assert np.all(hh[r] == 2 * dwall - 1)
    c = (h + 1) // 2
    if h % 2 == 1:
        assert np.all(hh[c] == h)
        assert np.allclose(kn[c], np.sqrt(np.pi / 6) * (tau - 0.5) / h, rtol=1e-15)
    assert np.all(hh[0] == 0) and np.all(kn[-1] == 0)


def test_pore_distance_is_the_minimum_over_solid_nodes():
    """Independent numpy restatement on a random mask: for every fluid node the
    squared distance equals the minimum over all solid nodes."""
    rng = np.random.default_rng(13)
    m = (rng.random((5, 7, 9)) < 0.15).astype(np.uint8)
    d2 = O.pore_d2(m)
    zs, ys, xs = np.nonzero(m)
    for (z, y, x) in zip(*np.nonzero(m == 0)):
        ref = ((zs - z) ** 2 + (ys - y) ** 2 + (xs - x) ** 2).min()
        assert d2[z, y, x] == ref


# ---------------------------------------------------------------------------
# Force-driven periodic flow: the 3D experiment of Sec. 2 (Eq. 2)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("eq", [0, 1])
def test_forced_all_fluid_box_gains_exactly_F_per_step(eq):
    """Fully periodic, no solid: the Guo forcing adds exactly F = rho_0 g to
    each node's post-collision momentum per step, and the flow stays uniform;
    mass is conserved."""
    m = np.zeros((4, 5), np.uint8)
    f = O.init(m, 1.0, 1.0)
    g = 1e-5
    for t in range(1, 4):
        f = O.run_forced(m, f, 0.8, g, 1, eq)
        rho, ux, uy = O.fields(m, f)
        assert (rho * ux).sum() == pytest.approx(t * m.size * g, rel=1e-12)
        assert np.ptp(ux) == 0 and np.abs(uy).max() < 1e-15
        assert rho.sum() == pytest.approx(m.size, rel=1e-14)


def test_forced_channel_slip_is_width_independent():
    """Between two bounce-back walls the bulk momentum balance makes the
    steady profile a parabola of curvature -g/nu, so the wall correction is
    the same for every width: k(h2) - k(h1) = (h2^2 - h1^2)/12 exactly, for
    each tau, with either equilibrium."""
    g = 1e-6
    for eq in (0, 1):
        for tau in (0.7, 1.2):
            ks = []
            for h in (6, 10):
                m = np.zeros((h + 2, 4), np.uint8)
                m[0] = m[-1] = 1
                f, rc, _, _ = O.run_forced_to_steady(m, O.init(m, 1.0, 1.0), tau, g, 1e-13, 400000, eq=eq)
                assert rc == 0
                ks.append(O.permeability_forced(m, f, tau, g) * (h + 2) / h)
            assert ks[1] - ks[0] == pytest.approx((100 - 36) / 12.0, rel=1e-9)


def test_forced_plates_3d_equal_the_2d_channel():
    """D3Q19 between two walls, periodic in x and z: the flow is z-invariant
    and D3Q19 projects onto the D2Q9 weights, so k equals the D2Q9 channel's."""
    h, tau, g = 6, 0.9, 1e-6
    m2 = np.zeros((h + 2, 4), np.uint8)
    m2[0] = m2[-1] = 1
    m3 = np.zeros((3, h + 2, 4), np.uint8)
    m3[:, 0] = m3[:, -1] = 1
    f2, rc2, _, _ = O.run_forced_to_steady(m2, O.init(m2, 1.0, 1.0), tau, g, 1e-11, 400000)
    f3, rc3, _, _ = O.run_forced_to_steady(m3, O.init(m3, 1.0, 1.0), tau, g, 1e-11, 400000)
    assert rc2 == 0 and rc3 == 0
    assert O.permeability_forced(m3, f3, tau, g) == pytest.approx(O.permeability_forced(m2, f2, tau, g),
                                                                 rel=1e-9)


def test_forced_k_is_force_independent_only_with_the_stokes_equilibrium():
    """Sec. 2's 3D finding (Fig. 5): with the linear (Stokes) equilibrium and
    a constant force density the whole update is linear in (f, g), so
    k = nu <u>/g does not depend on g; with the quadratic equilibrium inertia
    makes it depend on g."""
    mask, _ = O.qsgs((8, 10, 12), 4, 0.05, 0.75)
    tau = 0.8
    k = {}
    for eq in (0, 1):
        for g in (1e-6, 5e-4):
            f, rc, _, _ = O.run_forced_to_steady(mask, O.init(mask, 1.0, 1.0), tau, g, 1e-10, 100000, eq=eq)
            assert rc == 0
            k[eq, g] = O.permeability_forced(mask, f, tau, g)
    assert k[1, 1e-6] == pytest.approx(k[1, 5e-4], rel=1e-9)
    assert abs(k[0, 5e-4] - k[0, 1e-6]) > 1e-6 * abs(k[0, 1e-6])


def test_forced_step_without_force_equals_the_pressure_driven_bulk_step():
    """With g = 0 the force-driven step is the pressure-driven step away from
    the faces (same pull streaming, bounce-back and BGK): at nodes whose whole
    stencil and its sources lie inside the domain the two independent code
    paths agree exactly, from a random state, 2D and 3D."""
    rng = np.random.default_rng(17)
    for q, shape in ((9, (12, 20)), (19, (7, 8, 12))):
        mask = (rng.random(shape) < 0.2).astype(np.uint8)
        w = O.lattice(q)[1]
        f = w * (1 + 0.05 * rng.standard_normal(mask.shape + (q,)))
        f[mask.astype(bool)] = 0
        for eq in (0, 1):
            a = O.step_forced(mask, f, 0.8, 0.0, eq)
            b = O.step(mask, f, 0.8, 1.0, 1.0, eq)
            inner = (slice(1, -1),) * mask.ndim
            assert np.abs(a[inner] - b[inner]).max() < 1e-15


def test_forced_eq2_velocity_is_the_half_step_velocity():
    """All-fluid periodic box from rest: the post-collision momentum after t
    steps is t F; the fluid momentum of Guo's scheme is the pre-collision
    momentum (t - 1) F plus F/2, so k = nu <u>/g is exactly nu (t - 1/2)."""
    m = np.zeros((3, 4), np.uint8)
    tau, g = 0.9, 1e-5
    f = O.init(m, 1.0, 1.0)
    for t in range(1, 4):
        f = O.run_forced(m, f, tau, g, 1)
        assert O.permeability_forced(m, f, tau, g) == pytest.approx((tau - 0.5) / 3.0 * (t - 0.5), rel=1e-10)


@pytest.mark.parametrize("h", [6, 10])
@pytest.mark.parametrize("tau", [0.6, 1.2])
def test_forced_channel_closed_forms(h, tau):
    """Force-driven channel between bounce-back walls (periodic in x), linear
    equilibrium.  BGK reproduces the exact pressure-driven solution
    k = (h^2 - 1 + 8 (tau - 1/2)^2)/12 (a body force and a uniform pressure
    gradient drive the bulk alike).  TRT with Lambda = 3/16 gives the exact
    parabola u = g y (h - y)/(2 nu) with the walls half way between nodes; its
    mean over the h node rows is g (h^2 + 1/2)/(12 nu), so k = (h^2 + 1/2)/12
    for every tau."""
    g = 1e-6
    m = np.zeros((h + 2, 4), np.uint8)
    m[0] = m[-1] = 1
    f, rc, _, _ = O.run_forced_to_steady(m, O.init(m, 1.0, 1.0), tau, g, 1e-12, 400000, eq=O.EQ_LINEAR)
    assert rc == 0
    k = O.permeability_forced(m, f, tau, g) * (h + 2) / h
    assert k == pytest.approx((h * h - 1 + 8 * (tau - 0.5) ** 2) / 12.0, rel=1e-9)
    tm = O.tau_minus(tau, 3.0 / 16.0)
    f, rc, _, _ = O.run_forced_to_steady(m, O.init(m, 1.0, 1.0), tau, g, 1e-12, 400000, eq=O.EQ_LINEAR, tau_m=tm)
    assert rc == 0
    k = O.permeability_forced(m, f, tau, g) * (h + 2) / h
    assert k == pytest.approx((h * h + 0.5) / 12.0, rel=1e-9)


def test_forced_trt_with_equal_times_is_bgk():
    rng = np.random.default_rng(23)
    for q, shape in ((9, (7, 11)), (19, (4, 5, 9))):
        mask = (rng.random(shape) < 0.2).astype(np.uint8)
        w = O.lattice(q)[1]
        f = w * (1 + 0.05 * rng.standard_normal(mask.shape + (q,)))
        f[mask.astype(bool)] = 0
        for eq in (0, 1):
            a = O.step_forced(mask, f, 0.8, 1e-3, eq)
            b = O.step_forced(mask, f, 0.8, 1e-3, eq, tau_m=0.8)
            assert np.abs(a - b).max() < 1e-15
