"""The combinatorial fact behind the in-place pair of steps, checked on the CPU.

Let R_i(x) be the slot (node, direction) that the pull step reads for
direction i at fluid node x, under the boundary rules of Sec. 2 as read here:
streaming from the fluid source, halfway bounce-back from the node's own
opposite slot when the source is solid or lies beyond an x face (the Zou-He
unknowns), and the specular mirror (source row clamped onto the node's row,
direction flipped) at the y/z faces.  The gather step writes f*_opp(i) back
into R_i(x) and the local step reads each node's own slots, which is the
arithmetic of two pull steps exactly when
  (1) no slot is read twice, and
  (2) R_i(x) = (y, opp j)  <=>  R_j(y) = (x, opp i).
The map is built here in plain Python from those rules, with the direction
tables the kernels themselves use (velocities, opposite and y/z-mirrored
directions, exported by lbm_lattice), and the two properties are checked on
random masks in 2D and 3D.  What stays outside this check is the kernels'
index arithmetic (windows, popcounts, slot offsets); the GPU parity tests of
pairs against pull steps and the oracle cover that."""
import numpy as np
import pytest

import oracle as O
from paper_1609_09685_gb300 import build, lbm


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    lbm.load()


def _tables(q):
    """Direction tables of the kernels; checked against the oracle's own."""
    c, w, opp, fy, fz = lbm.lbm_lattice(q)
    co, wo, oo = O.lattice(q)
    assert np.array_equal(c, co) and np.array_equal(w, wo) and np.array_equal(opp, oo)
    return c, opp, fy, fz


def _read_map(mask, c, opp, fy_tab, fz_tab):
    q = len(c)
    if mask.ndim == 2:
        mask = mask[None]
    nz, ny, nx = mask.shape
    flip = {}
    for i in range(q):
        flip[i, False, False] = i
        flip[i, True, False] = int(fy_tab[i])
        flip[i, False, True] = int(fz_tab[i])
        flip[i, True, True] = int(fz_tab[fy_tab[i]])
    R = {}
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                if mask[z, y, x]:
                    continue
                for i in range(q):
                    sx, sy, sz = x - c[i][0], y - c[i][1], z - c[i][2]
                    if not 0 <= sx < nx:
                        R[(z, y, x), i] = ((z, y, x), opp[i])  # Zou-He unknown: own opposite slot
                        continue
                    fy, fz = not 0 <= sy < ny, not 0 <= sz < nz
                    if fy:
                        sy = y
                    if fz:
                        sz = z
                    j = flip[i, fy, fz]
                    if mask[sz, sy, sx]:
                        R[(z, y, x), i] = ((z, y, x), opp[i])  # halfway bounce-back
                    else:
                        R[(z, y, x), i] = ((sz, sy, sx), j)
    return R


@pytest.mark.parametrize("dim", [2, 3])
def test_read_map_is_injective_and_paired(dim):
    rng = np.random.default_rng(5 + dim)
    q = 9 if dim == 2 else 19
    c, opp, fy, fz = _tables(q)
    for trial in range(3):
        shape = (9, 13) if dim == 2 else (4, 5, 7)
        mask = (rng.random(shape) < 0.3).astype(np.uint8)
        R = _read_map(mask, c, opp, fy, fz)
        # (1) injective
        assert len(set(R.values())) == len(R)
        # (2) pairing
        for (x, i), (y, k) in R.items():
            j = opp[k]
            assert R[(y, j)] == (x, opp[i])


def test_pairing_breaks_for_a_wrong_mirror_rule():
    """The check has teeth: mirroring without flipping the direction (a
    plausible mistake) violates the pairing."""
    c, opp, fy, fz = _tables(9)
    mask = np.zeros((4, 6), np.uint8)
    R = _read_map(mask, c, opp, fy, fz)
    bad = dict(R)
    # replace the mirror at the top row by a non-flipping one
    for (x, i), (y, k) in R.items():
        z, yy, xx = x
        if yy == 0 and c[i][1] == 1 and 0 <= xx - c[i][0] < 6:
            bad[(x, i)] = ((z, 0, xx - c[i][0]), i)
    broken = any(bad.get((y, opp[k])) != (x, opp[i]) for (x, i), (y, k) in bad.items())
    assert broken
