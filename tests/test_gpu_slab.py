"""x-slabs of one domain on the GPU, through the C ABI: two and three slab
solvers in one process, advanced by the slab driver with a halo exchange
after every step (a cut inside a process is a copy through a device buffer).
The real columns must equal the whole-domain solver's bit for bit (the same
pull step on the same values; the whole-domain solver is run with pull steps
too), and the permeability from the observables summed over the slabs must
equal the whole domain's, and the FP64 oracle's within the FP32 tolerance."""
import numpy as np
import pytest

import oracle as O
from paper_1609_09685_gb300 import build, lbm, slabs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    lbm.load()


def _mask(dim):
    rng = np.random.default_rng(70 + dim)
    if dim == 2:
        m = (rng.random((37, 130)) < 0.3).astype(np.uint8)
    else:
        m = (rng.random((9, 12, 70)) < 0.3).astype(np.uint8)
    return m


@pytest.mark.parametrize("dim,parts", [(2, 2), (2, 3), (3, 2), (3, 3)])
def test_slabs_equal_the_whole_domain_bitwise(dim, parts):
    import torch
    mask = _mask(dim)
    tau, drho = 0.7, 1e-3
    nx = mask.shape[-1]
    create = lbm.lbm_create_domain if dim == 2 else lbm.lbm_create_domain_3d
    with create(mask, tau, drho, lbm.make_options(in_place_pairs=False)) as whole:
        lbm.lbm_step(whole, 25)
        f_whole = lbm.lbm_get_populations(whole, 0)
        k_whole, kn_whole = lbm.lbm_permeability(whole)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):  # the slabs and the driver's copies share this stream
        sl = [slabs.GpuSlab(mask, lo, hi, tau, drho) for lo, hi in slabs.split_columns(nx, parts)]
    try:
        with torch.cuda.stream(side):
            drv = slabs.SlabDriver(sl, 0, parts)
            drv.step(25)
        torch.cuda.synchronize()
        real = []
        for s in sl:
            f = lbm.lbm_get_populations(s.solver, 0)
            left, right = s.ghosts & 1, (s.ghosts >> 1) & 1
            real.append(f[..., left:f.shape[-2] - right, :])
        f_sl = np.concatenate(real, axis=mask.ndim - 1)
        assert np.array_equal(f_sl, f_whole)
        with torch.cuda.stream(side):
            k, kn, r = drv.observe()
    finally:
        for s in sl:
            s.close()
    assert k == pytest.approx(k_whole[0], rel=1e-6)
    assert kn == kn_whole[0]
    assert np.isfinite(r)
    k_o = O.permeability(mask, O.run(mask, O.init(mask, 1 + drho, 1.0), tau, 1 + drho, 1.0, 25), tau,
                         1 + drho, 1.0)
    assert k == pytest.approx(k_o, rel=1e-4)


def test_slab_arguments_and_refused_calls():
    mask = _mask(2)
    part = np.ascontiguousarray(mask[:, 0:40])
    with pytest.raises(lbm.LBMError):  # a cut needs a ghost column
        lbm.lbm_slab_create(part, 0.7, 1e-3, 0, 130, 0)
    with pytest.raises(lbm.LBMError):  # no cut at the global inlet
        lbm.lbm_slab_create(part, 0.7, 1e-3, 0, 130, 3)
    with lbm.lbm_slab_create(part, 0.7, 1e-3, 0, 130, 2) as s:
        with pytest.raises(lbm.LBMError):
            lbm.lbm_run_to_steady(s, 1e-9, 100)
        with pytest.raises(lbm.LBMError):
            lbm.lbm_permeability(s)
        with pytest.raises(lbm.LBMError):  # no neighbour on the left
            lbm.lbm_slab_halo_floats(s, 0)
        assert lbm.lbm_slab_halo_floats(s, 1) == 3 * int((part[:, 38] == 0).sum())
        assert lbm.lbm_slab_halo_floats(s, 1, incoming=True) == 3 * int((part[:, 39] == 0).sum())
