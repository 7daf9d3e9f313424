"""Failure detection without a GPU fault, through the C ABI.

* Allocator hook: a solver whose device memory comes from PyTorch's caching
  allocator computes exactly what a pool-backed solver computes and returns
  every block; an allocation that fails (injected by the hook returning NULL
  at the k-th call, for every k) makes creation return LBM_ERR_OOM after
  returning every block it had, and a failing scratch allocation after
  creation leaves the solver usable.
* Checked build: a window record corrupted on purpose (possible only in a
  build compiled with LBM_CHECKED) makes the next observation return
  LBM_ERR_INTERNAL; the checks skip every access the bad index would have
  made, so nothing outside the buffers is touched.
"""
import os

import numpy as np
import pytest

import oracle as O
from paper_1609_09685_gb300 import build, lbm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    lbm.load()


def _case():
    mask = O.qsgs((24, 70), 4, 0.02, 0.72)[0]
    return [mask, O.qsgs((12, 40), 5, 0.02, 0.7)[0]], [0.8, 1.1], [1e-3, 1e-3]


def _pops(s):
    return [lbm.lbm_get_populations(s, d) for d in range(s.n_domains)]


def test_torch_allocator_hook_gives_the_same_results_and_returns_every_block():
    import torch
    masks, taus, drhos = _case()
    with lbm.lbm_batch_create(masks, taus, drhos) as s:
        lbm.lbm_step(s, 9)
        ref = _pops(s)
    log = []
    with lbm.lbm_batch_create(masks, taus, drhos, lbm.make_options(allocator=lbm.torch_allocator(log=log))) as s:
        lbm.lbm_step(s, 9)
        got = _pops(s)
        lbm.lbm_local_knudsen(s, 0)  # scratch through the hook too
    torch.cuda.synchronize()
    for a, b in zip(ref, got):
        assert np.array_equal(a, b)
    alloc = [e[1] for e in log if e[0] == "alloc"]
    freed = [e[1] for e in log if e[0] == "free"]
    assert len(alloc) > 10 and sorted(alloc) == sorted(freed)


def test_injected_out_of_memory_at_every_allocation_of_creation():
    import torch
    masks, taus, drhos = _case()
    log = []
    with lbm.lbm_batch_create(masks, taus, drhos, lbm.make_options(allocator=lbm.torch_allocator(log=log))):
        n_create = sum(1 for e in log if e[0] == "alloc")
    for k in range(n_create):
        log = []
        opts = lbm.make_options(allocator=lbm.torch_allocator(fail_after=k, log=log))
        with pytest.raises(lbm.LBMError) as e:
            lbm.lbm_batch_create(masks, taus, drhos, opts)
        assert e.value.status == lbm.LBM_ERR_OOM, (k, str(e.value))
        torch.cuda.synchronize()
        alloc = sorted(x[1] for x in log if x[0] == "alloc")
        freed = sorted(x[1] for x in log if x[0] == "free")
        assert len(alloc) == k and alloc == freed, k


def test_injected_out_of_memory_after_creation_leaves_the_solver_usable():
    masks, taus, drhos = _case()
    log = []
    probe = lbm.make_options(allocator=lbm.torch_allocator(log=log))
    with lbm.lbm_batch_create(masks, taus, drhos, probe):
        n_create = sum(1 for e in log if e[0] == "alloc")
    with lbm.lbm_batch_create(masks, taus, drhos, lbm.make_options(
            allocator=lbm.torch_allocator(fail_after=n_create))) as s:
        with pytest.raises(lbm.LBMError) as e:
            lbm.lbm_time_steps(s, 4)
        assert e.value.status == lbm.LBM_ERR_OOM
        with pytest.raises(lbm.LBMError) as e:
            lbm.lbm_local_knudsen(s, 0)
        assert e.value.status == lbm.LBM_ERR_OOM
        lbm.lbm_step(s, 6)
        k, _ = lbm.lbm_permeability(s)
        assert np.all(np.isfinite(k))


def test_regular_build_refuses_the_fault_injection():
    masks, taus, drhos = _case()
    assert not lbm.lbm_build_checked()
    with lbm.lbm_batch_create(masks, taus, drhos) as s:
        with pytest.raises(lbm.LBMError) as e:
            lbm.lbm_debug_corrupt_window(s, 0, 0xF0000000)
        assert e.value.status == lbm.LBM_ERR_ARG


def test_checked_build_reports_a_corrupted_window_table():
    masks, taus, drhos = _case()
    with lbm.lbm_batch_create(masks, taus, drhos) as s:
        lbm.lbm_step(s, 8)
        ref = _pops(s)
    path = build.build(defines=("LBM_CHECKED",),
                       out=os.path.join(os.path.dirname(build.LIB), "liblbm_gb300_checked.so"))
    try:
        lbm.unload()
        lbm.load(path)
        assert lbm.lbm_build_checked()
        for pairs in (True, False):  # gather + local steps, and pull steps
            opts = lbm.make_options(in_place_pairs=pairs)
            with lbm.lbm_batch_create(masks, taus, drhos, opts) as s:
                lbm.lbm_step(s, 8)
                for a, b in zip(ref, _pops(s)):  # the checks do not change the arithmetic
                    assert np.array_equal(a, b)
                seg = 4  # row 1, segment 1 (x = 32 .. 63) of the first domain
                lbm.lbm_debug_corrupt_window(s, seg, 0xF0000000)
                lbm.lbm_step(s, 4)
                with pytest.raises(lbm.LBMError) as e:
                    lbm.lbm_step_observe(s, 1)
                assert e.value.status == lbm.LBM_ERR_INTERNAL
                assert "out of range" in str(e.value)
    finally:
        lbm.unload()
        lbm.load()
    assert not lbm.lbm_build_checked()
