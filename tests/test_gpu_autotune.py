"""Launch configurations and the runtime autotuner, through the C ABI.

Every launch configuration -- block size, strip rows, the direct gather
step's row batch, the staged gather step's tile rows, the band gather step's
band rows, the fused L2-blocked pair's block size -- maps the same step
onto the GPU differently and must give bit-identical populations; the tuner
picks among them by CUDA-event timing on the solver's stream and caches the
choice per (device, lattice, size bucket, equilibrium, collision, kernel
sources)."""
import numpy as np
import pytest

import oracle as O
from paper_1609_09685_gb300 import build, lbm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    lbm.load()


def _batch(dim):
    rng = np.random.default_rng(21 + dim)
    if dim == 2:
        shapes = [(37, 130), (1, 70), (64, 96), (20, 33)]
    else:
        shapes = [(9, 12, 70), (5, 7, 33)]
    masks = [(rng.random(s) < 0.3).astype(np.uint8) for s in shapes]
    return masks, [0.55 + 0.2 * i for i in range(len(masks))], [1e-3] * len(masks)


def _run(masks, taus, drhos, launch=None, tune=None, steps=(7, 10)):
    opts = lbm.make_options()
    with lbm.lbm_batch_create(masks, taus, drhos, opts) as s:
        res = None
        if launch is not None:
            lbm.lbm_set_launch(s, **launch)
            want = dict(dict(tile_rows=0, band_rows=0, pair_block_mb=0), **launch)
            assert lbm.lbm_get_launch(s) == want
        if tune is not None:
            res = lbm.lbm_autotune(s, tune, 8)
        for n in steps:
            lbm.lbm_step(s, n)
        obs = lbm.lbm_step_observe(s, 3)
        return [lbm.lbm_get_populations(s, d) for d in range(len(masks))], obs, res


@pytest.mark.parametrize("dim", [2, 3])
def test_every_launch_configuration_is_bit_identical(dim):
    masks, taus, drhos = _batch(dim)
    ref, _, _ = _run(masks, taus, drhos)
    lo, hi = (2, 4) if dim == 2 else (1, 2)
    configs = [dict(block_threads=bt, strip_rows=sr, gather_batch=gb)
               for bt in (32, 64, 256) for sr in (1, 5, 16) for gb in (lo, hi)]
    if dim == 2:
        configs += [dict(block_threads=128, strip_rows=8, gather_batch=4, tile_rows=tr) for tr in (1, 2, 3, 4)]
        configs += [dict(block_threads=128, strip_rows=8, gather_batch=4, band_rows=br) for br in (1, 7, 64)]
    # fused pairs over blocks of 1 MB (several blocks on these masks only in 2D)
    configs += [dict(block_threads=128, strip_rows=sr, gather_batch=hi, pair_block_mb=1) for sr in (4, 8)]
    for cfg in configs:
        got, _, _ = _run(masks, taus, drhos, launch=cfg)
        for a, b in zip(ref, got):
            assert np.array_equal(a, b), cfg


def test_launch_configuration_is_validated():
    masks, taus, drhos = _batch(2)
    with lbm.lbm_batch_create(masks, taus, drhos) as s:
        for bad in (dict(block_threads=48, strip_rows=8, gather_batch=4), dict(block_threads=128, strip_rows=0,
                    gather_batch=4), dict(block_threads=128, strip_rows=8, gather_batch=3),
                    dict(block_threads=128, strip_rows=8, gather_batch=4, tile_rows=5),
                    dict(block_threads=128, strip_rows=8, gather_batch=4, band_rows=65),
                    dict(block_threads=128, strip_rows=8, gather_batch=4, tile_rows=2, band_rows=8),
                    dict(block_threads=128, strip_rows=8, gather_batch=4, pair_block_mb=5000)):
            with pytest.raises(lbm.LBMError):
                lbm.lbm_set_launch(s, **bad)
    masks3, taus3, drhos3 = _batch(3)
    with lbm.lbm_batch_create(masks3, taus3, drhos3) as s:
        with pytest.raises(lbm.LBMError):  # no staged gather step for D3Q19
            lbm.lbm_set_launch(s, 128, 8, 2, 2)
        with pytest.raises(lbm.LBMError):  # nor a band gather step
            lbm.lbm_set_launch(s, 128, 8, 2, 0, 8)


def test_time_steps_leaves_the_state_alone():
    masks, taus, drhos = _batch(2)
    with lbm.lbm_batch_create(masks, taus, drhos) as s:
        lbm.lbm_step(s, 5)
        before = [lbm.lbm_get_populations(s, d) for d in range(len(masks))]
        step0 = lbm.lbm_get_step(s)
        us = lbm.lbm_time_steps(s, 20)
        assert us > 0
        assert lbm.lbm_get_step(s) == step0
        for d, b in enumerate(before):
            assert np.array_equal(lbm.lbm_get_populations(s, d), b)


@pytest.mark.parametrize("dim", [2, 3])
def test_autotuned_solver_matches_the_default_and_is_no_slower(dim, tmp_path):
    masks, taus, drhos = _batch(dim)
    cache = str(tmp_path / "tune.json")
    ref, ref_obs, _ = _run(masks, taus, drhos)
    got, obs, res = _run(masks, taus, drhos, tune=cache)
    for a, b in zip(ref, got):
        assert np.array_equal(a, b)
    assert res["candidates"] >= 18 and not res["from_cache"]
    assert res["us_per_step"] <= res["us_per_step_default"]
    # the second solver of the same kind takes the cached choice
    with lbm.lbm_batch_create(masks, taus, drhos, lbm.make_options(autotune=True, tune_cache=cache)) as s:
        assert lbm.lbm_get_launch(s) == res["chosen"]
        key = lbm.lbm_tune_key(s)
    assert lbm.lbm_tune_cache_get(cache, key)[0] == res["chosen"]
    # observables come from the same populations; their sums are FP32 within
    # a strip, so another strip height regroups them at FP32 rounding
    np.testing.assert_allclose(obs, ref_obs, rtol=1e-5, atol=1e-12)


def test_autotune_on_a_force_driven_solver_reports_its_configuration():
    mask = O.qsgs((6, 8, 20), 3, 0.05, 0.75)[0]
    with lbm.lbm_batch_create_forced([mask], [0.9], [1e-4]) as s:
        res = lbm.lbm_autotune(s)
        assert res["candidates"] == 0 and res["chosen"] == lbm.lbm_get_launch(s)
