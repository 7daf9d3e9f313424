"""The warm-start network's convolution on the tcgen05 tensor cores
(lbm_nn_set_conv_impl(LBM_NN_CONV_TCGEN05)) against the FP64 reference
(oracle/nn_ref.py) and against the mma.sync path, through the C ABI.

Inputs and weights are rounded to bfloat16 once; the FP32 copy of the output
(an FP32 sum of at most 9 x 256 products) is compared at 1e-4 of the largest
magnitude, the bf16 output and the data gradient at 1e-2.  Shapes cover one
and nine taps, one and several 16-channel chunks, one and two 128-channel
output tiles, image rows shorter than, equal to and longer than the
128-pixel tile (ragged tails), and several images."""
import numpy as np
import pytest

import oracle as O
from oracle import nn_ref as R
from paper_1609_09685_gb300 import build, lbm

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    lbm.load()
    O.build()


@pytest.fixture()
def tcgen05():
    old = lbm.lbm_nn_get_conv_impl()
    lbm.lbm_nn_set_conv_impl(lbm.LBM_NN_CONV_TCGEN05)
    yield
    lbm.lbm_nn_set_conv_impl(old)


def _bf(a):
    r = R.bf16_round(a)
    return r, torch.tensor(r, dtype=torch.float32, device="cuda").to(torch.bfloat16).contiguous()


def _np(t):
    return t.float().cpu().numpy().astype(np.float64)


def _close(a, b, rel):
    scale = max(np.abs(b).max(), 1e-30)
    assert np.abs(a - b).max() <= rel * scale, (np.abs(a - b).max(), scale)


def _conv(xt, n, h, w, cin, wtt, bt, taps, cout, relu):
    y = torch.empty((n, h, w, cout), dtype=torch.bfloat16, device="cuda")
    y32 = torch.empty((n, h, w, cout), dtype=torch.float32, device="cuda")
    lbm.lbm_nn_conv_fwd(xt, n, h, w, cin, wtt, bt, taps, cout, relu, y, y32)
    return y, y32


@pytest.mark.parametrize("taps,cin,cout,shape", [
    (9, 16, 16, (1, 3, 9)),       # one chunk, one short row tile
    (1, 16, 16, (2, 4, 6)),
    (9, 32, 48, (1, 7, 130)),     # two chunks, ragged second tile
    (9, 128, 128, (2, 5, 256)),   # eight chunks, full tiles
    (9, 48, 144, (1, 3, 40)),     # two output-channel tiles (128 + 16)
    (1, 64, 32, (3, 2, 200)),
])
def test_tcgen05_conv_matches_reference_and_mma_sync(tcgen05, taps, cin, cout, shape):
    n, h, w = shape
    rng = np.random.default_rng(taps * 1000 + cin + cout)
    x, xt = _bf(rng.standard_normal((n, h, w, cin)))
    wt_, wtt = _bf(rng.standard_normal((taps, cout, cin)) * 0.2)
    b = rng.standard_normal(cout).astype(np.float32)
    bt = torch.tensor(b, device="cuda")
    y, y32 = _conv(xt, n, h, w, cin, wtt, bt, taps, cout, 1)
    lbm.lbm_nn_sync_status()
    ref = R.conv(x, wt_, b.astype(np.float64), relu=True)
    _close(_np(y32), ref, 1e-4)
    _close(_np(y), ref, 1e-2)
    # the data gradient runs the same kernel with flipped taps
    gy, gyt = _bf(rng.standard_normal((n, h, w, cout)))
    gx = torch.empty((n, h, w, cin), dtype=torch.bfloat16, device="cuda")
    flip = torch.empty((taps, cin, cout), dtype=torch.bfloat16, device="cuda")
    lbm.lbm_nn_conv_bwd_data(gyt, n, h, w, cout, wtt, taps, cin, flip, gx)
    lbm.lbm_nn_sync_status()
    _close(_np(gx), R.conv_dx(gy, wt_), 1e-2)
    # the same numbers as the mma.sync path, to FP32 summation order
    lbm.lbm_nn_set_conv_impl(lbm.LBM_NN_CONV_MMA_SYNC)
    y_ms, y32_ms = _conv(xt, n, h, w, cin, wtt, bt, taps, cout, 1)
    lbm.lbm_nn_set_conv_impl(lbm.LBM_NN_CONV_TCGEN05)
    _close(_np(y32), _np(y32_ms), 1e-5)


def test_conv_impl_switch_is_validated():
    assert lbm.lbm_nn_get_conv_impl() == lbm.LBM_NN_CONV_AUTO  # the default
    with pytest.raises(lbm.LBMError):
        lbm.lbm_nn_set_conv_impl(7)


def test_automatic_choice_gives_the_same_network_output():
    """A wide layer on a large image takes the tcgen05 path under the
    automatic choice; its output equals the forced tcgen05 path's bit for bit
    and the mma.sync path's to FP32 summation order."""
    rng = np.random.default_rng(8)
    n, h, w, cin, cout = 2, 32, 64, 32, 64
    x, xt = _bf(rng.standard_normal((n, h, w, cin)))
    _, wtt = _bf(rng.standard_normal((9, cout, cin)) * 0.2)
    bt = torch.zeros(cout, device="cuda")
    outs = {}
    old = lbm.lbm_nn_get_conv_impl()
    try:
        for impl in (lbm.LBM_NN_CONV_AUTO, lbm.LBM_NN_CONV_TCGEN05, lbm.LBM_NN_CONV_MMA_SYNC):
            lbm.lbm_nn_set_conv_impl(impl)
            outs[impl] = _np(_conv(xt, n, h, w, cin, wtt, bt, 9, cout, 0)[1])
        lbm.lbm_nn_sync_status()
    finally:
        lbm.lbm_nn_set_conv_impl(old)
    assert np.array_equal(outs[lbm.LBM_NN_CONV_AUTO], outs[lbm.LBM_NN_CONV_TCGEN05])
    _close(outs[lbm.LBM_NN_CONV_AUTO], outs[lbm.LBM_NN_CONV_MMA_SYNC], 1e-5)
