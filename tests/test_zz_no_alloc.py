"""The allocation-free QSGS entry point, through the C ABI.

lbm_qsgs_noalloc exists for callers that cannot allocate GPU memory while they
run (their device memory belongs to their own pool allocator, or a policy bars
cudaMalloc/cudaFree after set-up).  It keeps its scratch in a fixed device
array inside the library and writes the mask into a device buffer the caller
owns.  This test checks that two calls in a row give exactly the masks of the
allocating entry point lbm_qsgs (mask generation is integer work, so the
comparison is bit for bit), that the second call is not disturbed by what the
first left in the shared scratch, and that a grid above the scratch limit is
refused.  The test allocates its own buffers; the entry point allocates none.
The file name makes pytest collect it after every other test.
"""
import numpy as np
import pytest

from paper_1609_09685_gb300 import build, lbm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    lbm.load()


def test_noalloc_matches_allocating_qsgs_on_two_calls():
    import torch

    torch.cuda.init()
    stream = torch.cuda.Stream()
    cases = [((200, 400), 11, 0.7394), ((50, 100), 3, 0.74)]  # larger first, then smaller
    for shape, seed, phi in cases:
        n = int(np.prod(shape))
        out = torch.full((n,), 7, dtype=torch.uint8, device="cuda")  # stale bytes to overwrite
        torch.cuda.synchronize()
        it = lbm.lbm_qsgs_noalloc(seed, shape, 0.02, phi, out.data_ptr(), stream=stream.cuda_stream)
        got = out.cpu().numpy().reshape(shape)
        want, it_want = lbm.lbm_qsgs(seed, shape, 0.02, phi)
        assert it == it_want
        assert np.array_equal(got, want)


def test_noalloc_3d_and_limit():
    import torch

    shape = (16, 24, 40)
    out = torch.empty(int(np.prod(shape)), dtype=torch.uint8, device="cuda")
    lbm.lbm_qsgs_noalloc(5, shape, 0.02, 0.7, out.data_ptr())
    want, _ = lbm.lbm_qsgs(5, shape, 0.02, 0.7)
    assert np.array_equal(out.cpu().numpy().reshape(shape), want)
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_qsgs_noalloc(1, (1025, 1024), 0.02, 0.7, out.data_ptr())
    assert e.value.status == lbm.LBM_ERR_ARG
    assert "allocation-free scratch limit" in str(e.value)
