"""polar_decode_noalloc: the decode for callers that cannot allocate device
memory (its alpha-stage scratch is a static device array instead of memory
taken with cudaMallocAsync). It must give exactly the bits polar_decode gives,
on consecutive calls that reuse the same static scratch.

Collected last on purpose (file name), so a stop at its first failure has
already run every other test."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1504_00353_gb300 import polar
from tests import _cases

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _noalloc(code, llr, out, stream):
    """Call the entry point through the C ABI with raw device pointers."""
    st = polar.lib().polar_decode_noalloc(code.handle, ctypes.c_void_p(llr.data_ptr()),
                                         ctypes.c_void_p(out.data_ptr()), llr.shape[0],
                                         ctypes.c_void_p(stream.cuda_stream))
    return st


@pytest.mark.parametrize("N,K,db,n", [(32768, 29492, 4.0, 700), (1024, 512, 2.5, 3000),
                                       (1 << 18, 220201, 3.5, 64)])
def test_noalloc_equals_decode_on_consecutive_calls(N, K, db, n):
    """Bits equal polar_decode's on two calls in a row. For N = 2^18 the
    launch's scratch (64 one-frame CTAs of about 0.9 MB each) is larger than the
    static array, so the entry point runs fewer CTAs than polar_decode does."""
    mask, d, llr = _cases.frames(N, K, db, n, seed=40, distinct=8 if N > 32768 else 48)
    code = polar.polar_code_create(N, K, mask)
    launch = polar.polar_code_get_launch(code, False, n)
    if N >= 32768:
        # this launch shape keeps alpha stages above the shared-memory cap in device scratch
        assert launch["scratch_bytes"] > 0
    if N == 1 << 18:
        assert launch["scratch_bytes"] > (32 << 20)  # the grid must shrink to fit the array
    stream = torch.cuda.current_stream()
    t = torch.from_numpy(llr).cuda()
    want = polar.polar_decode(code, t)
    torch.cuda.synchronize()
    outs = [torch.full_like(want, 0xA5) for _ in range(3)]
    assert _noalloc(code, t, outs[0], stream) == 0  # first call on this device: set-up
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for out in outs[1:]:
        assert _noalloc(code, t, out, stream) == 0
        torch.cuda.synchronize()
        polar.polar_code_check(code)
    # the calls took no device memory (cudaMemGetInfo before and after)
    assert torch.cuda.mem_get_info()[0] == free0
    for out in outs:
        assert torch.equal(out, want)
    sample = np.arange(0, n, max(1, n // 16))
    assert np.array_equal(want.cpu().numpy()[sample], oracle.decode_batch(mask, llr, frames=sample))


def test_noalloc_argument_errors():
    mask, d, llr = _cases.frames(64, 32, 2.0, 4, seed=41)
    code = polar.polar_code_create(64, 32, mask)
    stream = torch.cuda.current_stream()
    flat = torch.zeros(64 * 4 + 1, dtype=torch.float32, device="cuda")
    out = torch.zeros((4, 4), dtype=torch.uint8, device="cuda")
    st = polar.lib().polar_decode_noalloc(code.handle, ctypes.c_void_p(flat[1:].data_ptr()),
                                         ctypes.c_void_p(out.data_ptr()), 4,
                                         ctypes.c_void_p(stream.cuda_stream))
    assert st == -4  # POLAR_EALIGN
    assert polar.lib().polar_decode_noalloc(code.handle, None, None, 0, None) == 0
