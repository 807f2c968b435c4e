"""GPU decoder vs CPU oracle: decoded bits bit-exact, fp32 intermediate LLRs equal
(0 ULP, compared by value so +0 == -0), int8 intermediates exact. Every call goes
through the C ABI (include/polar_gb300.h) via the ctypes binding."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1504_00353_gb300 import polar, synth
from tests import _cases

pytestmark = pytest.mark.gpu

U = oracle.UNLIMITED


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def gpu_decode(code, llr, i8=False):
    t = torch.from_numpy(np.ascontiguousarray(llr)).cuda()
    out = (polar.polar_decode_i8 if i8 else polar.polar_decode)(code, t)
    torch.cuda.synchronize()
    polar.polar_code_check(code)
    return out.cpu().numpy()


def oracle_bits(mask, llr, max_rep=U, max_spc=U, frames=None):
    return oracle.decode_batch(mask, llr, max_rep=max_rep, max_spc=max_spc, frames=frames)


def both_types(llr):
    return [(llr, False), (synth.quantize_i8(llr), True)]


# ---------------------------------------------------------------- small codes

def test_listing1_code_many_frames():
    mask = np.array([1, 1, 0, 0, 1, 0, 0, 0], np.uint8)
    rng = np.random.default_rng(20)
    llr = (rng.standard_normal((5000, 8)) * 2).astype(np.float32)
    code = polar.polar_code_create(8, 5, mask)
    for y, i8 in both_types(llr):
        assert np.array_equal(gpu_decode(code, y, i8), oracle_bits(mask, y))


@pytest.mark.parametrize("N", [2, 4, 8, 16, 32, 64, 128, 256, 512, 1024, 2048, 4096])
def test_random_masks_all_sizes(N):
    """Random frozen sets (every node type and split pattern) with continuous and
    integer-valued LLRs (ties, zeros, saturation for int8)."""
    rng = np.random.default_rng(N)
    for trial in range(6):
        K = int(rng.integers(0, N + 1))
        mask = _cases.random_mask(rng, N, K)
        mr = int(rng.choice([U, 0, 4]))
        ms = int(rng.choice([U, 0, 16]))
        code = polar.polar_code_create(N, K, mask, max_rep=mr, max_spc=ms)
        n = 97
        llr_c = (rng.standard_normal((n, N)) * 3).astype(np.float32)
        llr_i = rng.integers(-4, 5, (n, N)).astype(np.float32)
        llr_s = rng.integers(-127, 128, (n, N)).astype(np.int8)
        for y, i8 in [(llr_c, False), (llr_i, False), (llr_i.astype(np.int8), True),
                      (llr_s, True), (synth.quantize_i8(llr_c), True)]:
            got = gpu_decode(code, y, i8)
            want = oracle_bits(mask, y, mr, ms)
            assert np.array_equal(got, want), (N, K, mr, ms, i8)


@pytest.mark.parametrize("N", [4, 32, 64, 1024, 32768])
def test_single_node_codes(N):
    """Rate-1 (K=N), Repetition (K=1), SPC (K=N-1), Rate-0 (K=0) as the whole code."""
    rng = np.random.default_rng(21)
    llr = (rng.standard_normal((33, N)) * 2).astype(np.float32)
    for K, mask in [(N, np.zeros(N, np.uint8)),
                    (1, np.r_[np.ones(N - 1, np.uint8), [0]].astype(np.uint8)),
                    (N - 1, np.r_[[1], np.zeros(N - 1, np.uint8)].astype(np.uint8))]:
        code = polar.polar_code_create(N, K, mask)
        for y, i8 in both_types(llr):
            assert np.array_equal(gpu_decode(code, y, i8), oracle_bits(mask, y)), (N, K, i8)
    code = polar.polar_code_create(N, 0, np.ones(N, np.uint8))
    out = gpu_decode(code, llr)
    assert out.shape == (33, 0)


# ---------------------------------------------------------------- workload codes

def test_n1024_k512_10000_frames_fp32():
    """(1024, 512) at 2.5 dB, 10,000 frames, one launch, every frame bit-exact."""
    mask, d, llr = _cases.frames(1024, 512, 2.5, 10000, seed=0, distinct=2000)
    code = polar.polar_code_create(1024, 512, mask)
    got = gpu_decode(code, llr)
    assert np.array_equal(got, oracle_bits(mask, llr))


def test_n1024_int8_and_noiseless():
    mask, d, llr = _cases.frames(1024, 512, 2.5, 3000, seed=1, distinct=500)
    code = polar.polar_code_create(1024, 512, mask)
    q = synth.quantize_i8(llr)
    assert np.array_equal(gpu_decode(code, q, True), oracle_bits(mask, q))
    x = np.stack([oracle.encode_systematic(mask, r) for r in d[:64]])
    clean = (1.0 - 2.0 * x).astype(np.float32) * 4
    assert np.array_equal(gpu_decode(code, clean), synth.pack_bits(d[:64]))


@pytest.mark.parametrize("i8", [False, True])
def test_n32768_batch4096_sampled(i8):
    """(32768, 29492) at 4.0 dB, batch 4096 in the benchmark's launch shape; 48
    sampled frames compared with the oracle one by one."""
    mask, d, llr = _cases.frames(32768, 29492, 4.0, 4096, seed=2, distinct=64)
    code = polar.polar_code_create(32768, 29492, mask)
    y = synth.quantize_i8(llr) if i8 else llr
    got = gpu_decode(code, y, i8)
    rng = np.random.default_rng(3)
    sample = np.sort(rng.choice(4096, 48, replace=False))
    want = oracle_bits(mask, y, frames=sample)
    assert np.array_equal(got[sample], want)


@pytest.mark.parametrize("i8", [False, True])
def test_n32768_batch1_latency_shape(i8):
    mask, d, llr = _cases.frames(32768, 29492, 4.0, 3, seed=4)
    code = polar.polar_code_create(32768, 29492, mask)
    y = synth.quantize_i8(llr) if i8 else llr
    for f in range(3):
        got = gpu_decode(code, y[f:f + 1], i8)
        assert np.array_equal(got, oracle_bits(mask, y[f:f + 1]))


@pytest.mark.parametrize("i8", [False, True])
def test_n1m_sampled(i8):
    """N = 2^20, K = 880,804 at 3.5 dB; 64 frames decoded, 3 compared."""
    N, K = 1 << 20, 880804
    mask, d, llr = _cases.frames(N, K, 3.5, 64, seed=5, distinct=4)
    code = polar.polar_code_create(N, K, mask)
    y = synth.quantize_i8(llr) if i8 else llr
    got = gpu_decode(code, y, i8)
    sample = np.array([0, 31, 63])
    assert np.array_equal(got[sample], oracle_bits(mask, y, frames=sample))


# ---------------------------------------------------------------- intermediate LLRs

@pytest.mark.parametrize("N,K,db", [(8, 5, None), (1024, 512, 2.5), (32768, 29492, 4.0)])
def test_alpha_trace_equals_oracle(N, K, db):
    """Every F/G/G_0R output equals the oracle's (fp32 by value, 0 ULP; int8 exact)."""
    if db is None:
        mask = np.array([1, 1, 0, 0, 1, 0, 0, 0], np.uint8)
        rng = np.random.default_rng(22)
        llr = (rng.standard_normal((16, 8)) * 2).astype(np.float32)
    else:
        mask, d, llr = _cases.frames(N, K, db, 6, seed=6)
    code = polar.polar_code_create(N, K, mask)
    for y, i8 in both_types(llr):
        t = torch.from_numpy(y).cuda()
        bits, trace = polar.polar_decode_trace(code, t)
        torch.cuda.synchronize()
        trace = trace.cpu().numpy()
        assert np.array_equal(bits.cpu().numpy(), oracle_bits(mask, y))
        for f in range(y.shape[0]):
            _, ops, alpha = oracle.fastssc_decode(mask, y[f], trace=True)
            assert np.array_equal(trace[f], alpha)  # == treats +0 and -0 as equal


# ---------------------------------------------------------------- launch shapes

SHAPES = [
    dict(threads=32, smem_stage_max=64, warp_stage_max=2, stage_channel=2),
    dict(threads=64, smem_stage_max=128, warp_stage_max=64, stage_channel=1),
    dict(threads=128, smem_stage_max=256, warp_stage_max=32, stage_channel=2),
    dict(threads=256, smem_stage_max=1024, warp_stage_max=256, stage_channel=1),
    dict(threads=512, smem_stage_max=4096, warp_stage_max=128, stage_channel=2),
    dict(threads=1024, smem_stage_max=8192, warp_stage_max=1024, stage_channel=1),
    dict(threads=96, smem_stage_max=64, warp_stage_max=16, stage_channel=1, ctas_per_sm=1),
]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("N,K,db", [(2048, 1723, 3.0), (16384, 14746, 3.0)])
def test_launch_shapes_agree(shape, N, K, db):
    """Any thread count, shared/device stage split, warp threshold and channel
    staging gives the same bits (device scratch and bulk-copy paths included)."""
    mask, d, llr = _cases.frames(N, K, db, 300, seed=7, distinct=40)
    code = polar.polar_code_create(N, K, mask)
    for y, i8 in both_types(llr):
        polar.polar_code_set_launch(code, i8, **shape)
        got = gpu_decode(code, y, i8)
        sample = np.arange(0, 300, 23)
        assert np.array_equal(got[sample], oracle_bits(mask, y, frames=sample)), (shape, i8)
        polar.polar_code_set_launch(code, i8)


# ---------------------------------------------------------------- edges and API

def test_zero_frames_is_noop_and_misaligned_pointer_rejected():
    mask = synth.frozen_mask(64, 32, 2.0)
    code = polar.polar_code_create(64, 32, mask)
    t = torch.zeros((4, 64), dtype=torch.float32, device="cuda")
    out = torch.zeros((4, 4), dtype=torch.uint8, device="cuda")
    polar.polar_decode(code, t, out, n_frames=0)
    flat = torch.zeros(64 * 4 + 1, dtype=torch.float32, device="cuda")
    with pytest.raises(polar.PolarError) as e:
        polar.polar_decode(code, flat[1:], out, n_frames=4)
    assert e.value.status == -4


def test_two_streams_same_handle():
    mask, d, llr = _cases.frames(2048, 1723, 3.0, 800, seed=8, distinct=100)
    code = polar.polar_code_create(2048, 1723, mask)
    t = torch.from_numpy(llr).cuda()
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(s1):
        a = polar.polar_decode(code, t[:400], stream=s1)
    with torch.cuda.stream(s2):
        b = polar.polar_decode(code, t[400:], stream=s2)
    torch.cuda.synchronize()
    got = torch.cat([a, b]).cpu().numpy()
    assert np.array_equal(got, oracle_bits(mask, llr))


def test_get_launch_reports_shape():
    mask = synth.frozen_mask(32768, 29492, 4.0)
    code = polar.polar_code_create(32768, 29492, mask)
    for i8 in (False, True):
        for n in (1, 4096):
            sh = polar.polar_code_get_launch(code, i8, n)
            assert sh["grid"] >= 1 and sh["threads"] % 32 == 0
            assert sh["smem_bytes"] <= 232448


# ---------------------------------------------------------------- failure path

def test_bounded_wait_reports_timeout_and_context_survives():
    """A device wait that nothing completes gives up after its limit and reports
    POLAR_ETIMEOUT through polar_code_check (once: the word is cleared); decoding
    on the same context still gives the oracle's bits afterwards."""
    import time
    mask, d, llr = _cases.frames(1024, 512, 2.5, 8, seed=38)
    code = polar.polar_code_create(1024, 512, mask)
    t0 = time.monotonic()
    polar.polar_selftest_bounded_wait(code, 2000)  # 2 ms
    with pytest.raises(polar.PolarError) as e:
        polar.polar_code_check(code)
    assert e.value.status == -5  # POLAR_ETIMEOUT
    assert time.monotonic() - t0 < 10
    polar.polar_code_check(code)  # cleared
    assert np.array_equal(gpu_decode(code, llr, False), oracle_bits(mask, llr))
    with pytest.raises(polar.PolarError):
        polar.polar_selftest_bounded_wait(code, 0)
