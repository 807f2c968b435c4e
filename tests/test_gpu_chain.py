"""GPU communication chain: Philox information bits, the device systematic
encoder, the AWGN channel, error counting and the whole frame-error run,
checked against the oracle's encoder and decoder and against Philox-4x32-10
computed on the host from its definition."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1504_00353_gb300 import polar, synth
from tests import _philox

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def cuda_u8(shape):
    return torch.zeros(shape, dtype=torch.uint8, device="cuda")


@pytest.mark.parametrize("K", [5, 128, 29492])
def test_random_info_is_philox(K):
    N = 1 << max(3, int(np.ceil(np.log2(K + 1))))
    code = polar.polar_code_create(N, K, synth.frozen_mask(N, K, 3.0))
    seed, frame0 = 0x1234_5678_9ABC, 77
    out = cuda_u8((6, (K + 7) // 8))
    polar.polar_random_info(code, out, seed, frame0)
    got = out.cpu().numpy()
    for f in range(6):
        assert np.array_equal(got[f], _philox.info_bytes(K, seed, frame0 + f)), f


@pytest.mark.parametrize("N,K,db,n", [(8, 4, 2.0, 40), (16, 11, 3.0, 40), (1024, 512, 2.5, 40),
                                      (2048, 1723, 3.0, 40), (32768, 29492, 4.0, 40),
                                      (1 << 20, 880804, 3.5, 2)])
def test_device_encoder_matches_oracle(N, K, db, n):
    mask = synth.frozen_mask(N, K, db)
    code = polar.polar_code_create(N, K, mask)
    rng = np.random.default_rng(N)
    d = synth.info_bits(rng, n, K)
    info = torch.from_numpy(synth.pack_bits(d)).cuda()
    cw = cuda_u8((n, (N + 7) // 8))
    polar.polar_encode_systematic_device(code, info, cw)
    got = synth.unpack_bits(cw.cpu().numpy(), N)
    for f in range(n):
        assert np.array_equal(got[f], oracle.encode_systematic(mask, d[f])), f


def test_device_encoder_rejects_non_systematic_mask():
    mask = np.ones(8, np.uint8)
    mask[[0, 1, 3]] = 0  # A = {0, 1, 3}: not domination-contiguous (2 lies between 0 and 3)
    code = polar.polar_code_create(8, 3, mask)
    info = cuda_u8((1, 1))
    with pytest.raises(polar.PolarError):
        polar.polar_encode_systematic_device(code, info, cuda_u8((1, 1)))


def test_channel_llrs():
    """float32 LLRs = 2 (s + sigma z) / sigma^2 with z the host Philox/Box-Muller
    normals (within float32 rounding of log, sqrt, sin/cos); int8 LLRs are exactly
    clamp(rint(8 LLR32)) of the device float32 values."""
    N, K, db, seed = 1024, 512, 2.5, 99
    mask = synth.frozen_mask(N, K, db)
    code = polar.polar_code_create(N, K, mask)
    rng = np.random.default_rng(3)
    d = synth.info_bits(rng, 8, K)
    x = np.stack([oracle.encode_systematic(mask, r) for r in d])
    cw = torch.from_numpy(synth.pack_bits(x)).cuda()
    l32 = torch.empty((8, N), dtype=torch.float32, device="cuda")
    l8 = torch.empty((8, N), dtype=torch.int8, device="cuda")
    polar.polar_channel_awgn(code, cw, l32, db, seed, frame0=5)
    polar.polar_channel_awgn(code, cw, l8, db, seed, frame0=5)
    g32, g8 = l32.cpu().numpy(), l8.cpu().numpy()
    s2 = synth.sigma2(db, K / N)
    for f in range(8):
        z = _philox.normals(N, seed, 5 + f)
        want = 2.0 * ((1.0 - 2.0 * x[f]) + np.sqrt(s2) * z) / s2
        assert np.allclose(g32[f], want, rtol=1e-5, atol=1e-4)
    assert np.array_equal(g8, np.clip(np.rint(8.0 * g32), -127, 127).astype(np.int8))


def test_channel_noise_statistics():
    N, K, db = 32768, 29492, 4.0
    code = polar.polar_code_create(N, K, synth.frozen_mask(N, K, db))
    cw = cuda_u8((64, N // 8))  # all-zero codewords: s = +1
    l32 = torch.empty((64, N), dtype=torch.float32, device="cuda")
    polar.polar_channel_awgn(code, cw, l32, db, seed=5)
    s2 = synth.sigma2(db, K / N)
    z = (l32.double().cpu().numpy() * s2 / 2.0 - 1.0) / np.sqrt(s2)
    assert abs(z.mean()) < 0.005 and abs(z.var() - 1.0) < 0.01
    assert abs(np.mean(z ** 3)) < 0.02 and abs(np.mean(z ** 4) - 3.0) < 0.05


def test_count_errors():
    N, K = 256, 100
    code = polar.polar_code_create(N, K, synth.frozen_mask(N, K, 3.0))
    rng = np.random.default_rng(4)
    a = synth.pack_bits(synth.info_bits(rng, 500, K))
    b = a.copy()
    flips = rng.integers(0, 4, 500)
    for f in range(500):
        for k in rng.choice(K, flips[f], replace=False):
            b[f, k >> 3] ^= 1 << (k & 7)
    cnt = torch.zeros(2, dtype=torch.int64, device="cuda")
    polar.polar_count_errors(code, torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), cnt)
    assert cnt.cpu().tolist() == [int((flips > 0).sum()), int(flips.sum())]


@pytest.mark.parametrize("i8", [False, True])
def test_chain_decodes_like_the_oracle(i8):
    """Bits drawn, encoded, sent and decoded on the GPU; the decoded bits equal
    the oracle's decode of the same LLRs, and the counters equal a host count."""
    N, K, db, n = 1024, 512, 2.0, 300
    mask = synth.frozen_mask(N, K, 2.5)
    code = polar.polar_code_create(N, K, mask)
    info = cuda_u8((n, K // 8))
    cw = cuda_u8((n, N // 8))
    llr = torch.empty((n, N), dtype=torch.int8 if i8 else torch.float32, device="cuda")
    polar.polar_random_info(code, info, seed=11)
    polar.polar_encode_systematic_device(code, info, cw)
    polar.polar_channel_awgn(code, cw, llr, db, seed=11)
    out = (polar.polar_decode_i8 if i8 else polar.polar_decode)(code, llr)
    cnt = torch.zeros(2, dtype=torch.int64, device="cuda")
    polar.polar_count_errors(code, out, info, cnt)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert np.array_equal(got, oracle.decode_batch(mask, llr.cpu().numpy()))
    diff = np.unpackbits(got ^ info.cpu().numpy(), axis=1)
    assert cnt.cpu().tolist() == [int(diff.any(axis=1).sum()), int(diff.sum())]
    assert 0 < cnt[0].item() < n  # 2.0 dB on a design-2.5 dB code: some errors, not all


def test_fer_run():
    """Whole GPU runs: repeatable for a seed; int8 (x8, +-127) loses little
    against float32 (the paper's saturating-adder claim, Sec. III-A); more
    Eb/N0, fewer errors."""
    N, K = 1024, 512
    code = polar.polar_code_create(N, K, synth.frozen_mask(N, K, 2.5))
    a = polar.polar_fer_run(code, False, 2.0, seed=1, n_frames=20000, batch=4096)
    assert a == polar.polar_fer_run(code, False, 2.0, seed=1, n_frames=20000, batch=4096)
    b = polar.polar_fer_run(code, True, 2.0, seed=1, n_frames=20000, batch=4096)
    fer32, fer8 = a[0] / 20000, b[0] / 20000
    assert 0.005 < fer32 < 0.5
    assert abs(fer8 - fer32) < 0.25 * fer32 + 0.005
    c = polar.polar_fer_run(code, False, 3.0, seed=1, n_frames=20000, batch=4096)
    assert c[0] < a[0]
