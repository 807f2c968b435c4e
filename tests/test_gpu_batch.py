"""Mixed-code batches (one persistent launch over frames of several codes):
every frame's bits must equal the oracle's for that frame's code, and the
launch must replay correctly from a captured CUDA graph."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1504_00353_gb300 import polar, synth

pytestmark = pytest.mark.gpu

CODES = [(256, 128), (1024, 512), (2048, 1723), (16384, 14746), (32768, 29492)]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def mixed_frames(n, seed, i8, id_seed=None):
    """Frames of random codes (longest first), LLRs concatenated, plus offsets.
    Code ids come from id_seed (default: seed), bits and noise from seed."""
    id_rng = np.random.default_rng(seed if id_seed is None else id_seed)
    rng = np.random.default_rng(seed + 1000)
    masks = [synth.frozen_mask(N, K, 3.0) for N, K in CODES]
    cid = np.sort(id_rng.integers(0, len(CODES), n))[::-1].copy()  # longest codes first
    llrs, outs, lo, oo = [], [], [0], [0]
    for c in cid:
        N, K = CODES[c]
        d = synth.info_bits(rng, 1, K)
        x = oracle.encode_systematic(masks[c], d[0])[None]
        y = synth.awgn_llr(rng, x, 3.0, K / N)[0]
        y = synth.quantize_i8(y) if i8 else y
        llrs.append(y)
        lo.append(lo[-1] + N)
        oo.append(oo[-1] + (K + 7) // 8)
    return masks, cid.astype(np.uint32), llrs, np.array(lo[:-1], np.uint64), np.array(oo[:-1], np.uint64), oo[-1]


def check(masks, cid, llrs, got, oo):
    for i, c in enumerate(cid):
        N, K = CODES[c]
        want = oracle.decode_batch(masks[c], llrs[i][None])[0]
        assert np.array_equal(got[oo[i]: oo[i] + (K + 7) // 8], want), (i, c)


@pytest.mark.parametrize("i8,threads", [(True, 32), (False, 32), (True, 128)])
def test_mixed_batch_matches_oracle(i8, threads):
    masks, cid, llrs, lo, oo, total_out = mixed_frames(300, 50 + threads, i8)
    codes = [polar.polar_code_create(N, K, m) for (N, K), m in zip(CODES, masks)]
    batch = polar.polar_batch_create(codes, i8, threads)
    assert polar.polar_batch_info(batch)["grid"] > 0
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    llr = dev(np.concatenate(llrs))
    out = torch.full((total_out,), 0xA5, dtype=torch.uint8, device="cuda")
    polar.polar_batch_decode(batch, dev(cid.view(np.int32)), dev(lo.view(np.int64)),
                             dev(oo.view(np.int64)), llr, out)
    torch.cuda.synchronize()
    check(masks, cid, llrs, out.cpu().numpy(), oo)


def test_mixed_batch_in_cuda_graph():
    masks, cid, llrs, lo, oo, total_out = mixed_frames(200, 60, True)
    codes = [polar.polar_code_create(N, K, m) for (N, K), m in zip(CODES, masks)]
    batch = polar.polar_batch_create(codes, True, 32)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    llr = dev(np.concatenate(llrs))
    ids, l_off, o_off = dev(cid.view(np.int32)), dev(lo.view(np.int64)), dev(oo.view(np.int64))
    out = torch.zeros((total_out,), dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):  # warm-up outside capture
        polar.polar_batch_decode(batch, ids, l_off, o_off, llr, out, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        polar.polar_batch_decode(batch, ids, l_off, o_off, llr, out)
    for rep in range(2):
        # new channel values for the same frames, then replay
        masks2, cid2, llrs2, lo2, oo2, _ = mixed_frames(200, 70 + rep, True, id_seed=60)
        assert np.array_equal(cid2, cid) and np.array_equal(lo2, lo)
        llr.copy_(dev(np.concatenate(llrs2)))
        out.zero_()
        g.replay()
        torch.cuda.synchronize()
        check(masks2, cid2, llrs2, out.cpu().numpy(), oo2)
