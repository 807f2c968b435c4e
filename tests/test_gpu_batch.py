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


@pytest.mark.parametrize("i8,threads,flags", [(True, 32, 0), (False, 32, 0), (True, 128, 0),
                                              (True, 32, polar.COMPILE_OUTLINE_SUBTREES),
                                              (False, 128, polar.COMPILE_OUTLINE_SUBTREES)])
def test_mixed_batch_matches_oracle(i8, threads, flags):
    """Every frame's bits equal the oracle's, for the inlined bodies and for
    bodies sharing one function per distinct register subtree across codes."""
    masks, cid, llrs, lo, oo, total_out = mixed_frames(300, 50 + threads, i8)
    codes = [polar.polar_code_create(N, K, m) for (N, K), m in zip(CODES, masks)]
    batch = polar.polar_batch_create(codes, i8, threads, flags=flags)
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


def test_mixed_full_size_sampled():
    """The full mixed workload in one launch: 65,536 frames drawn uniformly from
    the five codes (int8, 3.0 dB). About 90 sampled frames (random positions plus
    the first and last frame of every code) carry random codewords and must
    equal the oracle's decode; the other frames carry noisy all-zero codewords
    (a codeword of every code) so that the launch has its full size and mix."""
    nk = synth.MIXED_CODES
    n = synth.MIXED_FRAMES
    rng = np.random.default_rng(2024)
    masks = [synth.frozen_mask(N, K, synth.MIXED_DESIGN_DB) for N, K in nk]
    cid = np.sort(rng.integers(0, len(nk), n))[::-1].copy()  # longest codes first
    sizes = np.array([nk[c][0] for c in cid], np.int64)
    orow = np.array([(nk[c][1] + 7) // 8 for c in cid], np.int64)
    lo = np.concatenate([[0], np.cumsum(sizes)[:-1]])
    oo = np.concatenate([[0], np.cumsum(orow)[:-1]])
    flat = np.empty(int(sizes.sum()), np.int8)
    sample = set(rng.choice(n, 80, replace=False).tolist()) | {0, n - 1}
    for c in range(len(nk)):  # first and last frame of every code
        idx = np.flatnonzero(cid == c)
        sample |= {int(idx[0]), int(idx[-1])}
    for c, (N, K) in enumerate(nk):  # noisy all-zero codewords, one code at a time
        idx = np.flatnonzero(cid == c)
        y = synth.awgn_llr(rng, np.zeros((idx.size, N), np.uint8), synth.MIXED_DESIGN_DB, K / N)
        q = synth.quantize_i8(y)
        for j, i in enumerate(idx):
            flat[lo[i]: lo[i] + N] = q[j]
    want = {}
    for i in sorted(sample):  # sampled frames: random codewords from the oracle encoder
        N, K = nk[cid[i]]
        d = synth.info_bits(rng, 1, K)
        x = oracle.encode_systematic(masks[cid[i]], d[0])[None]
        q = synth.quantize_i8(synth.awgn_llr(rng, x, synth.MIXED_DESIGN_DB, K / N))[0]
        flat[lo[i]: lo[i] + N] = q
        want[i] = oracle.decode_batch(masks[cid[i]], q[None])[0]
    codes = [polar.polar_code_create(N, K, m) for (N, K), m in zip(nk, masks)]
    batch = polar.polar_batch_create(codes, True, 32)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    out = torch.full((int(orow.sum()),), 0xA5, dtype=torch.uint8, device="cuda")
    polar.polar_batch_decode(batch, dev(cid.astype(np.int32)), dev(lo), dev(oo), dev(flat), out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    for i, w in want.items():
        assert np.array_equal(got[oo[i]: oo[i] + orow[i]], w), i
    assert (got != 0xA5).any()


def test_batch_rejects_oversized_frame_count():
    codes = [polar.polar_code_create(N, K, synth.frozen_mask(N, K, 3.0)) for N, K in CODES[:2]]
    batch = polar.polar_batch_create(codes, True, 32)
    z = torch.zeros(16, dtype=torch.int64, device="cuda")
    with pytest.raises(polar.PolarError):
        polar.polar_batch_decode(batch, z, z, z, z, z.to(torch.uint8), n_frames=1 << 32)


@pytest.mark.parametrize("i8,F,flags,shuffled", [(True, 4, 0, False), (False, 2, 0, True),
                                                 (True, 4, 0, True),
                                                 (True, 2, polar.COMPILE_OUTLINE_SUBTREES, False)])
def test_mixed_batch_frame_per_warp(i8, F, flags, shuffled):
    """Several frames per CTA, one per warp: the CTA's warps decode consecutive
    frames of the list side by side. Frames in arrival order (shuffled) put
    frames of different codes in most groups, which the CTA then decodes code by
    code; 301 frames leave a ragged last group. Every frame equals the oracle."""
    masks, cid, llrs, lo, oo, total_out = mixed_frames(301, 70 + F + 10 * shuffled, i8)
    if shuffled:
        perm = np.random.default_rng(5).permutation(cid.size)
        cid, lo, oo = cid[perm], lo[perm], oo[perm]
        llrs = [llrs[i] for i in perm]
        # re-lay the LLR and output buffers in the new order
        lo = np.concatenate([[0], np.cumsum([CODES[c][0] for c in cid])[:-1]]).astype(np.uint64)
        oo = np.concatenate([[0], np.cumsum([(CODES[c][1] + 7) // 8 for c in cid])[:-1]]).astype(np.uint64)
    codes = [polar.polar_code_create(N, K, m) for (N, K), m in zip(CODES, masks)]
    batch = polar.polar_batch_create(codes, i8, 32 * F, flags=flags | polar.BATCH_FRAME_PER_WARP)
    assert polar.polar_batch_info(batch)["threads"] == 32 * F
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    llr = dev(np.concatenate(llrs))
    out = torch.full((total_out,), 0xA5, dtype=torch.uint8, device="cuda")
    polar.polar_batch_decode(batch, dev(cid.view(np.int32)), dev(lo.view(np.int64)),
                             dev(oo.view(np.int64)), llr, out)
    torch.cuda.synchronize()
    check(masks, cid, llrs, out.cpu().numpy(), oo)
