"""Specialised (code-unrolled) decoders vs the CPU oracle: the decoder generated
for one code and compiled at run time must give the same bits as the oracle
(and so as the operation-list interpreter) for float32 and int8 LLRs."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1504_00353_gb300 import polar, synth
from tests import _cases

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def decode(code, y, i8):
    t = torch.from_numpy(np.ascontiguousarray(y)).cuda()
    out = (polar.polar_decode_i8 if i8 else polar.polar_decode)(code, t)
    torch.cuda.synchronize()
    polar.polar_code_check(code)
    return out.cpu().numpy()


@pytest.mark.parametrize("i8", [False, True])
@pytest.mark.parametrize("n_frames", [1, 10000])
def test_n1024_unrolled(i8, n_frames):
    mask, d, llr = _cases.frames(1024, 512, 2.5, n_frames, seed=30, distinct=500)
    y = synth.quantize_i8(llr) if i8 else llr
    code = polar.polar_code_create(1024, 512, mask)
    assert polar.polar_code_get_launch(code, i8, n_frames)["unrolled"] == 0
    polar.polar_code_compile(code, i8, n_frames)
    assert polar.polar_code_get_launch(code, i8, n_frames)["unrolled"] == 256
    assert np.array_equal(decode(code, y, i8), oracle.decode_batch(mask, y))


@pytest.mark.parametrize("N,reg", [(8, 32), (64, 64), (512, 256), (4096, 512), (2048, 32),
                                   (8192, 1024)])
def test_random_masks_unrolled(N, reg):
    rng = np.random.default_rng(N + reg)
    K = int(rng.integers(1, N))
    mask = _cases.random_mask(rng, N, K)
    ms = int(rng.choice([0, 16, oracle.UNLIMITED]))
    code = polar.polar_code_create(N, K, mask, max_spc=ms)
    llr = (rng.standard_normal((200, N)) * 3).astype(np.float32)
    yi = rng.integers(-127, 128, (200, N)).astype(np.int8)
    for y, i8 in ((llr, False), (yi, True)):
        polar.polar_code_compile(code, i8, 200, reg)
        assert polar.polar_code_get_launch(code, i8, 200)["unrolled"] == reg
        assert np.array_equal(decode(code, y, i8), oracle.decode_batch(mask, y, max_spc=ms))


@pytest.mark.parametrize("i8", [False, True])
def test_n32768_unrolled_batch4096_sampled(i8):
    mask, d, llr = _cases.frames(32768, 29492, 4.0, 4096, seed=31, distinct=64)
    y = synth.quantize_i8(llr) if i8 else llr
    code = polar.polar_code_create(32768, 29492, mask)
    polar.polar_code_compile(code, i8, 4096)
    got = decode(code, y, i8)
    sample = np.sort(np.random.default_rng(5).choice(4096, 40, replace=False))
    assert np.array_equal(got[sample], oracle.decode_batch(mask, y, frames=sample))
    polar.polar_code_compile(code, i8, 1)
    one = decode(code, y[:1], i8)
    assert np.array_equal(one, oracle.decode_batch(mask, y[:1]))


@pytest.mark.parametrize("i8", [False, True])
@pytest.mark.parametrize("threads,reg,stage", [(256, 1024, 1), (512, 512, 2)])
def test_n32768_batch1_shapes(i8, threads, reg, stage):
    """Batch-1 (latency) shapes: one CTA, every stage in shared memory, register
    subtrees of 512 and 1024 leaves, staged or in-place channel."""
    mask, d, llr = _cases.frames(32768, 29492, 4.0, 3, seed=33)
    y = synth.quantize_i8(llr) if i8 else llr
    code = polar.polar_code_create(32768, 29492, mask)
    polar.polar_code_set_launch(code, i8, threads=threads, warp_stage_max=1024, stage_channel=stage)
    polar.polar_code_compile(code, i8, 1, reg)
    assert polar.polar_code_get_launch(code, i8, 1)["unrolled"] == reg
    for f in range(3):
        assert np.array_equal(decode(code, y[f:f + 1], i8), oracle.decode_batch(mask, y[f:f + 1]))


@pytest.mark.parametrize("seed", [0, 1])
def test_repspc_heavy_masks(seed):
    """Masks built from Repetition-SPC nodes of 8 and 16 leaves (decoded by the
    speculative register op) among random blocks: bits equal the oracle's."""
    rng = np.random.default_rng(40 + seed)

    def repspc(n):
        m = np.zeros(n, np.uint8)
        m[: n // 2 - 1] = 1
        m[n // 2] = 1
        return m
    blocks = []
    for _ in range(64):
        c = int(rng.integers(0, 3))
        blocks.append(repspc(16) if c == 0 else np.concatenate([repspc(8), repspc(8)]) if c == 1
                      else (rng.random(16) < 0.5).astype(np.uint8))
    mask = np.concatenate(blocks)
    N, K = mask.size, int((mask == 0).sum())
    code = polar.polar_code_create(N, K, mask)
    y32 = (rng.standard_normal((300, N)) * 2 + 1).astype(np.float32)
    yi = rng.integers(-127, 128, (300, N)).astype(np.int8)
    yi[:, ::7] = 127
    for y, i8 in ((y32, False), (yi, True)):
        for reg, flags in ((32, 0), (256, 0), (256, polar.COMPILE_LOCAL_LEAVES)):
            c = polar.polar_code_create(N, K, mask)
            polar.polar_code_compile(c, i8, 300, reg, flags)
            assert polar.polar_code_get_launch(c, i8, 300)["unrolled"] == reg
            assert np.array_equal(decode(c, y, i8), oracle.decode_batch(mask, y))


@pytest.mark.parametrize("i8", [False, True])
@pytest.mark.parametrize("form", ["compact", "subtrees", "memory"])
def test_outlined_forms(i8, form):
    """Out-of-line forms (subtree functions shared by equal frozen patterns,
    out-of-line memory operations, or both) give the oracle's bits, for a
    workload code at batch and batch-1 shapes and for random masks."""
    flags = {"compact": polar.COMPILE_COMPACT, "subtrees": polar.COMPILE_OUTLINE_SUBTREES,
             "memory": polar.COMPILE_OUTLINE_MEMORY}[form]
    mask, d, llr = _cases.frames(32768, 29492, 4.0, 256, seed=34, distinct=16)
    y = synth.quantize_i8(llr) if i8 else llr
    for n in (256, 1):
        code = polar.polar_code_create(32768, 29492, mask)
        polar.polar_code_compile(code, i8, n, 256, flags)
        assert polar.polar_code_get_launch(code, i8, n)["unrolled"] == 256
        got = decode(code, y[:n], i8)
        assert np.array_equal(got, oracle.decode_batch(mask, y[:n]))
    rng = np.random.default_rng(35)
    for N in (64, 2048):
        K = int(rng.integers(1, N))
        m = _cases.random_mask(rng, N, K)
        code = polar.polar_code_create(N, K, m)
        yy = rng.integers(-127, 128, (100, N)).astype(np.int8) if i8 else \
            (rng.standard_normal((100, N)) * 3).astype(np.float32)
        polar.polar_code_compile(code, i8, 100, 32, flags)
        assert np.array_equal(decode(code, yy, i8), oracle.decode_batch(m, yy))


def test_release_returns_to_interpreter():
    mask, d, llr = _cases.frames(256, 128, 3.0, 50, seed=32)
    code = polar.polar_code_create(256, 128, mask)
    polar.polar_code_compile(code, False, 50)
    assert polar.polar_code_get_launch(code, False, 50)["unrolled"] == 256
    polar.polar_code_compile(code, False, 0)
    assert polar.polar_code_get_launch(code, False, 50)["unrolled"] == 0
    assert np.array_equal(decode(code, llr, False), oracle.decode_batch(mask, llr))


@pytest.mark.parametrize("i8", [False, True])
def test_decode_from_host_buffers(i8):
    """polar_decode_host (chunked copies overlapped with decoding) gives the
    oracle's bits, with chunk sizes that leave a ragged last chunk."""
    mask, d, llr = _cases.frames(1024, 512, 2.5, 1000, seed=37, distinct=100)
    y = synth.quantize_i8(llr) if i8 else llr
    code = polar.polar_code_create(1024, 512, mask)
    want = oracle.decode_batch(mask, y)
    host = torch.from_numpy(np.ascontiguousarray(y)).pin_memory()
    for chunk in (0, 1, 128, 333, 1000, 5000):
        got = polar.polar_decode_host(code, host, chunk_frames=chunk)
        assert np.array_equal(got.numpy(), want), chunk
    got = polar.polar_decode_host(code, y)  # pageable numpy input also works
    assert np.array_equal(got.numpy(), want)


@pytest.mark.parametrize("i8", [False, True])
@pytest.mark.parametrize("F", [2, 4])
def test_frames_per_cta(i8, F):
    """Several frames per CTA, one per warp: the oracle's bits, including a
    ragged last group; the interpreter and batch-1 shapes keep one frame per CTA."""
    mask, d, llr = _cases.frames(1024, 512, 2.5, 1001, seed=39, distinct=200)
    y = synth.quantize_i8(llr) if i8 else llr
    code = polar.polar_code_create(1024, 512, mask)
    polar.polar_code_set_launch(code, i8, threads=32, stage_channel=2)
    polar.polar_code_set_frames_per_cta(code, i8, F)
    assert polar.polar_code_get_launch(code, i8, 1001)["frames_per_cta"] == 1  # not compiled yet
    assert np.array_equal(decode(code, y, i8), oracle.decode_batch(mask, y))
    polar.polar_code_compile(code, i8, 1001)
    launch = polar.polar_code_get_launch(code, i8, 1001)
    assert launch["frames_per_cta"] == F and launch["threads"] == 32 * F and launch["unrolled"]
    assert np.array_equal(decode(code, y, i8), oracle.decode_batch(mask, y))
    assert polar.polar_code_get_launch(code, i8, 1)["frames_per_cta"] == 1
    assert np.array_equal(decode(code, y[:1], i8), oracle.decode_batch(mask, y[:1]))


def test_frames_per_cta_n32768_sampled():
    mask, d, llr = _cases.frames(32768, 29492, 4.0, 4096, seed=40, distinct=64)
    y = synth.quantize_i8(llr)
    code = polar.polar_code_create(32768, 29492, mask)
    polar.polar_code_set_launch(code, True, threads=32, smem_stage_max=256, stage_channel=2)
    polar.polar_code_set_frames_per_cta(code, True, 4)
    polar.polar_code_compile(code, True, 4096)
    assert polar.polar_code_get_launch(code, True, 4096)["frames_per_cta"] == 4
    got = decode(code, y, True)
    sample = np.sort(np.random.default_rng(6).choice(4096, 40, replace=False))
    assert np.array_equal(got[sample], oracle.decode_batch(mask, y, frames=sample))
    with pytest.raises(polar.PolarError):
        polar.polar_code_set_frames_per_cta(code, True, 3)


@pytest.mark.parametrize("F", [2, 4])
def test_frames_per_cta_memory_level_nodes(F):
    """Repetition, SPC and Rate-1 nodes wider than the warp threshold run in
    memory on each warp's own frame (the top of a (4096, *) code built from one
    wide node of each kind)."""
    h = 1024
    rep = np.ones(h, np.uint8)
    rep[-1] = 0
    spc = np.zeros(h, np.uint8)
    spc[0] = 1
    mask = np.concatenate([rep, spc, np.zeros(h, np.uint8), rep])
    N, K = mask.size, int((mask == 0).sum())
    rng = np.random.default_rng(41 + F)
    for i8 in (False, True):
        y = rng.integers(-127, 128, (257, N)).astype(np.int8) if i8 else \
            (rng.standard_normal((257, N)) * 3).astype(np.float32)
        code = polar.polar_code_create(N, K, mask)
        polar.polar_code_set_launch(code, i8, threads=32, smem_stage_max=256, warp_stage_max=256,
                                    stage_channel=2)
        polar.polar_code_set_frames_per_cta(code, i8, F)
        polar.polar_code_compile(code, i8, 257, 256)
        assert polar.polar_code_get_launch(code, i8, 257)["frames_per_cta"] == F
        assert np.array_equal(decode(code, y, i8), oracle.decode_batch(mask, y))


@pytest.mark.parametrize("i8", [False, True])
@pytest.mark.parametrize("N,reg", [(64, 64), (1024, 256), (2048, 512)])
def test_local_leaves_random_masks(i8, N, reg):
    """The per-lane form of split nodes of 4 to 16 leaves (every lane decodes
    the node on its own) gives the oracle's bits on random masks, including
    ties in int8 (small integer LLRs), at batch and batch-1 shapes."""
    rng = np.random.default_rng(N + reg + i8)
    for trial in range(3):
        K = int(rng.integers(1, N))
        mask = _cases.random_mask(rng, N, K)
        y = rng.integers(-6, 7, (150, N)).astype(np.int8) if i8 else \
            (rng.standard_normal((150, N)) * 3).astype(np.float32)
        for n in (150, 1):
            code = polar.polar_code_create(N, K, mask)
            polar.polar_code_compile(code, i8, n, reg, polar.COMPILE_LOCAL_LEAVES)
            assert polar.polar_code_get_launch(code, i8, n)["unrolled"] == reg
            assert np.array_equal(decode(code, y[:n], i8), oracle.decode_batch(mask, y[:n]))


@pytest.mark.parametrize("i8", [False, True])
def test_local_leaves_n32768_batch1(i8):
    """(32768, 29492) batch-1 shape with the per-lane small-node form and
    Repetition-SPC-heavy masks."""
    mask, d, llr = _cases.frames(32768, 29492, 4.0, 3, seed=43)
    y = synth.quantize_i8(llr) if i8 else llr
    code = polar.polar_code_create(32768, 29492, mask)
    polar.polar_code_set_launch(code, i8, threads=256, warp_stage_max=1024)
    polar.polar_code_compile(code, i8, 1, 1024, polar.COMPILE_LOCAL_LEAVES)
    for f in range(3):
        assert np.array_equal(decode(code, y[f:f + 1], i8), oracle.decode_batch(mask, y[f:f + 1]))
