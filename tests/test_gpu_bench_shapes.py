"""The decoders the benchmark times, at exactly the launch shapes it times them
with, against the CPU oracle.

Every shape comes from the same place bench.py takes it from
(``autotune.shape_for`` / ``autotune.batch_shape``: the tuned table for this
device, else the measured fallback), so a re-tune cannot move the benchmark
off a tested shape. The specialised decoder is generated per code and per
shape (Sec. III-B, "Generating an Unrolled Decoder"), so each shape is its own
program and each gets its own comparison: bit-exact decoded bits on sampled
frames of a full-size batch, and on every frame where the oracle is quick."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1504_00353_gb300 import autotune, polar, synth
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


def bench_code(wl_name, dtype, n_frames, latency=False):
    """A code handle configured and compiled the way bench.py does it."""
    wl = synth.WORKLOADS[wl_name]
    N, K = wl["N"], wl["K"]
    mask = synth.frozen_mask(N, K, wl["design_db"])
    shape, _ = autotune.shape_for(N, K, mask, dtype, latency=latency)
    if not latency:
        shape.setdefault("stage_channel", 2)
    code = polar.polar_code_create(N, K, mask)
    autotune.configure(code, dtype, shape, n_frames)
    launch = polar.polar_code_get_launch(code, dtype == "i8", n_frames)
    assert launch["unrolled"], "the benchmarked decoder is the specialised one"
    for k in ("threads", "smem_stage_max", "warp_stage_max", "frames_per_cta"):
        want = shape.get(k)
        if k == "threads" and shape.get("frames_per_cta", 1) > 1:
            want = 32 * shape["frames_per_cta"]
        if want and k != "smem_stage_max":
            assert launch[k] == want, (k, launch, shape)
    return code, mask, launch


@pytest.mark.parametrize("dtype", ["i8", "f32"])
def test_throughput_shape_n32768(dtype):
    """(32768, 29492) at 4.0 dB, 4096 frames: the bench line's decoder."""
    wl = synth.WORKLOADS["n32768_k29492_4.0db"]
    code, mask, launch = bench_code("n32768_k29492_4.0db", dtype, 4096)
    _, d, llr = _cases.frames(32768, 29492, 4.0, 4096, seed=wl["seed"] + 77, distinct=48,
                              mask=mask)
    y = synth.quantize_i8(llr) if dtype == "i8" else llr
    got = decode(code, y, dtype == "i8")
    rng = np.random.default_rng(90)
    # sampled frames, plus the first and last frame slots of the launch grid
    sample = np.unique(np.concatenate([rng.choice(4096, 40, replace=False), [0, 4095],
                                       [min(4095, launch["grid"] * launch["frames_per_cta"])]]))
    assert np.array_equal(got[sample], oracle.decode_batch(mask, y, frames=sample))


@pytest.mark.parametrize("dtype", ["i8", "f32"])
def test_latency_shape_n32768(dtype):
    """(32768, 29492) batch-1: the latency line's decoder (one CTA)."""
    code, mask, launch = bench_code("n32768_k29492_4.0db", dtype, 1, latency=True)
    assert launch["grid"] == 1
    _, d, llr = _cases.frames(32768, 29492, 4.0, 4, seed=91, mask=mask)
    y = synth.quantize_i8(llr) if dtype == "i8" else llr
    for f in range(4):
        assert np.array_equal(decode(code, y[f:f + 1], dtype == "i8"),
                              oracle.decode_batch(mask, y[f:f + 1]))


@pytest.mark.parametrize("dtype", ["f32", "i8"])
def test_throughput_shape_n1024(dtype):
    """(1024, 512) at 2.5 dB, 10,000 frames in one launch: every frame."""
    code, mask, launch = bench_code("n1024_k512_2.5db", dtype, 10000)
    _, d, llr = _cases.frames(1024, 512, 2.5, 10000, seed=92, distinct=2000, mask=mask)
    y = synth.quantize_i8(llr) if dtype == "i8" else llr
    assert np.array_equal(decode(code, y, dtype == "i8"), oracle.decode_batch(mask, y))


@pytest.mark.parametrize("dtype", ["i8", "f32"])
def test_mixed_batch_tuned_shape(dtype):
    """The mixed-length batch kernel with the tuned block size, per-code stage
    caps and warp thresholds and resident-CTA cap, on 3,000 frames of the five
    codes in arrival order (descriptors longest code first)."""
    shape, src = autotune.batch_shape(dtype)
    nk = synth.MIXED_CODES
    masks = [synth.frozen_mask(N, K, synth.MIXED_DESIGN_DB) for N, K in nk]
    codes = [polar.polar_code_create(N, K, m) for (N, K), m in zip(nk, masks)]
    batch = polar.polar_batch_create(codes, dtype == "i8", shape["threads"],
                                     shape["smem_stage_max"], shape["warp_stage_max"],
                                     shape["ctas_per_sm"], shape.get("flags", 0))
    info = polar.polar_batch_info(batch)
    assert info["grid"] > 0
    rng = np.random.default_rng(93)
    n = 3000
    cid = rng.integers(0, len(nk), n)
    llrs, lo, oo = [], [0], [0]
    per_code = {}
    for c in range(len(nk)):
        m = int((cid == c).sum())
        N, K = nk[c]
        _, d, y = _cases.frames(N, K, synth.MIXED_DESIGN_DB, m, seed=94 + c, distinct=24,
                                mask=masks[c])
        per_code[c] = synth.quantize_i8(y) if dtype == "i8" else y
    pos = [0] * len(nk)
    rows = []
    for i in range(n):
        c = cid[i]
        rows.append(per_code[c][pos[c]])
        pos[c] += 1
        lo.append(lo[-1] + nk[c][0])
        oo.append(oo[-1] + (nk[c][1] + 7) // 8)
    order = np.lexsort((np.arange(n), -np.array([nk[c][0] for c in cid])))
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    llr = dev(np.concatenate(rows))
    out = torch.full((oo[-1],), 0xA5, dtype=torch.uint8, device="cuda")
    lo_a, oo_a = np.array(lo[:-1], np.int64), np.array(oo[:-1], np.int64)
    polar.polar_batch_decode(batch, dev(cid[order].astype(np.int32)), dev(lo_a[order]),
                             dev(oo_a[order]), llr, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    # every short frame, and a sample of the two long codes
    check = [i for i in range(n) if nk[cid[i]][0] <= 2048]
    long_ = [i for i in range(n) if nk[cid[i]][0] > 2048]
    check += list(rng.choice(long_, 30, replace=False))
    for i in check:
        c = cid[i]
        want = oracle.decode_batch(masks[c], rows[i][None])[0]
        assert np.array_equal(got[oo[i]: oo[i] + (nk[c][1] + 7) // 8], want), (i, nk[c], src)


@pytest.mark.parametrize("dtype", ["i8", "f32"])
def test_shape_n1m(dtype):
    """(2^20, 880,804) at 3.5 dB, 64 frames: the shape the N = 2^20 line uses
    (compact specialised form); three frames compared with the oracle."""
    wl = synth.WORKLOADS["n1048576_k880804_3.5db"]
    N, K = wl["N"], wl["K"]
    code, mask, launch = bench_code("n1048576_k880804_3.5db", dtype, 64)
    _, d, llr = _cases.frames(N, K, 3.5, 64, seed=95, distinct=3, mask=mask)
    y = synth.quantize_i8(llr) if dtype == "i8" else llr
    got = decode(code, y, dtype == "i8")
    sample = np.array([0, 41, 63])
    assert np.array_equal(got[sample], oracle.decode_batch(mask, y, frames=sample))
