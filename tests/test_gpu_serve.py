"""Serving loop (continuous batching onto the mixed-batch decoder): every
request's bits equal the oracle's decode of that frame alone, whatever else was
in flight with it; admission respects the device budget (a budget of a few
frames forces ring wrap-around and back-pressure); bad requests are refused."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1504_00353_gb300 import polar, synth

pytestmark = pytest.mark.gpu

CODES = [(256, 128), (1024, 512), (2048, 1723), (16384, 14746), (32768, 29492)]


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    masks = [synth.frozen_mask(N, K, 3.0) for N, K in CODES]
    codes = [polar.polar_code_create(N, K, m) for (N, K), m in zip(CODES, masks)]
    batch = polar.polar_batch_create(codes, False, 32)
    return masks, batch


def make_requests(masks, n, seed, shuffle_host=False):
    """n requests of random codes, Eb/N0 uniform in [2, 4.5] dB, fp32 LLRs laid
    out one after another in a pinned buffer (or in a shuffled order)."""
    rng = np.random.default_rng(seed)
    cid = rng.integers(0, len(CODES), n)
    llrs = []
    for c in cid:
        N, K = CODES[c]
        d = synth.info_bits(rng, 1, K)
        x = oracle.encode_systematic(masks[c], d[0])[None]
        llrs.append(synth.awgn_llr(rng, x, rng.uniform(2.0, 4.5), K / N)[0])
    order = rng.permutation(n) if shuffle_host else np.arange(n)
    reqs = np.zeros(n, polar.REQUEST_DTYPE)
    lpos, opos = 0, 0
    llr_off, out_off = np.zeros(n, np.uint64), np.zeros(n, np.uint64)
    for i in order:  # host placement order
        N, K = CODES[cid[i]]
        llr_off[i], out_off[i] = lpos, opos
        lpos += N * 4
        opos += (K + 7) // 8
    reqs["code_id"], reqs["llr_off"], reqs["out_off"] = cid, llr_off, out_off
    host_llr = torch.empty(lpos // 4, dtype=torch.float32).pin_memory()
    hv = host_llr.numpy()
    for i in range(n):
        hv[llr_off[i] // 4: llr_off[i] // 4 + CODES[cid[i]][0]] = llrs[i]
    host_out = torch.full((opos,), 0xA5, dtype=torch.uint8).pin_memory()
    return reqs, host_llr, host_out, llrs


def expected(masks, reqs, llrs, i):
    c = int(reqs["code_id"][i])
    return oracle.decode_batch(masks[c], llrs[i][None])[0]


def drain(server, n, timeout_s=60.0):
    t0 = time.monotonic()
    while True:
        done, admissions, launches = polar.polar_server_progress(server)
        if done >= n:
            return admissions, launches
        assert time.monotonic() - t0 < timeout_s, f"{done} of {n} requests completed"
        time.sleep(1e-3)


@pytest.mark.parametrize("budget_frames,slots,max_frames,shuffle",
                         [(64, 3, 16, False), (3, 2, 4, True), (1000, 4, 256, False)])
def test_served_bits_match_oracle(setup, budget_frames, slots, max_frames, shuffle):
    masks, batch = setup
    n = 400
    reqs, host_llr, host_out, llrs = make_requests(masks, n, 7 + budget_frames, shuffle)
    done_ns = np.zeros(n, np.uint64)
    budget = budget_frames * 32768 * 4  # frames of the longest code
    srv = polar.polar_server_create(batch, reqs, host_llr, host_out, done_ns, budget, max_frames,
                                    slots)
    t_pub = np.zeros(n, np.uint64)
    for k in range(0, n, 7):  # arrivals in bursts of 7 while earlier ones decode
        hi = min(n, k + 7)
        t_pub[k:hi] = time.monotonic_ns()
        polar.polar_server_publish(srv, hi)
        time.sleep(2e-5)
    admissions, launches = drain(srv, n)
    polar.polar_server_destroy(srv)
    assert admissions > 1 and launches == admissions
    assert (done_ns >= t_pub).all() and (done_ns > 0).all()
    out = host_out.numpy()
    for i in range(n):
        K = CODES[reqs["code_id"][i]][1]
        got = out[int(reqs["out_off"][i]): int(reqs["out_off"][i]) + (K + 7) // 8]
        assert np.array_equal(got, expected(masks, reqs, llrs, i)), i


def test_alone_equals_in_mix(setup):
    """The same frames decoded one request at a time (nothing else in flight)
    and all at once in a mix give identical bits."""
    masks, batch = setup
    n = 60
    reqs, host_llr, host_out, llrs = make_requests(masks, n, 99)
    done = np.zeros(n, np.uint64)
    srv = polar.polar_server_create(batch, reqs, host_llr, host_out, done, 1 << 26, 64, 4)
    for i in range(n):
        polar.polar_server_publish(srv, i + 1)
        drain(srv, i + 1)
    polar.polar_server_destroy(srv)
    alone = host_out.numpy().copy()
    host_out.fill_(0)
    srv = polar.polar_server_create(batch, reqs, host_llr, host_out, done, 1 << 26, 64, 4)
    polar.polar_server_publish(srv, n)
    drain(srv, n)
    polar.polar_server_destroy(srv)
    assert np.array_equal(alone, host_out.numpy())
    for i in range(n):
        K = CODES[reqs["code_id"][i]][1]
        o = int(reqs["out_off"][i])
        assert np.array_equal(alone[o: o + (K + 7) // 8], expected(masks, reqs, llrs, i))


def test_per_code_launch_policy(setup):
    """One launch per code in each admission (the plain baseline) gives the
    same bits, with more launches than admissions."""
    masks, batch = setup
    n = 120
    reqs, host_llr, host_out, llrs = make_requests(masks, n, 11)
    done = np.zeros(n, np.uint64)
    srv = polar.polar_server_create(batch, reqs, host_llr, host_out, done, 1 << 26, 64, 1,
                                    flags=polar.SERVE_LAUNCH_PER_CODE)
    polar.polar_server_publish(srv, n)
    admissions, launches = drain(srv, n)
    polar.polar_server_destroy(srv)
    assert launches > admissions
    out = host_out.numpy()
    for i in range(n):
        K = CODES[reqs["code_id"][i]][1]
        o = int(reqs["out_off"][i])
        assert np.array_equal(out[o: o + (K + 7) // 8], expected(masks, reqs, llrs, i)), i


def test_device_resident_pool(setup):
    """Request buffers in device memory (the copies stay in HBM) give the same
    bits as the oracle."""
    masks, batch = setup
    n = 150
    reqs, host_llr, host_out, llrs = make_requests(masks, n, 21)
    d_llr = host_llr.cuda()
    d_out = torch.zeros_like(host_out, device="cuda")
    done = np.zeros(n, np.uint64)
    srv = polar.polar_server_create(batch, reqs, d_llr, d_out, done, 1 << 26, 32, 3)
    polar.polar_server_publish(srv, n)
    drain(srv, n)
    polar.polar_server_destroy(srv)
    out = d_out.cpu().numpy()
    for i in range(n):
        K = CODES[reqs["code_id"][i]][1]
        o = int(reqs["out_off"][i])
        assert np.array_equal(out[o: o + (K + 7) // 8], expected(masks, reqs, llrs, i)), i


def test_request_ring_wraps(setup):
    """A request array shorter than the run: slots are reused once complete."""
    masks, batch = setup
    n, cap = 300, 32
    reqs_all, host_llr, host_out, llrs = make_requests(masks, n, 5)
    ring = np.zeros(cap, polar.REQUEST_DTYPE)
    done = np.zeros(cap, np.uint64)
    srv = polar.polar_server_create(batch, ring, host_llr, host_out, done, 1 << 24, 16, 3)
    pub = 0
    t0 = time.monotonic()
    while pub < n:
        completed = polar.polar_server_progress(srv)[0]
        hi = min(n, completed + cap)
        if hi > pub:
            for i in range(pub, hi):
                ring[i % cap] = reqs_all[i]
            polar.polar_server_publish(srv, hi)
            pub = hi
        assert time.monotonic() - t0 < 60
    drain(srv, n)
    polar.polar_server_destroy(srv)
    out = host_out.numpy()
    for i in range(n):
        K = CODES[reqs_all["code_id"][i]][1]
        o = int(reqs_all["out_off"][i])
        assert np.array_equal(out[o: o + (K + 7) // 8], expected(masks, reqs_all, llrs, i)), i


def test_bad_requests_refused(setup):
    masks, batch = setup
    reqs, host_llr, host_out, llrs = make_requests(masks, 8, 3)
    done = np.zeros(8, np.uint64)
    srv = polar.polar_server_create(batch, reqs, host_llr, host_out, done, 1 << 24, 8, 2)
    reqs["code_id"][2] = len(CODES)  # unknown code
    with pytest.raises(polar.PolarError):
        polar.polar_server_publish(srv, 3)
    reqs["code_id"][2] = 0
    reqs["llr_off"][2] = host_llr.numel() * 4 - 16  # runs past the input buffer
    with pytest.raises(polar.PolarError):
        polar.polar_server_publish(srv, 3)
    with pytest.raises(polar.PolarError):
        polar.polar_server_publish(srv, 9)  # beyond the request array
    polar.polar_server_publish(srv, 2)  # the valid prefix is still accepted
    drain(srv, 2)
    polar.polar_server_destroy(srv)
    with pytest.raises(polar.PolarError):  # budget below one frame of the longest code
        polar.polar_server_create(batch, reqs, host_llr, host_out, done, 1024, 8, 2)
