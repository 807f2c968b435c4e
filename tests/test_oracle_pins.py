"""Pins of the CPU oracle against things other than itself.

Each test names what fixes the expected answer: a value the paper prints
(tests/golden/), a closed form, brute-force enumeration on tiny codes, or an
invariant of polar codes. None of them calls the GPU library.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1504_00353_gb300 import synth
from tests import _brute

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
U = oracle.UNLIMITED


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        return [ln.strip() for ln in fh if ln.strip() and not ln.startswith("#")]


def _random_mask(rng, N, K):
    m = np.ones(N, np.uint8)
    m[rng.choice(N, K, replace=False)] = 0
    return m


def _int_llr(rng, n, lo=-8, hi=8):
    return rng.integers(lo, hi + 1, size=n).astype(np.float32)


# ---------------------------------------------------------------- encoder

def test_encoder_matches_printed_g4():
    """Rows of G_4 printed in Sec. II-A are the codewords of unit vectors."""
    rows = [[int(v) for v in r.split()] for r in _rows("g4_matrix.txt")]
    for i, row in enumerate(rows):
        e = np.zeros(4, np.uint8)
        e[i] = 1
        assert oracle.encode(e).tolist() == row


def test_encoder_n2_butterfly():
    """Fig. 1a: x0 = u0 xor u1, x1 = u1."""
    for u0 in (0, 1):
        for u1 in (0, 1):
            assert oracle.encode(np.array([u0, u1], np.uint8)).tolist() == [u0 ^ u1, u1]


@pytest.mark.parametrize("N", [2, 4, 8, 16, 64, 256])
def test_encoder_equals_kronecker_power(N):
    """x = u G_N with G_N built by numpy's Kronecker product."""
    rng = np.random.default_rng(N)
    for _ in range(20):
        u = rng.integers(0, 2, N).astype(np.uint8)
        assert np.array_equal(oracle.encode(u), _brute.encode(u))


@pytest.mark.parametrize("N,K,db", [(1024, 512, 2.5), (32768, 29492, 4.0), (256, 128, 3.0),
                                    (2048, 1723, 3.0), (16384, 14746, 3.0)])
def test_systematic_invariants_on_workload_codes(N, K, db):
    """x[A] = d, and x is a codeword: (x G)[A^c] = 0 since G is an involution."""
    mask = synth.frozen_mask(N, K, db)
    rng = np.random.default_rng(7)
    for _ in range(3):
        d = rng.integers(0, 2, K).astype(np.uint8)
        x = oracle.encode_systematic(mask, d)
        assert np.array_equal(x[mask == 0], d)
        u = oracle.encode(x)
        assert not u[mask == 1].any()


def test_systematic_brute_force_bijection_n16():
    """For a constructed (16, 9) code, d -> x enumerates the codebook exactly."""
    mask = synth.frozen_mask(16, 9, 2.0)
    cb = {tuple(c) for c in _brute.codebook(mask)}
    seen = set()
    for v in range(1 << 9):
        d = np.array([(v >> j) & 1 for j in range(9)], np.uint8)
        x = oracle.encode_systematic(mask, d)
        assert np.array_equal(x[mask == 0], d)
        seen.add(tuple(x))
    assert seen == cb


# ---------------------------------------------------------------- element operations

def test_f_is_the_maxlog_xor_marginal():
    """Eq. 1: sgn(a)sgn(b)min(|a|,|b|) equals (|a+b| - |a-b|)/2, the max-log LLR of a
    XOR of two bits; the right side is evaluated in exact rational arithmetic."""
    rng = np.random.default_rng(1)
    vals = np.concatenate([rng.standard_normal(2000) * 10,
                           [0.0, -0.0, 1e-30, -1e-30, 3.0, -3.0, 1e30, -1e30]]).astype(np.float32)
    for _ in range(3000):
        a, b = (float(v) for v in rng.choice(vals, 2))
        fa, fb = Fraction(a), Fraction(b)
        want = (abs(fa + fb) - abs(fa - fb)) / 2
        assert Fraction(oracle.f_f32(a, b)) == want


def test_f_i8_range():
    for a in range(-127, 128, 3):
        for b in range(-127, 128, 5):
            assert oracle.f_i8(a, b) == (abs(a + b) - abs(a - b)) // 2


def test_int8_g_saturation_golden():
    for r in _rows("int8_g_saturation.txt"):
        a, b, beta, want = (int(v) for v in r.split())
        assert oracle.g_i8(a, b, beta) == want, r


# ---------------------------------------------------------------- SC

@pytest.mark.parametrize("N", [2, 4, 8, 16])
def test_sc_equals_sequential_maxlog_brute_force(N):
    """Min-sum SC is exact max-log decoding of u_i given the earlier decisions.
    Integer LLRs keep every float32 step exact, so decisions must agree bit for bit
    (including a zero LLR, which both sides decide as 0)."""
    rng = np.random.default_rng(100 + N)
    for trial in range(150 if N < 16 else 40):
        K = int(rng.integers(0, N + 1))
        mask = _random_mask(rng, N, K)
        alpha = _int_llr(rng, N)
        want = _brute.sequential_maxlog(mask, alpha)
        assert np.array_equal(oracle.sc_decode(mask, alpha), want), (mask, alpha)
        # int8 SC: |sums| stay below 127 here, so it is the same integer arithmetic
        a8 = alpha.astype(np.int8)
        assert np.array_equal(oracle.sc_decode(mask, a8), want)


# ---------------------------------------------------------------- Fast-SSC nodes

def _single_node_masks(N):
    r0 = np.ones(N, np.uint8)
    r1 = np.zeros(N, np.uint8)
    rep = np.ones(N, np.uint8)
    rep[-1] = 0
    spc = np.zeros(N, np.uint8)
    spc[0] = 1
    return {"R0": r0, "R1": r1, "Rep": rep, "SPC": spc}


@pytest.mark.parametrize("N", [2, 4, 8, 16])
def test_single_node_codes_are_ml(N):
    """Rate-0/Rate-1/Repetition/SPC decoders are ML decoders of their codes: the
    output is a codeword of maximal correlation (any one of them on ties)."""
    rng = np.random.default_rng(200 + N)
    for name, mask in _single_node_masks(N).items():
        cb = {tuple(c) for c in _brute.codebook(mask)}
        for trial in range(200):
            alpha = _int_llr(rng, N, -6, 6)
            for llr in (alpha, alpha.astype(np.int8)):
                x, ops, _ = oracle.fastssc_decode(mask, llr, trace=True)
                assert tuple(x) in cb
                assert _brute.correlation(x, alpha) == _brute.ml_best_metric(mask, alpha)
                if N > 2 or name in ("R0", "R1"):
                    expect = {"R0": "R0", "R1": "Info", "Rep": "Rep", "SPC": "SPC"}[name]
                    assert ops == [(expect, N, 0)]


def test_rep_tie_decides_zero():
    """Repetition: a sum >= 0 decides 0, so a zero sum gives the all-zero word."""
    mask = _single_node_masks(4)["Rep"]
    x = oracle.fastssc_decode(mask, np.array([2, -3, 1, 0], np.float32))
    assert x.tolist() == [0, 0, 0, 0]


def test_size2_frozen_info_is_repetition():
    """[frozen, info] fits both Repetition and SPC; it is decoded as Repetition."""
    _, ops, _ = oracle.fastssc_decode(np.array([1, 0], np.uint8), np.array([1, -1], np.float32),
                                      trace=True)
    assert ops == [("Rep", 2, 0)]


def test_spc_lowest_index_tie_break_golden():
    for r in _rows("spc_tiebreak.txt"):
        a, b = r.split("|")
        alpha = np.array([float(v) for v in a.split()], np.float32)
        want = [int(v) for v in b.split()]
        mask = _single_node_masks(alpha.size)["SPC"]
        assert oracle.fastssc_decode(mask, alpha).tolist() == want, r
        assert oracle.fastssc_decode(mask, alpha.astype(np.int8)).tolist() == want, r


# ---------------------------------------------------------------- schedule order

def test_listing1_operation_sequence():
    rows = _rows("listing1_8_5.txt")
    frozen_idx = [int(v) for v in rows[0].split()[1:]]
    mask = np.zeros(8, np.uint8)
    mask[frozen_idx] = 1
    want = [(r.split()[0], int(r.split()[1])) for r in rows[1:]]
    _, ops, _ = oracle.fastssc_decode(mask, np.ones(8, np.float32), trace=True)
    assert [(o[0], o[1]) for o in ops] == want


def test_fig3_node_classification():
    """Fig. 3c: the left N=4 node of the (8,5) code is Rate-0 | Rate-1 and the right
    one is SPC; the Rate-1 child sits at leaves 2-3 and the SPC node at 4-7."""
    mask = np.array([1, 1, 0, 0, 1, 0, 0, 0], np.uint8)
    _, ops, _ = oracle.fastssc_decode(mask, np.ones(8, np.float32), trace=True)
    assert ("Info", 2, 2) in ops and ("SPC", 4, 4) in ops


# ---------------------------------------------------------------- whole decoders

@pytest.mark.parametrize("N,K,db", [(8, 5, None), (64, 32, 2.0), (1024, 512, 2.5),
                                    (2048, 1723, 3.0), (32768, 29492, 4.0)])
def test_noiseless_round_trip(N, K, db):
    """Large correct-sign LLRs: every decoder returns the transmitted data."""
    if db is None:
        mask = np.array([1, 1, 0, 0, 1, 0, 0, 0], np.uint8)
    else:
        mask = synth.frozen_mask(N, K, db)
    rng = np.random.default_rng(3)
    d = rng.integers(0, 2, K).astype(np.uint8)
    x = oracle.encode_systematic(mask, d)
    llr = (1.0 - 2.0 * x.astype(np.float32)) * 4.0
    for dec in (lambda m, l: oracle.fastssc_decode(m, l),
                lambda m, l: oracle.fastssc_decode(m, l, max_spc=0),
                lambda m, l: oracle.fastssc_decode(m, l, max_rep=0, max_spc=0),
                oracle.sc_decode):
        for l in (llr, llr.astype(np.int8)):
            xh = dec(mask, l)
            assert np.array_equal(xh, x)
            assert np.array_equal(oracle.extract_info(mask, xh), synth.pack_bits(d))


@pytest.mark.parametrize("N,K,db", [(64, 40, 1.0), (1024, 512, 2.5), (2048, 1723, 3.0)])
def test_fastssc_without_spc_equals_sc_on_awgn(N, K, db):
    """With SPC disabled every Fast-SSC node (Rate-0, Rate-1, Repetition) gives SC's
    result when no LLR is exactly zero; continuous AWGN LLRs make zeros absent."""
    mask = synth.frozen_mask(N, K, db)
    rng = np.random.default_rng(4)
    d = synth.info_bits(rng, 30, K)
    cw = np.stack([oracle.encode_systematic(mask, r) for r in d])
    llr = synth.awgn_llr(rng, cw, db - 1.0, K / N)
    for y in llr:
        a = oracle.fastssc_decode(mask, y, max_spc=0)
        b = oracle.sc_decode(mask, y)
        assert np.array_equal(a, b)
        c = oracle.fastssc_decode(mask, y, max_rep=0, max_spc=0)
        assert np.array_equal(c, b)


def test_rep_code_int8_fastssc_equals_sc_with_saturation():
    """Repetition-only codes: the saturating fold equals SC's saturating G_0R chain,
    bit for bit, even with large int8 LLRs (saturation active) and zeros."""
    rng = np.random.default_rng(5)
    for N in (2, 8, 64, 512):
        mask = np.ones(N, np.uint8)
        mask[-1] = 0
        for _ in range(100):
            y = rng.integers(-127, 128, N).astype(np.int8)
            assert np.array_equal(oracle.fastssc_decode(mask, y), oracle.sc_decode(mask, y))


@pytest.mark.parametrize("N,K,db", [(256, 128, 1.0), (1024, 512, 2.0)])
def test_outputs_are_codewords(N, K, db):
    """Every node decoder outputs a constituent codeword and Combine is the
    encoder's butterfly, so x_hat G has zeros on the frozen set."""
    mask = synth.frozen_mask(N, K, db)
    rng = np.random.default_rng(6)
    llr = synth.awgn_llr(rng, np.zeros((20, N), np.uint8), db - 2.0, K / N)
    for y in llr:
        for xh in (oracle.fastssc_decode(mask, y), oracle.sc_decode(mask, y),
                   oracle.fastssc_decode(mask, synth.quantize_i8(y))):
            assert not oracle.encode(xh)[mask == 1].any()


def test_int8_equals_float_without_saturation():
    """Small integer LLRs on N = 16: int8 and float32 decoders do the same integer
    arithmetic (no sum reaches 127), so outputs and traces agree exactly."""
    rng = np.random.default_rng(8)
    for _ in range(300):
        K = int(rng.integers(0, 17))
        mask = _random_mask(rng, 16, K)
        y = _int_llr(rng, 16, -7, 7)
        a, oa, aa = oracle.fastssc_decode(mask, y, trace=True)
        b, ob, ab = oracle.fastssc_decode(mask, y.astype(np.int8), trace=True)
        assert np.array_equal(a, b) and oa == ob and np.array_equal(aa, ab)


def test_ml_fer_not_worse_than_fastssc_n16():
    """Statistical sanity: brute-force ML errs no more often than Fast-SSC."""
    mask = synth.frozen_mask(16, 8, 2.0)
    cb = _brute.codebook(mask)
    rng = np.random.default_rng(9)
    cw = np.zeros((400, 16), np.uint8)
    llr = synth.awgn_llr(rng, cw, 1.0, 0.5)
    ml_err = fs_err = 0
    for y in llr:
        best = cb[np.argmax(_brute.correlation(cb, y))]
        ml_err += int(best.any())
        fs_err += int(oracle.fastssc_decode(mask, y).any())
    assert ml_err <= fs_err
    assert fs_err < 200  # far below a coin flip at this SNR


def test_batch_decode_matches_single():
    mask = synth.frozen_mask(256, 128, 3.0)
    rng = np.random.default_rng(10)
    d = synth.info_bits(rng, 16, 128)
    cw = np.stack([oracle.encode_systematic(mask, r) for r in d])
    llr = synth.awgn_llr(rng, cw, 3.0, 0.5)
    out = oracle.decode_batch(mask, llr)
    for f in range(16):
        assert np.array_equal(out[f], oracle.extract_info(mask, oracle.fastssc_decode(mask, llr[f])))
    assert np.array_equal(oracle.decode_batch(mask, llr, algo="sc")[3],
                          oracle.extract_info(mask, oracle.sc_decode(mask, llr[3])))


def _repspc_mask(n):
    """Node of n leaves: left half a Repetition code (only its last leaf carries
    information), right half an SPC code (only its first leaf frozen)."""
    h = n // 2
    m = np.zeros(n, np.uint8)
    m[: h - 1] = 1
    m[h] = 1
    return m


@pytest.mark.parametrize("n", [8, 16, 32, 64])
def test_repspc_speculative_equals_sequential(n):
    """Sec. II-D: the speculative Repetition-SPC decode (Repetition and two SPC
    hypotheses in parallel, then a selection) gives what the plain Fast-SSC
    order F, Repetition, G, SPC, Combine gives on the same node, for float32
    and for saturating int8 LLRs (ties and +-127 included); both Repetition
    outcomes occur in the sample, so a swapped selection would fail."""
    mask = _repspc_mask(n)
    rng = np.random.default_rng(n)
    _, ops, _ = oracle.fastssc_decode(mask, rng.standard_normal(n).astype(np.float32), trace=True)
    assert [o[0] for o in ops] == ["F", "Rep", "G", "SPC", "Combine"]
    reps = set()
    for t in range(400):
        if t % 2:
            y = rng.integers(-127, 128, n).astype(np.int8)
            if t % 4 == 1:
                y[rng.integers(0, n, 3)] = rng.choice([-127, 127, 0], 3).astype(np.int8)
        else:
            y = (rng.standard_normal(n) * 2 + rng.choice([-1, 1])).astype(np.float32)
        got = oracle.repspc(y)
        assert np.array_equal(got, oracle.fastssc_decode(mask, y)), (n, t)
        reps.add(int(got[0] ^ got[n // 2]))  # left = decision XOR right (Eq. 3)
        assert not oracle.encode(got)[mask == 1].any()  # a codeword of the node's code
    assert len(reps) == 2


def test_repspc_rejects_bad_size():
    with pytest.raises(RuntimeError):
        oracle.repspc(np.zeros(4, np.float32))
    with pytest.raises(RuntimeError):
        oracle.repspc(np.zeros(12, np.float32))
