"""Seeded synthetic inputs: code construction, random information bits, BPSK-AWGN.

This module feeds both the GPU decoder and the CPU oracle. It holds none of the
decoder's arithmetic (no F/G/Combine, no node decoder, no encoder); it chooses
the frozen set, draws bits and noise, and maps codeword bits to channel LLRs.

Readings where the paper is silent (Sec. III, "BPSK over an AWGN channel with
random codewords"; the paper's own codes follow Tal-Vardy, which the
workloads here replace by the Bhattacharyya recursion):

* Construction: ln Z_0 = -R * 10^(EbN0/10) (Bhattacharyya parameter of
  BPSK-AWGN, exp(-Es/N0) with Es = R*Eb). In natural index order the most
  significant index bit is the channel-level split: bit 0 takes
  Z- = 2Z - Z^2, bit 1 takes Z+ = Z^2. Computed in float64 logs, since Z^(2^20)
  underflows. The N-K largest ln Z are frozen; among equal values the lower
  index is frozen first.
* Channel: x -> s = 1 - 2x, y = s + sigma*n with sigma^2 = 1/(2 R 10^(EbN0/10)),
  LLR = 2y/sigma^2 rounded once to float32.
* int8 LLRs: q = clamp(rint(8 * llr32), -127, 127) with round-half-even, so -128
  never occurs.
* Random numbers: numpy PCG64 (default_rng(seed)); information bits are drawn
  first, then the noise, from the same generator.
"""
from __future__ import annotations

import numpy as np


def bhattacharyya_lnz(N: int, design_ebn0_db: float, rate: float) -> np.ndarray:
    """ln Z of every bit-channel, natural index order (float64)."""
    if N < 1 or N & (N - 1):
        raise ValueError("N must be a power of two")
    lz = np.array([-rate * 10.0 ** (design_ebn0_db / 10.0)], dtype=np.float64)
    while lz.size < N:
        # ln(2Z - Z^2) = ln Z + ln(2 - Z), with 2 - Z = 1 + (1 - Z) = 1 - expm1(ln Z)
        minus = lz + np.log1p(-np.expm1(lz))
        plus = 2.0 * lz
        # children of node with prefix p: index 2p (bit 0 = minus) and 2p+1 (plus);
        # appending bits on the right makes the first split the MSB.
        nxt = np.empty(lz.size * 2, dtype=np.float64)
        nxt[0::2] = minus
        nxt[1::2] = plus
        lz = nxt
    return lz


def frozen_mask(N: int, K: int, design_ebn0_db: float) -> np.ndarray:
    """uint8[N], 1 = frozen: the N-K least reliable bit-channels."""
    if not 0 <= K <= N:
        raise ValueError("need 0 <= K <= N")
    lz = bhattacharyya_lnz(N, design_ebn0_db, K / N)
    # sort by ln Z descending, ties by index ascending (lower index frozen first)
    order = np.lexsort((np.arange(N), -lz))
    mask = np.zeros(N, dtype=np.uint8)
    mask[order[: N - K]] = 1
    return mask


def sigma2(ebn0_db: float, rate: float) -> float:
    return 1.0 / (2.0 * rate * 10.0 ** (ebn0_db / 10.0))


def info_bits(rng: np.random.Generator, n_frames: int, K: int) -> np.ndarray:
    """Uniform information bits, uint8[n_frames, K]."""
    return rng.integers(0, 2, size=(n_frames, K), dtype=np.uint8)


def pack_bits(bits: np.ndarray) -> np.ndarray:
    """[..., K] bytes of 0/1 -> [..., ceil(K/8)] packed LSB first."""
    return np.packbits(np.asarray(bits, dtype=np.uint8), axis=-1, bitorder="little")


def unpack_bits(packed: np.ndarray, K: int) -> np.ndarray:
    return np.unpackbits(np.asarray(packed, dtype=np.uint8), axis=-1, count=K,
                         bitorder="little")


def awgn_llr(rng: np.random.Generator, codewords: np.ndarray, ebn0_db: float,
             rate: float, chunk: int = 1 << 22) -> np.ndarray:
    """BPSK over AWGN; codewords uint8[n, N] (0/1) -> float32 LLRs [n, N]."""
    cw = np.asarray(codewords, dtype=np.uint8)
    s2 = sigma2(ebn0_db, rate)
    sigma = np.sqrt(s2)
    out = np.empty(cw.shape, dtype=np.float32)
    flat_in = cw.reshape(-1)
    flat_out = out.reshape(-1)
    for s in range(0, flat_in.size, chunk):
        e = min(flat_in.size, s + chunk)
        y = (1.0 - 2.0 * flat_in[s:e].astype(np.float64)) + sigma * rng.standard_normal(e - s)
        flat_out[s:e] = (2.0 / s2) * y
    return out


def awgn_llr_mixed(rng: np.random.Generator, codewords: np.ndarray,
                   ebn0_db: np.ndarray, rate: float) -> np.ndarray:
    """Per-frame Eb/N0 (dB) variant of awgn_llr."""
    cw = np.asarray(codewords, dtype=np.uint8)
    s2 = 1.0 / (2.0 * rate * 10.0 ** (np.asarray(ebn0_db, dtype=np.float64) / 10.0))
    y = (1.0 - 2.0 * cw.astype(np.float64)) + np.sqrt(s2)[:, None] * rng.standard_normal(cw.shape)
    return ((2.0 / s2)[:, None] * y).astype(np.float32)


def quantize_i8(llr: np.ndarray, scale: float = 8.0) -> np.ndarray:
    """int8 LLRs: clamp(rint(scale * llr), -127, 127), round half to even."""
    q = np.rint(np.asarray(llr, dtype=np.float64) * scale)
    return np.clip(q, -127, 127).astype(np.int8)


def bits_from_packed_codewords(packed: np.ndarray, N: int) -> np.ndarray:
    return unpack_bits(packed, N)


# Workloads named by what they are (code, channel, size).
# Mixed-length set: frames drawn uniformly from these codes, every frozen set
# by the construction above at MIXED_DESIGN_DB, channel at the same Eb/N0.
MIXED_CODES = [(256, 128), (1024, 512), (2048, 1723), (16384, 14746), (32768, 29492)]
MIXED_DESIGN_DB = 3.0
MIXED_FRAMES = 65536

WORKLOADS = {
    "n1024_k512_2.5db": dict(N=1024, K=512, design_db=2.5, ebn0_db=2.5, seed=0,
                             n_frames=10000),
    "n32768_k29492_4.0db": dict(N=32768, K=29492, design_db=4.0, ebn0_db=4.0, seed=2,
                                n_frames=4096),
    "n1048576_k880804_3.5db": dict(N=1 << 20, K=880804, design_db=3.5, ebn0_db=3.5,
                                   seed=5, n_frames=64),
}
