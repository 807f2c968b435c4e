"""Brute-force references for tiny polar codes (N <= 16), plain numpy.

Nothing here shares code with the oracle or the GPU library: the generator
matrix comes from numpy's Kronecker product, and decisions come from
enumerating every input vector u.
"""
from __future__ import annotations

import functools

import numpy as np

F2 = np.array([[1, 0], [1, 1]], dtype=np.int64)


@functools.lru_cache(maxsize=None)
def gen_matrix(N: int) -> np.ndarray:
    """G_N = F_2^{(x) log2 N} (Sec. II-A), as an int64 0/1 matrix."""
    G = np.array([[1]], dtype=np.int64)
    while G.shape[0] < N:
        G = np.kron(G, F2)
    return G


@functools.lru_cache(maxsize=None)
def all_inputs(N: int) -> np.ndarray:
    """Every u in {0,1}^N, row r has u_j = bit (N-1-j) of r (u_0 is the MSB)."""
    r = np.arange(1 << N, dtype=np.int64)
    return ((r[:, None] >> (N - 1 - np.arange(N))[None, :]) & 1).astype(np.int64)


@functools.lru_cache(maxsize=None)
def all_codewords_signs(N: int) -> np.ndarray:
    """(1 - 2x) for x = u G_N over every u, as float64 rows (same row order)."""
    X = (all_inputs(N) @ gen_matrix(N)) % 2
    return (1.0 - 2.0 * X).astype(np.float64)


def encode(u) -> np.ndarray:
    u = np.asarray(u, dtype=np.int64)
    return ((u @ gen_matrix(u.shape[-1])) % 2).astype(np.uint8)


def codebook(frozen) -> np.ndarray:
    """All codewords of the code (frozen positions of u set to 0)."""
    frozen = np.asarray(frozen, dtype=bool)
    N = frozen.size
    U = all_inputs(N)
    keep = ~(U[:, frozen].any(axis=1))
    return ((U[keep] @ gen_matrix(N)) % 2).astype(np.uint8)


def correlation(x, alpha) -> np.ndarray:
    """sum_i (1 - 2 x_i) alpha_i (float64)."""
    x = np.asarray(x, dtype=np.float64)
    return (1.0 - 2.0 * x) @ np.asarray(alpha, dtype=np.float64)


def ml_best_metric(frozen, alpha) -> float:
    cb = codebook(frozen)
    return float(np.max(correlation(cb, alpha)))


def sequential_maxlog(frozen, alpha) -> np.ndarray:
    """Bit-by-bit max-log decisions in index order.

    For i = 0..N-1: u_i = 0 if frozen, else 0 when
    max{corr(uG) : u_<i = decided, u_i = 0, u_>i free} >=
    max{corr(uG) : u_<i = decided, u_i = 1, u_>i free}, else 1.
    Returns the codeword u G. With min-sum F this is what SC computes exactly:
    min(|a|,|b|) sgn(a) sgn(b) = (|a+b| - |a-b|)/2 is the max-log marginal of a
    XOR of two bits, and the SC recursion is exact on its tree.
    """
    frozen = np.asarray(frozen, dtype=bool)
    N = frozen.size
    metric = all_codewords_signs(N) @ np.asarray(alpha, dtype=np.float64)
    prefix = 0
    u = np.zeros(N, dtype=np.int64)
    for i in range(N):
        width = 1 << (N - i)          # block of inputs sharing the decided prefix
        base = prefix * width
        half = width // 2
        if frozen[i]:
            bit = 0
        else:
            m0 = metric[base: base + half].max()
            m1 = metric[base + half: base + width].max()
            bit = 0 if m0 >= m1 else 1
        u[i] = bit
        prefix = prefix * 2 + bit
    return encode(u)
