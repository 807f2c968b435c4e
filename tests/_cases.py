"""Seeded test workloads: codewords from the oracle's encoder, channel from synth."""
from __future__ import annotations

import numpy as np

import oracle
from paper_1504_00353_gb300 import synth


def frames(N, K, design_db, n, seed, ebn0_db=None, distinct=None, mask=None):
    """(mask, info bits [n, K], float32 LLRs [n, N]) for BPSK-AWGN frames.

    ``distinct`` limits how many different codewords are encoded (they are then
    repeated with fresh noise), which keeps large cases quick to build."""
    if mask is None:
        mask = synth.frozen_mask(N, K, design_db)
    rng = np.random.default_rng(seed)
    m = n if distinct is None else min(n, distinct)
    d = synth.info_bits(rng, m, K)
    cw = np.stack([oracle.encode_systematic(mask, r) for r in d]) if K else np.zeros((m, N), np.uint8)
    if m < n:
        idx = np.arange(n) % m
        d, cw = d[idx], cw[idx]
    llr = synth.awgn_llr(rng, cw, design_db if ebn0_db is None else ebn0_db, max(K, 1) / N)
    return mask, d, llr


def random_mask(rng, N, K):
    m = np.ones(N, np.uint8)
    if K:
        m[rng.choice(N, K, replace=False)] = 0
    return m
