"""Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
as 1, 2, 3", SC 2011) written from its published definition, for the tests of
the GPU chain: the same counters and keys must give the same words."""
import numpy as np

M0, M1 = 0xD2511F53, 0xCD9E8D57
W0, W1 = 0x9E3779B9, 0xBB67AE85
MASK = 0xFFFFFFFF


def philox(ctr, key):
    """Ten rounds on one 4-word counter with a 2-word key."""
    c = [int(v) & MASK for v in ctr]
    k0, k1 = int(key[0]) & MASK, int(key[1]) & MASK
    for r in range(10):
        if r:
            k0, k1 = (k0 + W0) & MASK, (k1 + W1) & MASK
        p0, p1 = M0 * c[0], M1 * c[2]
        c = [((p1 >> 32) ^ c[1] ^ k0) & MASK, p1 & MASK, ((p0 >> 32) ^ c[3] ^ k1) & MASK, p0 & MASK]
    return c


def philox_np(ctr, key):
    """Vectorised over rows of ctr (uint32 [n, 4]); key is two ints."""
    c = [ctr[:, i].astype(np.uint64) for i in range(4)]
    k0, k1 = np.uint64(key[0] & MASK), np.uint64(key[1] & MASK)
    m = np.uint64(MASK)
    for r in range(10):
        if r:
            k0, k1 = (k0 + np.uint64(W0)) & m, (k1 + np.uint64(W1)) & m
        p0 = np.uint64(M0) * c[0]
        p1 = np.uint64(M1) * c[2]
        c = [((p1 >> np.uint64(32)) ^ c[1] ^ k0) & m, p1 & m, ((p0 >> np.uint64(32)) ^ c[3] ^ k1) & m,
             p0 & m]
    return np.stack(c, axis=1).astype(np.uint32)


def counters(n_words, frame, stream):
    j = np.arange(n_words, dtype=np.uint64)
    f = np.uint64(frame)
    return np.stack([j, np.full_like(j, f & np.uint64(MASK)), np.full_like(j, f >> np.uint64(32)),
                     np.full_like(j, stream)], axis=1).astype(np.uint32)


def info_bytes(K, seed, frame):
    """The information-bit row polar_random_info writes for one frame."""
    row = (K + 7) // 8
    words = philox_np(counters((row + 15) // 16, frame, 1), (seed & MASK, seed >> 32))
    b = words.astype("<u4").view(np.uint8).reshape(-1)[:row].copy()
    if K % 8:
        b[-1] &= (1 << (K % 8)) - 1
    return b


def normals(N, seed, frame):
    """The N Box-Muller normals polar_channel_awgn uses for one frame (float64)."""
    w = philox_np(counters((N + 3) // 4, frame, 2), (seed & MASK, seed >> 32)).astype(np.float32)
    # the uniforms as the device forms them, in float32: (word + 1) 2^-32 and word 2^-32
    s = np.float32(2.0 ** -32)
    u = [((w[:, 0] + np.float32(1)) * s), w[:, 1] * s, ((w[:, 2] + np.float32(1)) * s), w[:, 3] * s]
    u1a, u2a, u1b, u2b = (x.astype(np.float64) for x in u)
    ra, rb = np.sqrt(-2 * np.log(u1a)), np.sqrt(-2 * np.log(u1b))
    z = np.stack([ra * np.cos(2 * np.pi * u2a), ra * np.sin(2 * np.pi * u2a),
                  rb * np.cos(2 * np.pi * u2b), rb * np.sin(2 * np.pi * u2b)], axis=1)
    return z.reshape(-1)[:N]
