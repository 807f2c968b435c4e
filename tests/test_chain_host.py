"""Host pins for the GPU chain's random-number generator (no GPU needed)."""
import numpy as np

from tests import _philox


def test_philox_known_answers():
    """Known-answer vectors of Philox-4x32-10 (the published reference set):
    zero counter and key, all-ones, and the digits of pi."""
    assert _philox.philox([0, 0, 0, 0], [0, 0]) == [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]
    assert _philox.philox([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2) == [0x408F276D, 0x41C83B0E,
                                                                  0xA20BC7C6, 0x6D5451FD]
    assert _philox.philox([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344],
                          [0xA4093822, 0x299F31D0]) == [0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]


def test_vectorised_equals_scalar():
    rng = np.random.default_rng(0)
    ctr = rng.integers(0, 2 ** 32, (50, 4), dtype=np.uint64).astype(np.uint32)
    key = (int(rng.integers(0, 2 ** 32)), int(rng.integers(0, 2 ** 32)))
    v = _philox.philox_np(ctr, key)
    for i in range(50):
        assert list(v[i]) == _philox.philox(ctr[i], key)


def test_normals_moments():
    z = np.concatenate([_philox.normals(4096, 7, f) for f in range(16)])
    assert abs(z.mean()) < 0.02 and abs(z.var() - 1) < 0.03
