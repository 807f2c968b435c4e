"""CPU-only checks of the C ABI library: it loads, exports every declared symbol,
and its host logic (operation-list compiler, systematic encoder, argument
validation) agrees with the oracle and the paper. No kernel is launched."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from paper_1504_00353_gb300 import build, polar, synth
from tests import _cases

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLDEN = os.path.join(ROOT, "tests", "golden")


def test_header_declares_exactly_the_exported_entry_points():
    hdr = open(os.path.join(ROOT, "include", "polar_gb300.h")).read()
    declared = set(re.findall(r"\b(polar_[a-z0-9_]+)\s*\(", hdr))
    assert declared == set(polar.EXPORTS)
    L = ctypes.CDLL(build.LIB)
    for name in declared:
        assert hasattr(L, name), name


def test_library_is_in_tree_and_built_for_sm103a():
    assert os.path.dirname(build.LIB) == os.path.join(ROOT, "paper_1504_00353_gb300")
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)


def test_listing1_schedule_from_library():
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "listing1_8_5.txt"))
            if ln.strip() and not ln.startswith("#")]
    mask = np.zeros(8, np.uint8)
    mask[[int(v) for v in rows[0][1:]]] = 1
    code = polar.polar_code_create(8, 5, mask)
    assert [(o[0], o[1]) for o in polar.polar_code_schedule(code)] == [(r[0], int(r[1])) for r in rows[1:]]


@pytest.mark.parametrize("N,K,db", [(256, 128, 3.0), (1024, 512, 2.5), (2048, 1723, 3.0),
                                    (16384, 14746, 3.0), (32768, 29492, 4.0)])
def test_schedule_equals_oracle_recursion(N, K, db):
    mask = synth.frozen_mask(N, K, db)
    code = polar.polar_code_create(N, K, mask)
    _, ops, alpha = oracle.fastssc_decode(mask, np.ones(N, np.float32), trace=True)
    assert polar.polar_code_schedule(code) == ops
    assert polar.polar_code_trace_len(code) == alpha.size


def test_schedule_counts_of_workload_codes():
    """Operation-list lengths of the three workload codes."""
    for (N, K, db), n in [((1024, 512, 2.5), 265), ((32768, 29492, 4.0), 1649),
                          ((1 << 20, 880804, 3.5), 28465)]:
        code = polar.polar_code_create(N, K, synth.frozen_mask(N, K, db))
        assert polar.polar_code_info(code) == (N, K, n)


def test_schedule_random_masks_and_limits():
    rng = np.random.default_rng(11)
    for _ in range(60):
        N = int(2 ** rng.integers(1, 11))
        K = int(rng.integers(0, N + 1))
        mask = _cases.random_mask(rng, N, K)
        mr = int(rng.choice([0, 2, 8, oracle.UNLIMITED]))
        ms = int(rng.choice([0, 4, 64, oracle.UNLIMITED]))
        code = polar.polar_code_create(N, K, mask, max_rep=mr, max_spc=ms)
        _, ops, _ = oracle.fastssc_decode(mask, np.ones(N, np.float32), max_rep=mr,
                                          max_spc=ms, trace=True)
        assert polar.polar_code_schedule(code) == ops


@pytest.mark.parametrize("N,K,db", [(2, 1, 1.0), (4, 2, 1.0), (16, 9, 2.0), (1024, 512, 2.5),
                                    (32768, 29492, 4.0)])
def test_library_encoder_matches_oracle(N, K, db):
    mask = synth.frozen_mask(N, K, db)
    code = polar.polar_code_create(N, K, mask)
    rng = np.random.default_rng(12)
    d = rng.integers(0, 2, (8, K)).astype(np.uint8)
    x = polar.polar_encode_systematic(code, synth.pack_bits(d))
    want = np.stack([oracle.encode_systematic(mask, r) for r in d])
    assert np.array_equal(synth.unpack_bits(x, N), want)


def test_encoder_rejects_non_systematic_mask():
    """A = {0, 1, 3} in N = 8 is not domination-contiguous (0 <= 2 <= 3 bitwise, with
    0 and 3 in A but 2 frozen), so the two-step encoder is not systematic for some
    data; the library reports those data words as errors exactly where the oracle's
    encoder does, instead of returning a codeword whose x[A] differs from d."""
    mask = np.ones(8, np.uint8)
    mask[[0, 1, 3]] = 0
    code = polar.polar_code_create(8, 3, mask)
    bad = 0
    for v in range(8):
        d = np.array([(v >> j) & 1 for j in range(3)], np.uint8)
        try:
            oracle.encode_systematic(mask, d)
            ok_oracle = True
        except ValueError:
            ok_oracle = False
        try:
            polar.polar_encode_systematic(code, synth.pack_bits(d[None]))
            ok_lib = True
        except polar.PolarError as e:
            assert e.status == -1
            ok_lib = False
        assert ok_lib == ok_oracle
        bad += not ok_lib
    assert bad > 0


@pytest.mark.parametrize("N,K,mask", [(3, 1, [1, 0, 0]), (1, 1, [0]), (4, 3, [1, 0, 0, 1]),
                                      (4, 2, [1, 0, 2, 0]), (1 << 21, 0, None)])
def test_create_rejects_bad_arguments(N, K, mask):
    m = np.ones(N, np.uint8) if mask is None else np.array(mask, np.uint8)
    with pytest.raises(polar.PolarError) as e:
        polar.polar_code_create(N, K, m)
    assert e.value.status == -1


def test_status_strings():
    for s in (0, -1, -2, -3, -4, -5):
        assert polar.polar_status_str(s)


def test_public_header_is_plain_c(tmp_path):
    """include/polar_gb300.h is a C header: it compiles as strict C99 with no
    warnings (no C++ or torch types in the boundary)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    src = tmp_path / "h.c"
    src.write_text('#include "polar_gb300.h"\nint main(void) { return 0; }\n')
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only",
                        "-I", inc, str(src)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
