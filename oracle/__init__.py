"""Plain CPU oracle for Fast-SSC decoding of systematic polar codes.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package. The GPU
library never imports, links or executes anything here, and this package
imports nothing from the GPU library.

The arithmetic lives in ``polar_oracle.c`` (plain C, compiled with
``-O2 -ffp-contract=off``, no fast-math). This module only compiles it and
marshals numpy arrays into it with ctypes.

Citations are to Giard et al., "Low-Latency Software Polar Decoders"
(arXiv 1504.00353): Sec. II-A (G_N), Eqs. 1-3 (SC), Sec. II-D (Fast-SSC
nodes, Eq. 4), Listing 1 (operation order), Listing 2 (SPC tie-break),
Sec. III-A and Listing 4 (saturating int8 G).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "polar_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OP_NAMES = ["F", "G", "G_0R", "Combine", "Combine_0R", "R0", "Info", "Rep", "SPC"]
UNLIMITED = 0xFFFFFFFF


def build(force: bool = False) -> str:
    """Compile polar_oracle.c into liboracle.so next to it (gcc, plain C11)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "polar_oracle.h"))
    ):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = [
        "gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
        "-fno-fast-math", "-Wall", "-Wextra", "-o", tmp, _SRC,
    ]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Trace(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.POINTER(ctypes.c_uint32)),
        ("nv", ctypes.POINTER(ctypes.c_uint32)),
        ("off", ctypes.POINTER(ctypes.c_uint32)),
        ("alpha", ctypes.POINTER(ctypes.c_float)),
        ("cap_ops", ctypes.c_size_t),
        ("cap_alpha", ctypes.c_size_t),
        ("n_ops", ctypes.c_size_t),
        ("n_alpha", ctypes.c_size_t),
        ("overflow", ctypes.c_int),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            u8p = ctypes.POINTER(ctypes.c_uint8)
            i8p = ctypes.POINTER(ctypes.c_int8)
            fp = ctypes.POINTER(ctypes.c_float)
            u32 = ctypes.c_uint32
            L.oracle_encode.argtypes = [u32, u8p, u8p]
            L.oracle_encode.restype = None
            L.oracle_encode_systematic.argtypes = [u32, u8p, u8p, u8p]
            L.oracle_sc_decode_f32.argtypes = [u32, u8p, fp, u8p]
            L.oracle_sc_decode_i8.argtypes = [u32, u8p, i8p, u8p]
            L.oracle_fastssc_decode_f32.argtypes = [u32, u8p, fp, u32, u32, u8p,
                                                    ctypes.POINTER(_Trace)]
            L.oracle_fastssc_decode_i8.argtypes = [u32, u8p, i8p, u32, u32, u8p,
                                                   ctypes.POINTER(_Trace)]
            L.oracle_extract_info.argtypes = [u32, u8p, u8p, u8p]
            L.oracle_extract_info.restype = None
            L.oracle_decode_batch_f32.argtypes = [u32, u8p, fp, ctypes.c_size_t,
                                                  ctypes.c_int, u32, u32, u8p]
            L.oracle_decode_batch_i8.argtypes = [u32, u8p, i8p, ctypes.c_size_t,
                                                 ctypes.c_int, u32, u32, u8p]
            L.oracle_f_f32.argtypes = [ctypes.c_float, ctypes.c_float]
            L.oracle_f_f32.restype = ctypes.c_float
            L.oracle_g_f32.argtypes = [ctypes.c_float, ctypes.c_float, ctypes.c_uint8]
            L.oracle_g_f32.restype = ctypes.c_float
            L.oracle_f_i8.argtypes = [ctypes.c_int8, ctypes.c_int8]
            L.oracle_f_i8.restype = ctypes.c_int8
            L.oracle_g_i8.argtypes = [ctypes.c_int8, ctypes.c_int8, ctypes.c_uint8]
            L.oracle_g_i8.restype = ctypes.c_int8
            L.oracle_repspc_f32.argtypes = [fp, u32, u8p]
            L.oracle_repspc_i8.argtypes = [i8p, u32, u8p]
            _lib = L
        return _lib


def _p(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _mask(frozen) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(frozen, dtype=np.uint8))


def encode(u) -> np.ndarray:
    """x = u * F_2^{(x)n} (Sec. II-A), one byte per bit."""
    u = np.ascontiguousarray(np.asarray(u, dtype=np.uint8))
    x = np.empty_like(u)
    lib().oracle_encode(u.size, _p(u, ctypes.c_uint8), _p(x, ctypes.c_uint8))
    return x


def encode_systematic(frozen, d) -> np.ndarray:
    """Systematic codeword whose information positions carry d (K bytes)."""
    m = _mask(frozen)
    d = np.ascontiguousarray(np.asarray(d, dtype=np.uint8))
    assert d.size == int((m == 0).sum())
    x = np.empty(m.size, dtype=np.uint8)
    rc = lib().oracle_encode_systematic(m.size, _p(m, ctypes.c_uint8),
                                        _p(d, ctypes.c_uint8), _p(x, ctypes.c_uint8))
    if rc != 0:
        raise ValueError("mask is not systematic-encodable by the two-step encoder")
    return x


def sc_decode(frozen, llr) -> np.ndarray:
    """Plain SC (Eqs. 1-3); returns the codeword estimate, one byte per bit."""
    m = _mask(frozen)
    x = np.empty(m.size, dtype=np.uint8)
    if np.asarray(llr).dtype == np.int8:
        y = np.ascontiguousarray(llr, dtype=np.int8)
        rc = lib().oracle_sc_decode_i8(m.size, _p(m, ctypes.c_uint8), _p(y, ctypes.c_int8),
                                       _p(x, ctypes.c_uint8))
    else:
        y = np.ascontiguousarray(llr, dtype=np.float32)
        rc = lib().oracle_sc_decode_f32(m.size, _p(m, ctypes.c_uint8),
                                        _p(y, ctypes.c_float), _p(x, ctypes.c_uint8))
    if rc != 0:
        raise RuntimeError(f"oracle SC failed: {rc}")
    return x


def fastssc_decode(frozen, llr, max_rep=UNLIMITED, max_spc=UNLIMITED, trace=False):
    """Plain recursive Fast-SSC (Sec. II-D).

    Returns the codeword estimate, or (estimate, ops, alphas) when trace is set:
    ops is a list of (name, N_v, offset) in execution order and alphas the
    concatenated F/G/G_0R outputs (float32; int8 values for int8 input).
    """
    m = _mask(frozen)
    N = m.size
    x = np.empty(N, dtype=np.uint8)
    tr_ptr = None
    if trace:
        cap_ops = 4 * N + 8
        cap_alpha = 2 * N * max(1, int(np.log2(N)) + 1)
        kind = np.zeros(cap_ops, np.uint32)
        nv = np.zeros(cap_ops, np.uint32)
        off = np.zeros(cap_ops, np.uint32)
        alpha = np.zeros(cap_alpha, np.float32)
        tr = _Trace(_p(kind, ctypes.c_uint32), _p(nv, ctypes.c_uint32),
                    _p(off, ctypes.c_uint32), _p(alpha, ctypes.c_float),
                    cap_ops, cap_alpha, 0, 0, 0)
        tr_ptr = ctypes.byref(tr)
    if np.asarray(llr).dtype == np.int8:
        y = np.ascontiguousarray(llr, dtype=np.int8)
        rc = lib().oracle_fastssc_decode_i8(N, _p(m, ctypes.c_uint8), _p(y, ctypes.c_int8),
                                            max_rep, max_spc, _p(x, ctypes.c_uint8), tr_ptr)
    else:
        y = np.ascontiguousarray(llr, dtype=np.float32)
        rc = lib().oracle_fastssc_decode_f32(N, _p(m, ctypes.c_uint8),
                                             _p(y, ctypes.c_float), max_rep, max_spc,
                                             _p(x, ctypes.c_uint8), tr_ptr)
    if rc != 0:
        raise RuntimeError(f"oracle Fast-SSC failed: {rc}")
    if not trace:
        return x
    ops = [(OP_NAMES[kind[i]], int(nv[i]), int(off[i])) for i in range(tr.n_ops)]
    return x, ops, alpha[: tr.n_alpha].copy()


def extract_info(frozen, xhat) -> np.ndarray:
    """Packed information bits x_hat[A] (LSB first), ceil(K/8) bytes."""
    m = _mask(frozen)
    xhat = np.ascontiguousarray(xhat, dtype=np.uint8)
    K = int((m == 0).sum())
    out = np.zeros((K + 7) // 8, dtype=np.uint8)
    lib().oracle_extract_info(m.size, _p(m, ctypes.c_uint8), _p(xhat, ctypes.c_uint8),
                              _p(out, ctypes.c_uint8))
    return out


def decode_batch(frozen, llr, algo="fastssc", max_rep=UNLIMITED, max_spc=UNLIMITED,
                 frames=None) -> np.ndarray:
    """Decode llr[n, N] frame by frame; returns packed info bits [n, ceil(K/8)].

    ``frames`` restricts the work to a slice of rows (returns only those rows).
    The C loop runs without the GIL, so several Python threads may call this
    on disjoint slices at once.
    """
    m = _mask(frozen)
    N = m.size
    K = int((m == 0).sum())
    arr = np.asarray(llr)
    if frames is not None:
        arr = arr[frames]
    arr = arr.reshape(-1, N)
    n = arr.shape[0]
    out = np.zeros((n, (K + 7) // 8), dtype=np.uint8)
    a = 1 if algo == "sc" else 0
    if arr.dtype == np.int8:
        y = np.ascontiguousarray(arr)
        rc = lib().oracle_decode_batch_i8(N, _p(m, ctypes.c_uint8), _p(y, ctypes.c_int8), n,
                                          a, max_rep, max_spc, _p(out, ctypes.c_uint8))
    else:
        y = np.ascontiguousarray(arr, dtype=np.float32)
        rc = lib().oracle_decode_batch_f32(N, _p(m, ctypes.c_uint8), _p(y, ctypes.c_float),
                                           n, a, max_rep, max_spc, _p(out, ctypes.c_uint8))
    if rc != 0:
        raise RuntimeError(f"oracle batch decode failed: {rc}")
    return out


def f_f32(a, b):
    return lib().oracle_f_f32(a, b)


def g_f32(a, b, beta):
    return lib().oracle_g_f32(a, b, beta)


def f_i8(a, b):
    return lib().oracle_f_i8(a, b)


def g_i8(a, b, beta):
    return lib().oracle_g_i8(a, b, beta)


def repspc(llr) -> np.ndarray:
    """Speculative Repetition-SPC node decode (Sec. II-D) of one node's LLRs
    (float32, or int8 for the saturating decoder): its n estimates."""
    n = np.asarray(llr).size
    beta = np.empty(n, dtype=np.uint8)
    if np.asarray(llr).dtype == np.int8:
        y = np.ascontiguousarray(llr, dtype=np.int8)
        rc = lib().oracle_repspc_i8(_p(y, ctypes.c_int8), n, _p(beta, ctypes.c_uint8))
    else:
        y = np.ascontiguousarray(llr, dtype=np.float32)
        rc = lib().oracle_repspc_f32(_p(y, ctypes.c_float), n, _p(beta, ctypes.c_uint8))
    if rc != 0:
        raise RuntimeError(f"oracle Repetition-SPC failed: {rc}")
    return beta
