"""Python binding of libpolar_gb300 (include/polar_gb300.h), same names as the C ABI.

Argument marshalling only: torch tensors become device pointers, torch streams
become cudaStream_t handles, numpy arrays become host pointers. Every step of
the decode runs in the library's CUDA kernels; there is no CPU or PyTorch
fallback, and importing this module raises if the library is not built.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

UNLIMITED = 0xFFFFFFFF
OP_NAMES = ["F", "G", "G_0R", "Combine", "Combine_0R", "R0", "Info", "Rep", "SPC"]
STATUS = {0: "POLAR_OK", -1: "POLAR_EINVAL", -2: "POLAR_ENOMEM", -3: "POLAR_ECUDA",
          -4: "POLAR_EALIGN", -5: "POLAR_ETIMEOUT"}

# Every symbol include/polar_gb300.h declares.
EXPORTS = [
    "polar_status_str", "polar_code_create", "polar_code_create_ex", "polar_code_destroy",
    "polar_code_info", "polar_code_schedule", "polar_encode_systematic", "polar_decode",
    "polar_decode_i8", "polar_code_trace_len", "polar_decode_trace", "polar_code_set_launch",
    "polar_code_get_launch", "polar_code_check", "polar_code_compile", "polar_code_compile_ex",
    "polar_code_compile_log",
    "polar_decode_noalloc", "polar_batch_create", "polar_batch_create_ex", "polar_batch_destroy",
    "polar_batch_decode",
    "polar_batch_info", "polar_batch_log", "polar_server_create", "polar_server_publish",
    "polar_server_progress", "polar_server_destroy", "polar_random_info",
    "polar_encode_systematic_device", "polar_channel_awgn", "polar_count_errors", "polar_fer_run",
    "polar_decode_host", "polar_selftest_bounded_wait", "polar_code_set_frames_per_cta",
    "polar_code_get_frames_per_cta",
]

# struct polar_request
REQUEST_DTYPE = np.dtype([("code_id", "<u4"), ("reserved", "<u4"), ("llr_off", "<u8"),
                          ("out_off", "<u8")])


class PolarError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {STATUS.get(status, status)} "
                         f"({_lib.polar_status_str(status).decode()})")


def _load():
    path = _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with "
                          "`python -m paper_1504_00353_gb300.build` (or __graft_entry__.build())")
    L = ctypes.CDLL(path)
    vp, u8p, u32p = ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint8), ctypes.POINTER(ctypes.c_uint32)
    u32, sz, st = ctypes.c_uint32, ctypes.c_size_t, ctypes.c_int
    szp = ctypes.POINTER(ctypes.c_size_t)
    sig = {
        "polar_status_str": ([st], ctypes.c_char_p),
        "polar_code_create": ([u32, u32, u8p, ctypes.POINTER(vp)], st),
        "polar_code_create_ex": ([u32, u32, u8p, u32, u32, ctypes.POINTER(vp)], st),
        "polar_code_destroy": ([vp], None),
        "polar_code_info": ([vp, u32p, u32p, u32p], st),
        "polar_code_schedule": ([vp, u32p, u32p, u32p, sz, szp], st),
        "polar_encode_systematic": ([vp, u8p, u8p, sz], st),
        "polar_decode": ([vp, vp, vp, sz, vp], st),
        "polar_decode_i8": ([vp, vp, vp, sz, vp], st),
        "polar_decode_noalloc": ([vp, vp, vp, sz, vp], st),
        "polar_code_trace_len": ([vp], sz),
        "polar_decode_trace": ([vp, vp, st, vp, vp, sz, vp], st),
        "polar_code_set_launch": ([vp, st, u32, u32, u32, u32, u32], st),
        "polar_code_get_launch": ([vp, st, sz, u32p, u32p, u32p, u32p, u32p, u32p, szp, szp, u32p], st),
        "polar_code_compile": ([vp, st, sz, u32], st),
        "polar_code_compile_ex": ([vp, st, sz, u32, u32], st),
        "polar_code_compile_log": ([vp], ctypes.c_char_p),
        "polar_code_check": ([vp, vp], st),
        "polar_batch_create": ([ctypes.POINTER(vp), u32, st, u32, u32p, u32p, u32,
                                ctypes.POINTER(vp)], st),
        "polar_batch_create_ex": ([ctypes.POINTER(vp), u32, st, u32, u32p, u32p, u32, u32,
                                ctypes.POINTER(vp)], st),
        "polar_batch_destroy": ([vp], None),
        "polar_batch_decode": ([vp, vp, vp, vp, vp, vp, sz, vp], st),
        "polar_batch_info": ([vp, u32p, u32p, szp, szp], st),
        "polar_batch_log": ([vp], ctypes.c_char_p),
        "polar_server_create": ([vp, vp, sz, vp, sz, vp, sz, vp, sz, u32, u32, u32,
                                 ctypes.POINTER(vp)], st),
        "polar_server_publish": ([vp, ctypes.c_uint64], st),
        "polar_server_progress": ([vp, ctypes.POINTER(ctypes.c_uint64),
                                   ctypes.POINTER(ctypes.c_uint64),
                                   ctypes.POINTER(ctypes.c_uint64)], st),
        "polar_server_destroy": ([vp], st),
        "polar_random_info": ([vp, vp, sz, ctypes.c_uint64, ctypes.c_uint64, vp], st),
        "polar_decode_host": ([vp, st, vp, vp, sz, sz], st),
        "polar_selftest_bounded_wait": ([vp, u32, vp], st),
        "polar_code_set_frames_per_cta": ([vp, st, u32], st),
        "polar_code_get_frames_per_cta": ([vp, st, sz, u32p], st),
        "polar_encode_systematic_device": ([vp, vp, vp, sz, vp], st),
        "polar_channel_awgn": ([vp, vp, vp, st, sz, ctypes.c_float, ctypes.c_uint64,
                                ctypes.c_uint64, vp], st),
        "polar_count_errors": ([vp, vp, vp, sz, vp, vp], st),
        "polar_fer_run": ([vp, st, ctypes.c_float, ctypes.c_uint64, sz, sz,
                           ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)], st),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    return L


_lib = _load()


def lib():
    return _lib


def _check(status: int, what: str):
    if status != 0:
        raise PolarError(status, what)


class PolarCode:
    """Owns a polar_code_t handle (destroyed with the object)."""

    def __init__(self, handle: int, N: int, K: int, frozen: np.ndarray):
        self.handle = ctypes.c_void_p(handle)
        self.N, self.K = N, K
        self.frozen = frozen
        self.out_row = (K + 7) // 8

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            _lib.polar_code_destroy(h)
            self.handle = ctypes.c_void_p(0)


def polar_code_create(N: int, K: int, frozen_mask, max_rep: int | None = None,
                      max_spc: int | None = None) -> PolarCode:
    m = np.ascontiguousarray(np.asarray(frozen_mask, dtype=np.uint8))
    if m.size != N:
        raise ValueError("frozen_mask must have N entries")
    h = ctypes.c_void_p()
    p = m.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
    if max_rep is None and max_spc is None:
        _check(_lib.polar_code_create(N, K, p, ctypes.byref(h)), "polar_code_create")
    else:
        _check(_lib.polar_code_create_ex(N, K, p, UNLIMITED if max_rep is None else max_rep,
                                         UNLIMITED if max_spc is None else max_spc,
                                         ctypes.byref(h)), "polar_code_create_ex")
    return PolarCode(h.value, N, K, m.copy())


def polar_code_destroy(code: PolarCode):
    code.__del__()


def polar_code_info(code: PolarCode):
    N, K, n = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
    _check(_lib.polar_code_info(code.handle, ctypes.byref(N), ctypes.byref(K), ctypes.byref(n)),
           "polar_code_info")
    return N.value, K.value, n.value


def polar_code_schedule(code: PolarCode):
    """[(name, N_v, offset)] in depth-first order."""
    n = polar_code_info(code)[2]
    kind = np.zeros(max(n, 1), np.uint32)
    nv = np.zeros(max(n, 1), np.uint32)
    off = np.zeros(max(n, 1), np.uint32)
    cnt = ctypes.c_size_t()
    P = ctypes.POINTER(ctypes.c_uint32)
    _check(_lib.polar_code_schedule(code.handle, kind.ctypes.data_as(P), nv.ctypes.data_as(P),
                                    off.ctypes.data_as(P), kind.size, ctypes.byref(cnt)),
           "polar_code_schedule")
    return [(OP_NAMES[kind[i]], int(nv[i]), int(off[i])) for i in range(cnt.value)]


def polar_code_trace_len(code: PolarCode) -> int:
    return int(_lib.polar_code_trace_len(code.handle))


def polar_encode_systematic(code: PolarCode, info_packed) -> np.ndarray:
    """Host systematic encoder: info_packed uint8[n, ceil(K/8)] -> uint8[n, ceil(N/8)]."""
    d = np.ascontiguousarray(np.asarray(info_packed, dtype=np.uint8))
    d = d.reshape(-1, code.out_row) if code.out_row else d.reshape(-1, 0)
    n = d.shape[0]
    x = np.zeros((n, (code.N + 7) // 8), np.uint8)
    P = ctypes.POINTER(ctypes.c_uint8)
    src = d.ctypes.data_as(P) if d.size else P()
    _check(_lib.polar_encode_systematic(code.handle, src, x.ctypes.data_as(P), n),
           "polar_encode_systematic")
    return x


def _stream_handle(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _out_tensor(code, llr, bits_out, n):
    import torch
    if bits_out is None:
        bits_out = torch.empty((n, code.out_row), dtype=torch.uint8, device=llr.device)
    if bits_out.dtype != torch.uint8 or not bits_out.is_contiguous() or bits_out.numel() < n * code.out_row:
        raise ValueError("bits_out must be a contiguous uint8 tensor of n*ceil(K/8) bytes")
    return bits_out


def _decode(fn, name, code, llr, bits_out, n_frames, stream, dtype):
    import torch
    if not isinstance(llr, torch.Tensor) or not llr.is_cuda:
        raise TypeError(f"{name}: llr must be a CUDA tensor")
    if llr.dtype != dtype or not llr.is_contiguous():
        raise TypeError(f"{name}: llr must be a contiguous {dtype} tensor")
    n = llr.numel() // code.N if n_frames is None else int(n_frames)
    if n * code.N > llr.numel():
        raise ValueError(f"{name}: llr holds fewer than n_frames*N values")
    bits_out = _out_tensor(code, llr, bits_out, n)
    _check(fn(code.handle, ctypes.c_void_p(llr.data_ptr()), ctypes.c_void_p(bits_out.data_ptr()),
              n, _stream_handle(stream)), name)
    return bits_out


def polar_decode(code: PolarCode, llr, bits_out=None, n_frames=None, stream=None):
    """Decode float32 LLRs [n, N] (CUDA tensor) into packed info bits [n, ceil(K/8)]."""
    import torch
    return _decode(_lib.polar_decode, "polar_decode", code, llr, bits_out, n_frames, stream,
                   torch.float32)


def polar_decode_noalloc(code: PolarCode, llr, bits_out, n_frames=None, stream=None):
    """polar_decode without device allocation (static device scratch); bits_out is
    required, since creating it would allocate."""
    import torch
    if bits_out is None:
        raise ValueError("polar_decode_noalloc: bits_out must be provided")
    return _decode(_lib.polar_decode_noalloc, "polar_decode_noalloc", code, llr, bits_out,
                   n_frames, stream, torch.float32)


def polar_decode_i8(code: PolarCode, llr, bits_out=None, n_frames=None, stream=None):
    """Decode int8 LLRs in [-127, 127] [n, N] (CUDA tensor)."""
    import torch
    return _decode(_lib.polar_decode_i8, "polar_decode_i8", code, llr, bits_out, n_frames,
                   stream, torch.int8)


def polar_decode_host(code: PolarCode, llr, bits_out=None, chunk_frames: int = 0):
    """Decode LLRs held in host memory (a CPU tensor, pinned for overlap, or a
    numpy array; float32 or int8 [n, N]) into host bits [n, ceil(K/8)]; copies
    overlap decoding through chunked internal streams. Blocking."""
    import torch
    if isinstance(llr, np.ndarray):
        llr = torch.from_numpy(np.ascontiguousarray(llr))
    if llr.is_cuda or not llr.is_contiguous() or llr.dtype not in (torch.float32, torch.int8):
        raise TypeError("llr must be a contiguous host float32 or int8 tensor")
    n = llr.numel() // code.N
    if bits_out is None:
        bits_out = torch.empty((n, code.out_row), dtype=torch.uint8)
    if bits_out.is_cuda or bits_out.dtype != torch.uint8 or bits_out.numel() < n * code.out_row:
        raise ValueError("bits_out must be a host uint8 tensor of n*ceil(K/8) bytes")
    _check(_lib.polar_decode_host(code.handle, 1 if llr.dtype == torch.int8 else 0,
                                  ctypes.c_void_p(llr.data_ptr()),
                                  ctypes.c_void_p(bits_out.data_ptr()), n, chunk_frames),
           "polar_decode_host")
    return bits_out


def polar_decode_trace(code: PolarCode, llr, bits_out=None, trace=None, stream=None):
    """Decode and record every F/G/G_0R output; returns (bits_out, trace[n, trace_len])."""
    import torch
    if not llr.is_cuda or not llr.is_contiguous() or llr.dtype not in (torch.float32, torch.int8):
        raise TypeError("llr must be a contiguous CUDA float32 or int8 tensor")
    n = llr.numel() // code.N
    bits_out = _out_tensor(code, llr, bits_out, n)
    tl = polar_code_trace_len(code)
    if trace is None:
        trace = torch.empty((n, tl), dtype=torch.float32, device=llr.device)
    _check(_lib.polar_decode_trace(code.handle, ctypes.c_void_p(llr.data_ptr()),
                                   1 if llr.dtype == torch.int8 else 0,
                                   ctypes.c_void_p(bits_out.data_ptr()),
                                   ctypes.c_void_p(trace.data_ptr()), n, _stream_handle(stream)),
           "polar_decode_trace")
    return bits_out, trace


def polar_code_set_launch(code: PolarCode, is_i8: bool, threads=0, smem_stage_max=0,
                          warp_stage_max=0, ctas_per_sm=0, stage_channel=0):
    _check(_lib.polar_code_set_launch(code.handle, int(bool(is_i8)), threads, smem_stage_max,
                                      warp_stage_max, ctas_per_sm, stage_channel),
           "polar_code_set_launch")


def polar_code_get_launch(code: PolarCode, is_i8: bool, n_frames: int) -> dict:
    v = [ctypes.c_uint32() for _ in range(6)]
    s = [ctypes.c_size_t() for _ in range(2)]
    unrolled = ctypes.c_uint32()
    _check(_lib.polar_code_get_launch(code.handle, int(bool(is_i8)), n_frames,
                                      *[ctypes.byref(x) for x in v], *[ctypes.byref(x) for x in s],
                                      ctypes.byref(unrolled)),
           "polar_code_get_launch")
    keys = ["threads", "smem_stage_max", "warp_stage_max", "ctas_per_sm", "stage_channel", "grid"]
    d = {k: x.value for k, x in zip(keys, v)}
    d["smem_bytes"], d["scratch_bytes"] = s[0].value, s[1].value
    d["unrolled"] = unrolled.value
    f = ctypes.c_uint32()
    _check(_lib.polar_code_get_frames_per_cta(code.handle, int(bool(is_i8)), n_frames,
                                              ctypes.byref(f)), "polar_code_get_frames_per_cta")
    d["frames_per_cta"] = f.value
    return d


def polar_code_set_frames_per_cta(code: PolarCode, is_i8: bool, frames: int):
    """Several frames per CTA, one per warp (2, 4, 8; 0/1 = one), for the
    specialised decoder of one-warp-per-frame shapes (compile afterwards)."""
    _check(_lib.polar_code_set_frames_per_cta(code.handle, int(bool(is_i8)), frames),
           "polar_code_set_frames_per_cta")


COMPILE_OUTLINE_SUBTREES, COMPILE_OUTLINE_MEMORY, COMPILE_COMPACT, COMPILE_FULL = 1, 2, 3, 4
COMPILE_LOCAL_LEAVES = 8
BATCH_FRAME_PER_WARP = 16


def polar_code_compile(code: PolarCode, is_i8: bool, n_frames: int, reg_subtree: int = 0,
                       flags: int = 0):
    """Compile the decoder specialised to this code for the shape of an n_frames
    decode (flags: COMPILE_OUTLINE_SUBTREES, COMPILE_OUTLINE_MEMORY, COMPILE_COMPACT,
    COMPILE_FULL to force a form; COMPILE_LOCAL_LEAVES for the per-lane form of small
    nodes)."""
    st = _lib.polar_code_compile_ex(code.handle, int(bool(is_i8)), n_frames, reg_subtree, flags)
    if st != 0:
        raise PolarError(st, "polar_code_compile: " + polar_code_compile_log(code)[-2000:])


def polar_code_compile_log(code: PolarCode) -> str:
    return (_lib.polar_code_compile_log(code.handle) or b"").decode(errors="replace")


def polar_code_check(code: PolarCode, stream=None):
    _check(_lib.polar_code_check(code.handle, _stream_handle(stream)), "polar_code_check")


def polar_selftest_bounded_wait(code: PolarCode, limit_us: int, stream=None):
    """Launch a device wait that nothing completes; it gives up after limit_us and
    marks the handle, so the next polar_code_check raises POLAR_ETIMEOUT."""
    _check(_lib.polar_selftest_bounded_wait(code.handle, limit_us, _stream_handle(stream)),
           "polar_selftest_bounded_wait")


def polar_status_str(status: int) -> str:
    return _lib.polar_status_str(status).decode()


class PolarBatch:
    """Owns a polar_batch_t (mixed-code batch decoder); keeps its codes alive."""

    def __init__(self, handle: int, codes, is_i8: bool):
        self.handle = ctypes.c_void_p(handle)
        self.codes = list(codes)
        self.is_i8 = is_i8

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            _lib.polar_batch_destroy(h)
            self.handle = ctypes.c_void_p(0)


def polar_batch_create(codes, is_i8: bool, threads: int = 0, smem_stage_max=None,
                       warp_stage_max=None, ctas_per_sm: int = 0, flags: int = 0) -> PolarBatch:
    """One persistent decoder for frames of any of `codes`; per-code shared-memory
    stage cap and warp threshold (lists, 0 = default)."""
    arr = (ctypes.c_void_p * len(codes))(*[c.handle.value for c in codes])

    def per_code(v):
        return None if v is None else (ctypes.c_uint32 * len(codes))(*[int(x) for x in v])

    h = ctypes.c_void_p()
    st = _lib.polar_batch_create_ex(arr, len(codes), int(bool(is_i8)), threads,
                                    per_code(smem_stage_max), per_code(warp_stage_max), ctas_per_sm,
                                    flags, ctypes.byref(h))
    if st != 0:
        raise PolarError(st, "polar_batch_create: " +
                         (_lib.polar_batch_log(None) or b"").decode(errors="replace")[-3000:])
    return PolarBatch(h.value, codes, bool(is_i8))


def polar_batch_destroy(batch: PolarBatch):
    batch.__del__()


def polar_batch_decode(batch: PolarBatch, code_id, llr_off, out_off, llr, bits_out, n_frames=None,
                       stream=None):
    """code_id (int32/uint32), llr_off / out_off (int64) and llr / bits_out are CUDA tensors."""
    n = code_id.numel() if n_frames is None else int(n_frames)
    _check(_lib.polar_batch_decode(batch.handle, ctypes.c_void_p(code_id.data_ptr()),
                                   ctypes.c_void_p(llr_off.data_ptr()),
                                   ctypes.c_void_p(out_off.data_ptr()),
                                   ctypes.c_void_p(llr.data_ptr()), ctypes.c_void_p(bits_out.data_ptr()),
                                   n, _stream_handle(stream)), "polar_batch_decode")
    return bits_out


def polar_batch_info(batch: PolarBatch) -> dict:
    t, g = ctypes.c_uint32(), ctypes.c_uint32()
    sm, sc = ctypes.c_size_t(), ctypes.c_size_t()
    _check(_lib.polar_batch_info(batch.handle, ctypes.byref(t), ctypes.byref(g), ctypes.byref(sm),
                                 ctypes.byref(sc)), "polar_batch_info")
    return dict(threads=t.value, grid=g.value, smem_bytes=sm.value, scratch_bytes=sc.value)


def polar_batch_log(batch: PolarBatch) -> str:
    return (_lib.polar_batch_log(batch.handle) or b"").decode(errors="replace")


def _buf_ptr(buf):
    """Address and size in bytes of a request buffer: a numpy array, a CPU tensor
    (pinned for asynchronous copies) or a CUDA tensor."""
    if isinstance(buf, np.ndarray):
        if not buf.flags.c_contiguous:
            raise ValueError("request buffers must be contiguous")
        return buf.ctypes.data, buf.nbytes
    if not buf.is_contiguous():
        raise ValueError("request buffers must be contiguous tensors")
    return buf.data_ptr(), buf.numel() * buf.element_size()


class PolarServer:
    """Owns a polar_server_t; keeps the batch decoder and the host buffers alive."""

    def __init__(self, handle: int, keep):
        self.handle = ctypes.c_void_p(handle)
        self._keep = keep

    def destroy(self) -> int:
        h = getattr(self, "handle", None)
        st = 0
        if h is not None and h.value:
            st = _lib.polar_server_destroy(h)
            self.handle = ctypes.c_void_p(0)
        return st

    def __del__(self):
        self.destroy()


SERVE_LAUNCH_PER_CODE = 1


def polar_server_create(batch: PolarBatch, reqs: np.ndarray, host_llr, host_out, done_ns: np.ndarray,
                        device_budget_bytes: int, max_frames: int, slots: int,
                        flags: int = 0) -> PolarServer:
    """Serving loop over `batch`. reqs: REQUEST_DTYPE array (circular, capacity =
    len); host_llr / host_out: pinned CPU tensors (or CUDA tensors: copies stay
    on the device);
    done_ns: uint64 array of len(reqs) receiving completion times; flags:
    SERVE_LAUNCH_PER_CODE for one launch per code in each admission."""
    if reqs.dtype != REQUEST_DTYPE or not reqs.flags.c_contiguous:
        raise TypeError("reqs must be a contiguous REQUEST_DTYPE array")
    if done_ns.dtype != np.uint64 or done_ns.size != reqs.size or not done_ns.flags.c_contiguous:
        raise TypeError("done_ns must be a contiguous uint64 array of len(reqs) entries")
    lp, lb = _buf_ptr(host_llr)
    op, ob = _buf_ptr(host_out)
    h = ctypes.c_void_p()
    _check(_lib.polar_server_create(batch.handle, ctypes.c_void_p(reqs.ctypes.data), reqs.size,
                                    ctypes.c_void_p(lp), lb, ctypes.c_void_p(op), ob,
                                    ctypes.c_void_p(done_ns.ctypes.data), device_budget_bytes,
                                    max_frames, slots, flags, ctypes.byref(h)),
           "polar_server_create")
    return PolarServer(h.value, (batch, reqs, host_llr, host_out, done_ns))


def polar_server_publish(server: PolarServer, n_published: int):
    _check(_lib.polar_server_publish(server.handle, n_published), "polar_server_publish")


def polar_server_progress(server: PolarServer):
    """(completed, admissions, launches); raises on the loop's sticky error."""
    c, a, n = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    _check(_lib.polar_server_progress(server.handle, ctypes.byref(c), ctypes.byref(a),
                                      ctypes.byref(n)), "polar_server_progress")
    return c.value, a.value, n.value


def polar_server_destroy(server: PolarServer):
    _check(server.destroy(), "polar_server_destroy")


# ---- communication chain on the GPU

def _dptr(t):
    return ctypes.c_void_p(t.data_ptr())


def polar_random_info(code: PolarCode, info_out, seed: int, frame0: int = 0, n_frames=None,
                      stream=None):
    """Fill a CUDA uint8 tensor [n, ceil(K/8)] with Philox information bits."""
    n = info_out.numel() // max(code.out_row, 1) if n_frames is None else int(n_frames)
    _check(_lib.polar_random_info(code.handle, _dptr(info_out), n, seed, frame0,
                                  _stream_handle(stream)), "polar_random_info")
    return info_out


def polar_encode_systematic_device(code: PolarCode, info, codeword_out, n_frames=None, stream=None):
    """Device systematic encoder: CUDA uint8 [n, ceil(K/8)] -> [n, ceil(N/8)]."""
    n = info.numel() // max(code.out_row, 1) if n_frames is None else int(n_frames)
    _check(_lib.polar_encode_systematic_device(code.handle, _dptr(info), _dptr(codeword_out), n,
                                               _stream_handle(stream)),
           "polar_encode_systematic_device")
    return codeword_out


def polar_channel_awgn(code: PolarCode, codewords, llr_out, ebn0_db: float, seed: int,
                       frame0: int = 0, n_frames=None, stream=None):
    """BPSK-AWGN channel LLRs into llr_out (CUDA float32 or int8 [n, N])."""
    import torch
    n = llr_out.numel() // code.N if n_frames is None else int(n_frames)
    _check(_lib.polar_channel_awgn(code.handle, _dptr(codewords), _dptr(llr_out),
                                   1 if llr_out.dtype == torch.int8 else 0, n, ebn0_db, seed, frame0,
                                   _stream_handle(stream)), "polar_channel_awgn")
    return llr_out


def polar_count_errors(code: PolarCode, decoded, sent, counters, n_frames=None, stream=None):
    """counters (CUDA int64 [2]) += (frame errors, bit errors)."""
    n = decoded.numel() // max(code.out_row, 1) if n_frames is None else int(n_frames)
    _check(_lib.polar_count_errors(code.handle, _dptr(decoded), _dptr(sent), n, _dptr(counters),
                                   _stream_handle(stream)), "polar_count_errors")
    return counters


def polar_fer_run(code: PolarCode, is_i8: bool, ebn0_db: float, seed: int, n_frames: int,
                  batch: int = 0):
    """(frame errors, bit errors) of a GPU simulation of n_frames frames."""
    fe, be = ctypes.c_uint64(), ctypes.c_uint64()
    _check(_lib.polar_fer_run(code.handle, int(bool(is_i8)), ebn0_db, seed, n_frames, batch,
                              ctypes.byref(fe), ctypes.byref(be)), "polar_fer_run")
    return fe.value, be.value
