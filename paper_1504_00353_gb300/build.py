"""Compile libpolar_gb300.so in place (nvcc, sm_103a only).

    python -m paper_1504_00353_gb300.build

One shared library holds the host code (handles, operation-list compiler,
encoder, launch selection, the C ABI) and the CUDA kernels. Floating point is
strict IEEE: no --use_fast_math, so F/G/Repetition match a scalar evaluation.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libpolar_gb300.so")
SOURCES = [os.path.join(CSRC, "polar_host.cpp"), os.path.join(CSRC, "polar_codegen.cpp"),
           os.path.join(CSRC, "polar_batch.cpp"), os.path.join(CSRC, "polar_serve.cpp"),
           os.path.join(CSRC, "polar_kernels.cu"), os.path.join(CSRC, "polar_chain.cu"),
           os.path.join(CSRC, "polar_hostio.cpp")]
GEN = os.path.join(HERE, "_build")  # generated include: polar_ops.cuh as a C++ string
HEADERS = [os.path.join(CSRC, "polar_internal.h"), os.path.join(CSRC, "polar_ops.cuh"),
           os.path.join(CSRC, "polar_ring.h"),
           os.path.join(ROOT, "include", "polar_gb300.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(p) > t for p in SOURCES + HEADERS)


def _embed_ops_header() -> None:
    """Write _build/polar_ops_embed.inc: polar_ops.cuh as a raw string literal, the
    header the run-time (NVRTC) compilation of specialised decoders includes."""
    os.makedirs(GEN, exist_ok=True)
    src = open(os.path.join(CSRC, "polar_ops.cuh")).read()
    assert ")POLAROPS\"" not in src
    text = 'R"POLAROPS(' + src + ')POLAROPS"\n'
    path = os.path.join(GEN, "polar_ops_embed.inc")
    if not os.path.exists(path) or open(path).read() != text:
        with open(path, "w") as fh:
            fh.write(text)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every translation unit in parallel (one nvcc per source, object
    files in _build/), then link the shared library."""
    if not force and not _stale():
        return LIB
    _embed_ops_header()
    from concurrent.futures import ThreadPoolExecutor
    common = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", *ARCH, "-lineinfo",
              "-I" + os.path.join(ROOT, "include"), "-I" + CSRC, "-I" + GEN]
    if verbose:
        common.insert(0, "-Xptxas=-v")
    tag = f".{os.getpid()}.o"
    objs = [os.path.join(GEN, os.path.basename(src) + tag) for src in SOURCES]

    def compile_one(pair):
        src, obj = pair
        subprocess.run([nvcc(), *common, "-c", src, "-o", obj], check=True)

    try:
        with ThreadPoolExecutor(max_workers=min(len(SOURCES), os.cpu_count() or 1)) as ex:
            list(ex.map(compile_one, zip(SOURCES, objs)))
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.run([nvcc(), "-shared", *ARCH, "-o", tmp, *objs, "-ldl", "-lpthread"], check=True)
        os.replace(tmp, LIB)
    finally:
        for obj in objs:
            if os.path.exists(obj):
                os.remove(obj)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
