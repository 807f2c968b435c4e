"""The code-specialised decoders are generated as CUDA source at run time
(Sec. III-B, "Generating an Unrolled Decoder": here one program per code and
launch shape) and compiled on the GPU with NVRTC. This host test emits that
source for the launch shapes the benchmark and the mixed batch use (int8 and
float32 throughput, batch-1, the compact form, the mixed-code batch) and
compiles each for sm_103a with nvcc, so a generator or kernel-header change that
does not compile fails here, without a GPU. Bits are checked by the GPU tests."""
import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

import pytest

from paper_1504_00353_gb300 import build, synth

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
PKG = os.path.join(ROOT, "paper_1504_00353_gb300")
CSRC = os.path.join(PKG, "csrc")
CUDA_INC = "/usr/local/cuda/include"

# (name, (N, K, design dB), is_i8, threads, S, W, frames per CTA, stage channel,
#  register subtree, outline flags, CTAs per SM)
CASES = [
    ("i8_throughput", (32768, 29492, 4.0), 1, 128, 1024, 2048, 4, 0, 512, 1, 7),
    ("f32_throughput", (32768, 29492, 4.0), 0, 128, 2048, 2048, 1, 0, 256, 1, 10),
    ("i8_batch1", (32768, 29492, 4.0), 1, 256, 16384, 2048, 1, 1, 1024, 0, 1),
    ("i8_compact", (16384, 14746, 3.0), 1, 64, 1024, 512, 1, 0, 256, 3, 0),
]
MIXED = dict(is_i8=1, threads=128, min_blocks=7, outline=1, warp_frames=1,
             S=[128, 512, 1024, 1024, 1024], W=[256, 1024, 2048, 2048, 2048], R=256)


def _tools():
    cxx = shutil.which("g++") or shutil.which("c++")
    nvcc = build.nvcc()
    if not cxx or not (os.path.exists(nvcc) or shutil.which(nvcc)):
        pytest.skip("no host compiler or nvcc")
    if not os.path.isdir(CUDA_INC):
        pytest.skip("no CUDA headers")
    return cxx, nvcc


def _mask_file(tmp, N, K, db):
    path = tmp / f"mask_{N}_{K}_{db}.bin"
    if not path.exists():
        path.write_bytes(synth.frozen_mask(N, K, db).astype("uint8").tobytes())
    return str(path)


def test_generated_decoders_compile_for_sm103a(tmp_path):
    cxx, nvcc = _tools()
    lib = build.build()
    exe = tmp_path / "codegen_source"
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", CSRC, "-I", os.path.join(ROOT, "include"),
                    "-I", CUDA_INC, os.path.join(HERE, "cpp", "codegen_source.cpp"),
                    "-L", os.path.dirname(lib), "-lpolar_gb300",
                    "-Wl,-rpath," + os.path.dirname(lib), "-o", str(exe)], check=True)
    sources = []
    for name, (N, K, db), i8, T, S, W, F, stage, reg, outline, ctas in CASES:
        out = tmp_path / f"{name}.cu"
        args = [str(exe), "code", str(out), _mask_file(tmp_path, N, K, db), N, K, i8, T, S, W, F,
                stage, reg, outline, ctas]
        r = subprocess.run([str(a) for a in args], capture_output=True, text=True, timeout=120)
        assert r.returncode == 0 and r.stdout.startswith("OK"), r.stdout
        sources.append(out)
    out = tmp_path / "i8_mixed.cu"
    args = [str(exe), "batch", str(out), MIXED["is_i8"], MIXED["threads"], MIXED["min_blocks"],
            MIXED["outline"], MIXED["warp_frames"]]
    for (N, K), S, W in zip(synth.MIXED_CODES, MIXED["S"], MIXED["W"]):
        args += [_mask_file(tmp_path, N, K, synth.MIXED_DESIGN_DB), N, K, S, W, MIXED["R"]]
    r = subprocess.run([str(a) for a in args], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.startswith("OK"), r.stdout
    sources.append(out)

    def compile_one(src):
        return subprocess.run([nvcc, "-std=c++17", "-cubin", *build.ARCH, "-I", CSRC,
                               "-o", str(src.with_suffix(".cubin")), str(src)],
                              capture_output=True, text=True, timeout=900)

    with ThreadPoolExecutor(max_workers=len(sources)) as ex:
        results = list(ex.map(compile_one, sources))
    for src, r in zip(sources, results):
        assert r.returncode == 0, f"{src.name}:\n{r.stderr[-3000:]}"
        assert src.with_suffix(".cubin").stat().st_size > 0
        # the kernel the library launches is in the program
        text = src.read_text()
        assert ("polar_batch(" in text) if src.name == "i8_mixed.cu" else ("polar_unrolled(" in text)
