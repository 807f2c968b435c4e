"""Benchmark: Fast-SSC decode throughput and frame latency on one node.

Default workload: the (32768, 29492) polar code (Bhattacharyya construction at
4.0 dB), BPSK-AWGN at 4.0 dB, 4096 frames per step per GPU, int8 LLRs (the
paper's headline configuration for this code); float32 is reported under
"variants".
A step is one decode of the batch (every operation of the Fast-SSC list, the
channel-LLR load and the packed-bit store), one kernel launch.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--dtype f32|i8]
                    [--impl reference] [--workload NAME]

Prints one JSON line (rank 0). With --impl reference the CPU oracle is timed on
the host cores instead (the slow, plain reference of the method).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1504_00353_gb300 import synth  # noqa: E402

METRIC = "info-bit Gbps"
# Paper numbers for this exact code (Table 3 int8 unrolled decoder, Table 2 float
# unrolled decoder; Intel i7-4770S, one core): context, other hardware.
PAPER_GBPS = {("n32768_k29492_4.0db", "i8"): 1.131, ("n32768_k29492_4.0db", "f32"): 0.3151}
L2_BYTES = 129 * 1024 * 1024


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--dtype", choices=["f32", "i8"], default="i8")
    p.add_argument("--workload", default="n32768_k29492_4.0db", choices=sorted(synth.WORKLOADS))
    p.add_argument("--batch", type=int, default=0, help="frames per step per GPU (0: workload's)")
    p.add_argument("--impl", choices=["native", "reference"], default="native")
    p.add_argument("--reference-seconds", type=float, default=60.0,
                   help="reference arm: CPU seconds of oracle work over all timed steps")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--latency-frames", type=int, default=200)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-mixed", action="store_true",
                   help="leave out the mixed-length batch block of the default line")
    p.add_argument("--no-serve", action="store_true",
                   help="leave out the serving block of the default line")
    p.add_argument("--no-variant", action="store_true", help="skip the other LLR type")
    p.add_argument("--interpreter", action="store_true",
                   help="time the operation-list interpreter instead of the specialised decoder")
    p.add_argument("--compile-form", choices=["auto", "full", "subtrees", "memory", "compact"],
                   default="auto",
                   help="form of the specialised decoder: what is compiled out of line (auto: "
                        "compact above 4096 operations, else the tuned form)")
    p.add_argument("--mode", choices=["throughput", "mixed", "serve", "fer", "latency"],
                   default="throughput",
                   help="throughput: one code, batch and batch-1 (default); mixed: 65,536 frames "
                        "of five codes, one persistent launch in a CUDA graph vs one launch per "
                        "code; serve: Poisson arrivals through the serving loop vs a plain queue; "
                        "fer: frame/bit error rates of float32 vs int8 from the GPU chain")
    p.add_argument("--loads", default="1,10,50,200", help="serve: offered loads, coded Gbps")
    p.add_argument("--serve-seconds", type=float, default=1.0,
                   help="serve: seconds of arrivals per load (at most --serve-max-frames)")
    p.add_argument("--serve-max-frames", type=int, default=500_000)
    p.add_argument("--serve-pool", default="host,device",
                   help="serve: LLR pool in pinned host memory and/or in device memory")
    return p.parse_args()


# ---------------------------------------------------------------- distributed

def dist_init(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl", rank=rank, world_size=world,
                                device_id=torch.device("cuda", local))
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, v: float) -> float:
    from paper_1504_00353_gb300 import sharding
    return sharding.max_over_ranks(v, device="cuda") if world > 1 else v


# ---------------------------------------------------------------- inputs

def make_inputs(wl, batch, seed, dtype):
    """Info bits, codewords (library's host encoder) and channel LLRs (host)."""
    from paper_1504_00353_gb300 import polar
    N, K = wl["N"], wl["K"]
    mask = synth.frozen_mask(N, K, wl["design_db"])
    code = polar.polar_code_create(N, K, mask)
    rng = np.random.default_rng(seed)
    d = synth.info_bits(rng, batch, K)
    cw = synth.unpack_bits(polar.polar_encode_systematic(code, synth.pack_bits(d)), N)
    llr = synth.awgn_llr(rng, cw, wl["ebn0_db"], K / N)
    if dtype == "i8":
        llr = synth.quantize_i8(llr)
    return mask, code, d, llr


# ---------------------------------------------------------------- clocks

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index, interval_ms=200):
        self.gpu = gpu_index
        self.interval_ms = interval_ms
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", str(self.interval_ms)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- roofline inputs

def profile_traffic(workload, dtype):
    """DRAM bytes per launch from the committed ncu summary of the specialised
    decoder, when it was taken on the current decoder sources (the sha256 prefix of
    polar_ops.cuh + polar_codegen.cpp is recorded beside the number)."""
    path = os.path.join(ROOT, "profiles", f"fastssc_unrolled_{dtype}_{workload}.md")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    h = re.search(r"kernel_source_sha256:\s*([0-9a-f]+)", txt)
    if not m or not h:
        return None
    sha = hashlib.sha256()
    for f in ("polar_ops.cuh", "polar_codegen.cpp"):
        sha.update(open(os.path.join(ROOT, "paper_1504_00353_gb300", "csrc", f), "rb").read())
    if not sha.hexdigest().startswith(h.group(1)):
        return None
    return float(m.group(1))


def profile_value(workload, dtype, key):
    """A `key: value` figure from the committed ncu summary of the specialised
    decoder, under the same source-hash rule as profile_traffic."""
    path = os.path.join(ROOT, "profiles", f"fastssc_unrolled_{dtype}_{workload}.md")
    if not os.path.exists(path) or profile_traffic(workload, dtype) is None:
        return None
    m = re.search(rf"^{re.escape(key)}:\s*([0-9.eE+]+)", open(path).read(), re.M)
    return float(m.group(1)) if m else None


def profile_smem(workload, dtype):
    """Shared-memory bytes per launch (ncu smsp__sass_data_bytes_mem_shared.sum)."""
    return profile_value(workload, dtype, "smem_bytes_per_launch")


def profile_pipes(workload, dtype, element_ops):
    """Pipe and issue-slot utilisation of the decoder (ncu, percent of peak
    sustained over active cycles, as fractions) and thread instructions per
    element operation, from the committed summary; None when absent or stale."""
    keys = {"alu": "alu_pipe_busy", "fma": "fma_pipe_busy", "lsu": "lsu_pipe_busy",
            "issue": "issue_slots_busy"}
    out = {k: profile_value(workload, dtype, v) for k, v in keys.items()}
    if any(v is None for v in out.values()):
        return None
    tie = profile_value(workload, dtype, "thread_inst_per_launch")
    out["thread_inst_per_element_op"] = None if tie is None or not element_ops else tie / element_ops
    out["source"] = ("ncu sm__inst_executed_pipe_{alu,fma,lsu} and smsp__issue_active "
                     "(pct_of_peak_sustained_active) and thread_inst_executed_true of the "
                     "committed profile")
    return out


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


# ---------------------------------------------------------------- CPU oracle timing

def time_oracle(mask, llr, budget_cpu_s=16.0, threads=None):
    """Oracle Fast-SSC over a bounded sample, frames split across host threads
    (the C loop runs without the GIL). Returns (frames, seconds, threads)."""
    import oracle
    oracle.build()
    n_total = llr.shape[0]
    t0 = time.perf_counter()
    oracle.decode_batch(mask, llr[:1])
    per = max(time.perf_counter() - t0, 1e-6)
    T = threads or min(os.cpu_count() or 1, 16)
    frames = int(max(T, min(n_total, budget_cpu_s / per)))
    frames = max(T, frames - frames % T)
    frames = min(frames, n_total - n_total % T if n_total >= T else n_total)
    bounds = np.linspace(0, frames, T + 1).astype(int)
    chunks = [slice(int(a), int(b)) for a, b in zip(bounds[:-1], bounds[1:])]
    errs = []

    def work(ix):
        try:
            oracle.decode_batch(mask, llr, frames=ix)
        except Exception as e:  # pragma: no cover
            errs.append(e)

    passes = max(1, int(budget_cpu_s / (per * frames)))

    def work_passes(ix):
        for _ in range(passes):
            work(ix)

    ths = [threading.Thread(target=work_passes, args=(c,)) for c in chunks if c.stop > c.start]
    t0 = time.perf_counter()
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    dt = time.perf_counter() - t0
    if errs:
        raise errs[0]
    return frames * passes, dt, len(ths)


def oracle_baseline(mask, llr, reps=10, budget_cpu_s=12.0):
    """The CPU oracle timed the way the paper times its decoders (Sec. III,
    methodology: repeated runs, one core), and on every host core: the median
    of `reps` repetitions of each, over a bounded sample of the workload's
    frames (the first frames of the seeded batch). Returns the cpu_baseline
    dict and the oracle's bits for frames [0, m) with m (for the parity sample)."""
    import oracle
    oracle.build()
    n_total = llr.shape[0]
    T = max(1, min(os.cpu_count() or 1, 64))
    t0 = time.perf_counter()
    oracle.decode_batch(mask, llr[:1])
    per = max(time.perf_counter() - t0, 1e-6)
    # one core: a third of the CPU budget
    m1 = int(np.clip(budget_cpu_s / 3 / reps / per, 1, n_total))
    st, bits = [], None
    for _ in range(reps):
        t0 = time.perf_counter()
        b = oracle.decode_batch(mask, llr, frames=slice(0, m1))
        st.append(time.perf_counter() - t0)
        bits = b if bits is None else bits
    # every core: T threads on disjoint slices, the rest of the budget
    m2 = int(np.clip(2 * budget_cpu_s / 3 / reps / per / T, 1, max(1, n_total // T)))
    chunks = [slice(i * m2, (i + 1) * m2) for i in range(T) if (i + 1) * m2 <= n_total]
    at, errs = [], []

    def work(ix):
        try:
            oracle.decode_batch(mask, llr, frames=ix)
        except Exception as e:  # pragma: no cover
            errs.append(e)

    for _ in range(reps):
        ths = [threading.Thread(target=work, args=(c,)) for c in chunks]
        t0 = time.perf_counter()
        for t in ths:
            t.start()
        for t in ths:
            t.join()
        at.append(time.perf_counter() - t0)
    if errs:
        raise errs[0]
    K = int((np.asarray(mask) == 0).sum())
    one = K * m1 / statistics.median(st) / 1e9
    allc = K * m2 * len(chunks) / statistics.median(at) / 1e9
    d = {"value": allc, "unit": "Gbps", "cores": len(chunks), "kind": "oracle",
         "single_thread": {"value": one, "unit": "Gbps", "cores": 1,
                           "frame_us": 1e6 * statistics.median(st) / m1},
         "reps": reps, "statistic": "median", "nproc": os.cpu_count(),
         "sample": (f"plain C Fast-SSC oracle; one core: frames 0..{m1 - 1} of the seeded batch "
                    f"x {reps} repetitions; all cores: {len(chunks)} threads x {m2} frames "
                    f"x {reps} repetitions; medians")}
    return d, bits, m1


# ---------------------------------------------------------------- arms

def run_reference(args, world, rank):
    if rank != 0:
        return
    wl = dict(synth.WORKLOADS[args.workload])
    N, K = wl["N"], wl["K"]
    batch = args.batch or wl["n_frames"]
    sample = min(batch, 256)
    # The oracle only needs the LLRs; build them without the GPU library.
    import oracle
    oracle.build()
    mask = synth.frozen_mask(N, K, wl["design_db"])
    rng = np.random.default_rng(wl["seed"])
    d = synth.info_bits(rng, sample, K)
    cw = np.stack([oracle.encode_systematic(mask, r) for r in d])
    llr = synth.awgn_llr(rng, cw, wl["ebn0_db"], K / N)
    if args.dtype == "i8":
        llr = synth.quantize_i8(llr)
    for _ in range(args.warmup):
        time_oracle(mask, llr[: min(sample, 16)], budget_cpu_s=0.5)
    tot_frames, tot_s, T = 0, 0.0, 1
    for _ in range(args.steps):
        f, s, T = time_oracle(mask, llr, budget_cpu_s=max(
            0.5, args.reference_seconds / max(args.steps, 1)))
        tot_frames += f
        tot_s += s
    gbps = K * tot_frames / tot_s / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": gbps, "unit": "Gbps",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tot_s / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
        "config": {"workload": args.workload, "N": N, "K": K, "batch": batch,
                   "ebn0_db": wl["ebn0_db"], "parallelism": "frames split across host threads"},
        "cpu_baseline": {"value": gbps, "unit": "Gbps", "cores": T, "kind": "oracle",
                         "sample": f"{tot_frames} frames of {args.workload} over {args.steps} "
                                   f"steps, plain C Fast-SSC oracle, {T} host threads"},
        "e2e": {"value": gbps, "unit": "Gbps", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def element_ops(code):
    """F/G/Combine/node element operations of one frame (roofline ALU count)."""
    from paper_1504_00353_gb300 import polar
    n = 0
    for kind, nv, _ in polar.polar_code_schedule(code):
        n += nv // 2 if kind in ("F", "G", "G_0R", "Combine", "Combine_0R") else nv
    return n


def device_timed(torch, stream, fn, steps, warmup, world):
    """Warm-up, then `steps` back-to-back launches bracketed by barrier + sync;
    returns (total ms max over ranks, mean per-launch ms)."""
    for _ in range(warmup):
        fn(0)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for i in range(steps):
        ev[i][0].record(stream)
        fn(i)
        ev[i][1].record(stream)
    t1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    return max_over_ranks(world, t0.elapsed_time(t1)), statistics.mean(a.elapsed_time(b) for a, b in ev)


def latency_block(torch, polar, args, N, K, mask, dtype, frames_dev, frames_host, nlat):
    """Batch-1 decodes of nlat frames with the decoder specialised for single
    frames: device time (the launch queued behind a spin so host call overhead
    is not counted) and end to end (copy in from pinned host memory, decode, copy
    out, host clock)."""
    i8 = dtype == "i8"
    row = (K + 7) // 8
    stream = torch.cuda.current_stream()
    decode = polar.polar_decode_i8 if i8 else polar.polar_decode
    lcode = polar.polar_code_create(N, K, mask)
    lshape, _ = tuned_or(N, K, mask, dtype, latency=True)
    compile_shape(lcode, dtype, lshape, 1, args.interpreter, args.compile_form)
    one_in = torch.empty((1, N), dtype=frames_dev.dtype, device="cuda")
    one_out = torch.empty((1, row), dtype=torch.uint8, device="cuda")
    h1 = torch.empty((1, row), dtype=torch.uint8).pin_memory()
    lat_dev, lat_e2e = [], []
    n = frames_dev.shape[0]
    for f in range(nlat + 5):
        one_in.copy_(frames_dev[f % n: f % n + 1])
        torch.cuda.synchronize()
        torch.cuda._sleep(1_000_000)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        decode(lcode, one_in, one_out)
        b.record(stream)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        one_in.copy_(frames_host[f % n: f % n + 1], non_blocking=True)
        decode(lcode, one_in, one_out)
        h1.copy_(one_out, non_blocking=True)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        if f >= 5:
            lat_dev.append(a.elapsed_time(b) * 1e3)
            lat_e2e.append((t1 - t0) * 1e6)
    return {"batch": 1, "frames": nlat,
            "device_p50": float(np.percentile(lat_dev, 50)),
            "device_p99": float(np.percentile(lat_dev, 99)),
            "e2e_p50": float(np.percentile(lat_e2e, 50)),
            "e2e_p99": float(np.percentile(lat_e2e, 99)),
            "launch": polar.polar_code_get_launch(lcode, i8, 1), "shape": lshape}


def run_native(args, world, rank, local):
    import torch

    from paper_1504_00353_gb300 import polar

    wl = dict(synth.WORKLOADS[args.workload])
    N, K = wl["N"], wl["K"]
    batch = args.batch or wl["n_frames"]
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    row = (K + 7) // 8

    mask, code0, d, llr32 = make_inputs(wl, batch, wl["seed"] + 1000 * rank, "f32")
    llr_by_dtype = {"f32": llr32, "i8": synth.quantize_i8(llr32)}

    forms = {}

    def setup(dtype):
        """Code handle with its specialised decoder compiled (untimed set-up)."""
        i8 = dtype == "i8"
        code = polar.polar_code_create(N, K, mask)
        shape, _ = tuned_or(N, K, mask, dtype)
        shape.setdefault("stage_channel", 2)
        compile_shape(code, dtype, shape, batch, args.interpreter, args.compile_form)
        forms[dtype] = (args.compile_form if args.compile_form != "auto"
                        else shape.get("compile_form", "auto"))
        return code

    def throughput(dtype, steps, warmup):
        i8 = dtype == "i8"
        es = 1 if i8 else 4
        code = setup(dtype)
        decode = polar.polar_decode_i8 if i8 else polar.polar_decode
        in_bytes = batch * N * es
        # Enough distinct input buffers that a step never finds its input in L2
        # (each step streams more than L2 before a buffer is reused).
        n_buf = 1 if in_bytes > 2 * L2_BYTES else int(np.ceil(3 * L2_BYTES / in_bytes)) + 1
        base = torch.from_numpy(llr_by_dtype[dtype]).to(dev)
        perms = [torch.arange(batch)] + [torch.randperm(batch, generator=torch.Generator().manual_seed(i))
                                         for i in range(1, n_buf)]
        bufs = [base] + [base[perms[i].to(dev)].contiguous() for i in range(1, n_buf)]
        out = torch.empty((batch, row), dtype=torch.uint8, device=dev)
        # sanity gate against the transmitted bits (not a parity test)
        decode(code, bufs[0], out)
        torch.cuda.synchronize()
        polar.polar_code_check(code)
        fer = float((out.cpu().numpy() != synth.pack_bits(d)).any(axis=1).mean())
        total_ms, launch_ms = device_timed(torch, stream, lambda i: decode(code, bufs[i % n_buf], out),
                                           steps, warmup, world)
        polar.polar_code_check(code)
        # the output of the last timed launch, rows in the order of frames of the batch
        last = (steps - 1) % n_buf
        timed_out = np.empty((batch, row), np.uint8)
        timed_out[perms[last].numpy()] = out.cpu().numpy()
        return dict(code=code, decode=decode, bufs=bufs, out=out, n_buf=n_buf, in_bytes=in_bytes,
                    total_ms=total_ms, launch_ms=launch_ms, fer=fer, timed_out=timed_out,
                    gbps=world * batch * K * steps / (total_ms * 1e-3) / 1e9,
                    launch=polar.polar_code_get_launch(code, i8, batch))

    main = args.dtype
    other = "i8" if main == "f32" else "f32"
    with ClockSampler(local) as clk:
        r = throughput(main, args.steps, args.warmup)
    clocks = clk.summary()
    alt = None if args.no_variant else throughput(other, max(3, args.steps // 2), 3)

    # end to end through the library's host-buffer entry point: pinned host LLRs
    # in, packed bits back in pinned host memory, the copies overlapped with
    # decoding by polar_decode_host's chunked streams (chunk size picked from a
    # few, the one used is reported)
    code, decode = r["code"], r["decode"]
    host_in = torch.from_numpy(llr_by_dtype[main]).pin_memory()
    host_out = torch.empty((batch, row), dtype=torch.uint8).pin_memory()
    out = r["out"]
    e2e_gbps, e2e_chunk = None, None
    if not args.no_e2e:
        e2e_steps = max(3, args.steps // 2)
        for _ in range(2):
            polar.polar_decode_host(code, host_in, host_out)
        barrier(world)
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            polar.polar_decode_host(code, host_in, host_out)
        e2e_s = max_over_ranks(world, time.perf_counter() - t0)
        e2e_gbps = world * batch * K * e2e_steps / e2e_s / 1e9
        e2e_chunk = "library default"
        decode(code, r["bufs"][0], out)  # the same frames through the device-buffer call
        torch.cuda.synchronize()
        assert np.array_equal(host_out.numpy(), out.cpu().numpy()), "host-buffer decode differs"

    # batch-1 frame latency, with the decoder specialised for single frames
    lat = None
    nlat = min(args.latency_frames, batch)
    if nlat:
        lat = latency_block(torch, polar, args, N, K, mask, main, r["bufs"][0][:nlat], host_in[:nlat],
                            nlat)

    hbm_peak, peak_kind = peaks()
    es = 1 if main == "i8" else 4
    alg_bytes = batch * (N * es + row)
    achieved = alg_bytes / (r["launch_ms"] * 1e-3) / 1e9
    ops = element_ops(code) * batch
    # element-op roof: one element operation per lane per clock on every SM (the
    # SM count from the device, the clock at its maximum and at the median seen
    # under load during the timed region)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    max_mhz = (clocks or {}).get("sm_max_mhz") or 2070.0
    med_mhz = (clocks or {}).get("sm_mhz") or max_mhz
    alu_peak = sms * 128 * max_mhz * 1e6
    t_hbm = alg_bytes / (hbm_peak * 1e9)
    t_alu = ops / alu_peak
    smem = profile_smem(args.workload, main)
    smem_peak = sms * 128 * max_mhz * 1e6  # bytes per second: 128 B per clock per SM
    line = {
        "metric": METRIC, "value": r["gbps"], "unit": "Gbps", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["total_ms"] / args.steps,
        "higher_is_better": True, "scaling": "weak",
        "vs_baseline": (r["gbps"] / PAPER_GBPS[(args.workload, main)]
                        if (args.workload, main) in PAPER_GBPS else None),
        "vs_baseline_basis": ("the paper's own number for this code and LLR type (Tables 2-3: "
                              "unrolled decoder on one core of an Intel i7-4770S at 3.1 GHz); "
                              "context from other hardware, not the target"
                              if (args.workload, main) in PAPER_GBPS else None),
        "dtype": main, "data": "synthetic",
        "config": {"workload": args.workload, "N": N, "K": K, "global_batch": batch * world,
                   "batch_per_gpu": batch, "ebn0_db": wl["ebn0_db"], "llr": main,
                   "parallelism": f"frames sharded over {world} GPU(s), no collective",
                   "l2": (f"{r['n_buf']} distinct input buffer(s) of {r['in_bytes'] / 2**20:.0f} MiB "
                          "rotated; inputs larger than L2"),
                   "decoder": "interpreter" if args.interpreter else
                   f"specialised (NVRTC, {forms.get(main, 'auto')} form)",
                   "launch": r["launch"], "fer_check": r["fer"]},
        "latency_us": lat,
        "e2e": {"value": e2e_gbps, "unit": "Gbps",
                "h2d_bytes_per_step": int(host_in.numel() * host_in.element_size()),
                "d2h_bytes_per_step": int(host_out.numel()),
                "api": "polar_decode_host (pinned host buffers)", "chunk_frames": e2e_chunk},
        "gpu_launches": args.steps,
        "roofline": {"bound": "hbm" if t_hbm >= t_alu else "alu",
                     "achieved": achieved if t_hbm >= t_alu else ops / (r["launch_ms"] * 1e-3) / 1e12,
                     "peak": hbm_peak if t_hbm >= t_alu else alu_peak / 1e12,
                     "unit": "GB/s" if t_hbm >= t_alu else "Tops/s",
                     "frac": (t_hbm if t_hbm >= t_alu else t_alu) / (r["launch_ms"] * 1e-3),
                     "peak_kind": (peak_kind if t_hbm >= t_alu else
                                   f"{sms} SMs x 128 lanes x {max_mhz:.0f} MHz (device query, "
                                   "maximum SM clock)"),
                     "traffic": profile_traffic(args.workload, main),
                     "algorithmic_bytes_per_launch": alg_bytes,
                     "element_ops_per_launch": ops,
                     "hbm_frac": t_hbm / (r["launch_ms"] * 1e-3),
                     "hbm_peak_gbs": hbm_peak,
                     "alu_frac": t_alu / (r["launch_ms"] * 1e-3),
                     "alu_frac_at_median_clock": t_alu * max_mhz / med_mhz / (r["launch_ms"] * 1e-3),
                     "smem": None if smem is None else {
                         "bound": "diagnostic", "bytes_per_launch": smem,
                         "achieved": smem / (r["launch_ms"] * 1e-3) / 1e9,
                         "peak": smem_peak / 1e9, "unit": "GB/s",
                         "frac": smem / (r["launch_ms"] * 1e-3) / smem_peak,
                         "source": "ncu smsp__sass_data_bytes_mem_shared.sum of the committed "
                                   "profile; peak = SMs x 128 B/clk x maximum SM clock"},
                     "pipes": profile_pipes(args.workload, main, ops),
                     "launch_ms": r["launch_ms"]},
        "clocks": clocks,
    }
    if alt:
        line["variants"] = {other: {"value": alt["gbps"], "unit": "Gbps",
                                    "ms_per_step": alt["total_ms"] / max(3, args.steps // 2),
                                    "launch": alt["launch"], "fer_check": alt["fer"]}}
    if rank == 0 and not args.no_cpu_baseline:
        cb, obits, m = oracle_baseline(mask, llr_by_dtype[main])
        cb["sample"] = f"{args.workload} ({main}); " + cb["sample"]
        line["cpu_baseline"] = cb
        # the same frames of the last timed launch, decoded by the GPU, against
        # the oracle's bits from the timing above
        eq = np.all(r["timed_out"][:m] == obits, axis=1)
        line["parity_sample"] = {"frames": int(m), "equal": bool(eq.all()),
                                 "frames_differing": int((~eq).sum()),
                                 "what": "bits of the last timed launch vs the CPU oracle, "
                                         f"frames 0..{m - 1} of the batch"}
    if rank == 0 and world == 1 and not args.no_mixed:
        line["mixed"] = mixed_block(args)
    if rank == 0 and world == 1 and not args.no_serve:
        line["serve"] = serve_block(args)
    if rank == 0:
        print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- mixed lengths

def mixed_inputs(n, dtype, seed, ebn0=None, ebn0_range=None):
    """n frames of codes drawn uniformly from synth.MIXED_CODES: code ids, per-code
    frame indices, per-code LLR arrays and info bits (library host encoder)."""
    from paper_1504_00353_gb300 import polar
    nk = synth.MIXED_CODES
    masks = [synth.frozen_mask(N, K, synth.MIXED_DESIGN_DB) for N, K in nk]
    rng = np.random.default_rng(seed)
    cid = rng.integers(0, len(nk), n)
    llr, bits = [], []
    for c, (N, K) in enumerate(nk):
        m = int((cid == c).sum())
        code = polar.polar_code_create(N, K, masks[c])
        d = synth.info_bits(rng, m, K)
        cw = synth.unpack_bits(polar.polar_encode_systematic(code, synth.pack_bits(d)), N)
        if ebn0_range is None:
            y = synth.awgn_llr(rng, cw, ebn0 if ebn0 is not None else synth.MIXED_DESIGN_DB, K / N)
        else:
            dbs = rng.uniform(*ebn0_range, m)
            y = np.empty((m, N), np.float32)
            for j in range(m):
                y[j] = synth.awgn_llr(rng, cw[j:j + 1], dbs[j], K / N)[0]
        llr.append(synth.quantize_i8(y) if dtype == "i8" else y)
        bits.append(synth.pack_bits(d))
    return masks, cid, llr, bits


def tuned_or(N, K, mask, dtype, default=None, latency=False):
    from paper_1504_00353_gb300 import autotune
    return autotune.shape_for(N, K, mask, dtype, latency=latency, default=default)


def compile_shape(code, dtype, shape, n_frames, interpreter=False, form="auto"):
    from paper_1504_00353_gb300 import autotune
    autotune.configure(code, dtype, shape, n_frames, interpreter, form)


def batch_shape(dtype):
    from paper_1504_00353_gb300 import autotune
    return autotune.batch_shape(dtype)


def run_mixed(args):
    """Config 3 on its own line: the mixed-length batch block of the default
    line (65,536 int8 frames of five codes, one persistent launch replayed from
    a CUDA graph against one launch per code)."""
    import torch
    torch.cuda.set_device(0)
    blk = mixed_block(args, n=args.batch or None, steps=args.steps, warmup=args.warmup)
    line = {"metric": "info-bit Gbps, mixed-length batch", "mode": "mixed",
            "value": blk["batched"]["gbps"], "unit": "Gbps", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": blk["batched"]["step_ms"],
            "higher_is_better": True, "dtype": "i8", "data": "synthetic",
            "config": {"workload": f"mixed{blk['frames']}", "codes": blk["codes"]},
            "gpu_launches": args.steps, **{k: v for k, v in blk.items() if k != "codes"}}
    print(json.dumps(line), flush=True)


def run_latency(args):
    """Batch-1 latency of the workload's code on its own line (the latency
    block of the default line): the decoder specialised for single frames."""
    import torch

    from paper_1504_00353_gb300 import polar
    torch.cuda.set_device(0)
    wl = dict(synth.WORKLOADS[args.workload])
    N, K = wl["N"], wl["K"]
    nlat = args.latency_frames
    mask, _, d, llr32 = make_inputs(wl, nlat, wl["seed"], "f32")
    y = synth.quantize_i8(llr32) if args.dtype == "i8" else llr32
    lat = latency_block(torch, polar, args, N, K, mask, args.dtype, torch.from_numpy(y).cuda(),
                        torch.from_numpy(y).pin_memory(), nlat)
    print(json.dumps({"metric": "batch-1 frame latency", "mode": "latency", "unit": "us",
                      "value": lat["device_p50"], "higher_is_better": False, "dtype": args.dtype,
                      "data": "synthetic", "config": {"workload": args.workload, "N": N, "K": K},
                      "latency_us": lat}), flush=True)


# ---------------------------------------------------------------- serving

def serve_pool(P, seed):
    """P frames of codes drawn uniformly from the mixed set, Eb/N0 uniform in
    [2.0, 4.5] dB per frame, float32 LLRs, in one pinned buffer in arrival order."""
    import torch

    from paper_1504_00353_gb300 import polar
    nk = synth.MIXED_CODES
    masks, cid, llr, bits = mixed_inputs(P, "f32", seed, ebn0_range=(2.0, 4.5))
    sizes = np.array([nk[c][0] for c in cid], np.int64)
    orow = np.array([(nk[c][1] + 7) // 8 for c in cid], np.int64)
    lo = np.concatenate([[0], np.cumsum(sizes)[:-1]])
    oo = np.concatenate([[0], np.cumsum(orow)[:-1]])
    host_llr = torch.empty(int(sizes.sum()), dtype=torch.float32).pin_memory()
    hv = host_llr.numpy()
    pos = [0] * len(nk)
    want = []
    for i in range(P):
        c = cid[i]
        hv[lo[i]: lo[i] + sizes[i]] = llr[c][pos[c]]
        want.append(bits[c][pos[c]])
        pos[c] += 1
    reqs = np.zeros(P, polar.REQUEST_DTYPE)
    reqs["code_id"], reqs["llr_off"], reqs["out_off"] = cid, lo * 4, oo
    host_out = torch.zeros(int(orow.sum()), dtype=torch.uint8).pin_memory()
    return masks, cid, reqs, host_llr, host_out, want, oo, orow


def serve_run(polar, batch, reqs, host_llr, host_out, rate_fps, n_total, flags, slots,
              budget, max_frames, seed):
    """Poisson arrivals at rate_fps frames/s; requests i use pool entry i % P.
    Returns per-request latencies (ns) and the wall time from the first arrival
    to the last completion."""
    P = reqs.size
    done = np.zeros(P, np.uint64)
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1e9 / rate_fps, n_total)
    srv = polar.polar_server_create(batch, reqs, host_llr, host_out, done, budget, max_frames,
                                    slots, flags)
    t0 = time.monotonic_ns() + 2_000_000
    arr = (t0 + np.cumsum(gaps)).astype(np.int64)
    lat = np.zeros(n_total, np.int64)
    published = harvested = 0
    while harvested < n_total:
        completed, adm, launches = polar.polar_server_progress(srv)
        if completed > harvested:
            idx = np.arange(harvested, completed)
            lat[harvested:completed] = done[idx % P].astype(np.int64) - arr[harvested:completed]
            harvested = completed
        if published < n_total:
            due = int(np.searchsorted(arr, time.monotonic_ns(), side="right"))
            hi = min(due, completed + P, n_total)
            if hi > published:
                polar.polar_server_publish(srv, hi)
                published = hi
    t_end = int(done[(n_total - 1) % P])
    polar.polar_server_destroy(srv)
    return lat, (t_end - arr[0]) * 1e-9, adm, launches


def run_serve(args):
    """Serving loop at offered loads of coded Gbps: Poisson arrivals of frames of
    the mixed code set (float32 LLRs, Eb/N0 uniform in [2, 4.5] dB), continuous
    batching (overlapping launches, admission by device-memory budget) against
    a plain queue decoding one launch per code, one batch at a time."""
    import torch

    from paper_1504_00353_gb300 import polar
    torch.cuda.set_device(0)
    nk = synth.MIXED_CODES
    P = 16384
    masks, cid, reqs, host_llr, host_out, want, oo, orow = serve_pool(P, seed=4)
    mean_coded = float(np.mean([N for N, K in nk]))
    mean_info = float(np.mean([K for N, K in nk]))
    codes = [polar.polar_code_create(N, K, m) for (N, K), m in zip(nk, masks)]
    bshape, bsrc = batch_shape("f32")
    batch = polar.polar_batch_create(codes, False, bshape["threads"], bshape["smem_stage_max"],
                                     bshape["warp_stage_max"], bshape["ctas_per_sm"],
                                     bshape.get("flags", 0))
    budget = 4 << 30
    arms = {"served": dict(flags=0, slots=4, max_frames=4096),
            "plain": dict(flags=polar.SERVE_LAUNCH_PER_CODE, slots=1, max_frames=4096)}
    pools = [p for p in args.serve_pool.split(",") if p]
    # host-to-device copy bandwidth from pinned memory: float32 LLRs cross this
    # link, so it bounds the coded rate the loop can take (4 bytes per coded bit)
    big = torch.empty(1 << 28, dtype=torch.float32).pin_memory()
    dbig = torch.empty(1 << 28, dtype=torch.float32, device="cuda")
    dbig.copy_(big, non_blocking=True)
    torch.cuda.synchronize()
    a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a_.record()
    for _ in range(3):
        dbig.copy_(big, non_blocking=True)
    b_.record()
    torch.cuda.synchronize()
    h2d_gbs = 3 * big.numel() * 4 / (a_.elapsed_time(b_) * 1e-3) / 1e9
    del big, dbig
    results = {}
    gates = {}
    reps = 2
    # clocks sampled once a second here: the serving loop's latency tail is what
    # is measured, and the sampler's device queries are kept rare
    with ClockSampler(0, interval_ms=1000) as clk:
        for pool in pools:
            # pinned host memory (copies over the host link) or device memory (LLR
            # pool in HBM: isolates the scheduler from the host link)
            llr_buf, out_buf = (host_llr, host_out) if pool == "host" else \
                (host_llr.cuda(), host_out.cuda())
            # correctness gate: one pass over the pool through each arm
            gate = {}
            for name, a in arms.items():
                out_buf.zero_()
                serve_run(polar, batch, reqs, llr_buf, out_buf, 2e6, P, a["flags"], a["slots"],
                          budget, a["max_frames"], seed=1)
                gate[name] = out_buf.cpu().numpy().copy()
            gates[pool] = {
                "bits_agree": bool(np.array_equal(gate["served"], gate["plain"])),
                "frame_errors_in_pool": sum(
                    int(not np.array_equal(gate["served"][oo[i]: oo[i] + orow[i]], want[i]))
                    for i in range(P))}
            results[pool] = []
            for load in [float(x) for x in args.loads.split(",")]:
                rate = load * 1e9 / mean_coded
                n_total = int(min(args.serve_max_frames, max(1000, rate * args.serve_seconds)))
                row = {"offered_coded_gbps": load, "frames": n_total, "reps": reps}
                runs = {name: [] for name in arms}
                for r in range(reps):  # arms interleaved, each run with its own arrivals
                    for name, a in arms.items():
                        lat, wall, adm, launches = serve_run(
                            polar, batch, reqs, llr_buf, out_buf, rate, n_total, a["flags"],
                            a["slots"], budget, a["max_frames"], seed=int(load * 7) + 11 + 1000 * r)
                        us = lat * 1e-3
                        runs[name].append({"p50_us": float(np.percentile(us, 50)),
                                           "p99_us": float(np.percentile(us, 99)),
                                           "p999_us": float(np.percentile(us, 99.9)),
                                           "info_gbps": n_total * mean_info / wall / 1e9,
                                           "coded_gbps": n_total * mean_coded / wall / 1e9,
                                           "admissions": adm, "launches": launches,
                                           "frames_per_admission": n_total / max(adm, 1)})
                for name, rs in runs.items():
                    # median over repetitions of each statistic, every repetition kept
                    row[name] = {k: float(np.median([x[k] for x in rs])) for k in rs[0]}
                    row[name]["runs"] = rs
                results[pool].append(row)
                print(json.dumps({"pool": pool, "load": row}), file=sys.stderr, flush=True)
            del llr_buf, out_buf
    top = max(results[pools[0]], key=lambda r: r["offered_coded_gbps"])
    line = {
        "metric": "served info-bit Gbps and p50/p99 frame latency (us)", "mode": "serve",
        "value": top["served"]["info_gbps"], "unit": "Gbps", "n_gpus": 1,
        "higher_is_better": True, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "serve_mixed", "codes": nk, "value_pool": pools[0],
                   "design_db": synth.MIXED_DESIGN_DB, "pools": pools,
                   "ebn0_db": [2.0, 4.5], "arrivals": "Poisson", "pool_frames": P,
                   "device_budget_bytes": budget, "arms": arms, "batch_shape": dict(bshape, source=bsrc),
                   "latency": "completion seen by the serving thread minus scheduled arrival",
                   "h2d_pinned_gbs": h2d_gbs,
                   "h2d_bound_coded_gbps": h2d_gbs * 8 / 32},
        "loads": results, "gates": gates, "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- blocks of the default line

def device_mixed(torch, polar, codes, cid, dtype, seed, ebn0=None, ebn0_range=None):
    """Frames of the mixed code set generated on the device by the library's
    chain: Philox information bits, the device systematic encoder and the BPSK-AWGN
    channel (one Eb/N0, or one drawn per frame from ebn0_range). Frames are
    stored code by code in one flat LLR buffer. Returns (flat LLRs, per-code
    views [m_c, N_c], per-code info bits [m_c, ceil(K_c/8)], per-code element
    offsets of the views in flat)."""
    dt = torch.int8 if dtype == "i8" else torch.float32
    counts = [int((cid == c).sum()) for c in range(len(codes))]
    sizes = [m * code.N for m, code in zip(counts, codes)]
    flat = torch.empty(sum(sizes), dtype=dt, device="cuda")
    views, infos, bases = [], [], []
    base = 0
    rng = np.random.default_rng(seed)
    for c, (code, m) in enumerate(zip(codes, counts)):
        v = flat[base: base + m * code.N].view(m, code.N)
        info = torch.empty((m, code.out_row), dtype=torch.uint8, device="cuda")
        cw = torch.empty((m, (code.N + 7) // 8), dtype=torch.uint8, device="cuda")
        if m:
            polar.polar_random_info(code, info, seed + c)
            polar.polar_encode_systematic_device(code, info, cw)
            if ebn0_range is None:
                polar.polar_channel_awgn(code, cw, v, ebn0, seed + 100 + c)
            else:
                for j, db in enumerate(rng.uniform(*ebn0_range, m)):
                    polar.polar_channel_awgn(code, cw[j:j + 1], v[j:j + 1], float(db), seed + 100 + c,
                                             frame0=j)
        views.append(v)
        infos.append(info)
        bases.append(base)
        base += m * code.N
    torch.cuda.synchronize()
    return flat, views, infos, bases


def mixed_block(args, n=None, steps=10, warmup=3):
    """Config-3 comparison for the default line: 65,536 int8 frames of the five
    mixed codes, one persistent launch of the mixed-batch decoder replayed from a
    CUDA graph, against one launch per code with each code's own tuned decoder.
    Inputs come from the library's device chain (seeded)."""
    import torch
    from concurrent.futures import ThreadPoolExecutor

    from paper_1504_00353_gb300 import autotune, polar
    dtype = "i8"
    n = n or synth.MIXED_FRAMES
    nk = synth.MIXED_CODES
    masks = [synth.frozen_mask(N, K, synth.MIXED_DESIGN_DB) for N, K in nk]
    codes = [polar.polar_code_create(N, K, m) for (N, K), m in zip(nk, masks)]
    cid = np.random.default_rng(3).integers(0, len(nk), n)
    counts = [int((cid == c).sum()) for c in range(len(nk))]
    shapes = []
    for c, (N, K) in enumerate(nk):
        sh, src = autotune.shape_for(N, K, masks[c], dtype,
                                     default=dict(threads=32, smem_stage_max=512,
                                                  warp_stage_max=2048, ctas_per_sm=0))
        sh.setdefault("stage_channel", 2)
        shapes.append((sh, src))
    bshape, bsrc = autotune.batch_shape(dtype)
    t_c = time.perf_counter()
    with ThreadPoolExecutor(max_workers=6) as ex:
        futs = [ex.submit(autotune.configure, codes[c], dtype, shapes[c][0], counts[c])
                for c in range(len(nk))]
        # the batch kernel gets handles of its own (compiled concurrently)
        bcodes = [polar.polar_code_create(N, K, m) for (N, K), m in zip(nk, masks)]
        fb = ex.submit(polar.polar_batch_create, bcodes, True, bshape["threads"],
                       bshape["smem_stage_max"], bshape["warp_stage_max"], bshape["ctas_per_sm"],
                       bshape.get("flags", 0))
        for f in futs:
            f.result()
        batch = fb.result()
    t_c = time.perf_counter() - t_c
    flat, views, infos, bases = device_mixed(torch, polar, codes, cid, dtype, seed=3,
                                             ebn0=synth.MIXED_DESIGN_DB)
    orow = [code.out_row for code in codes]
    obase = np.concatenate([[0], np.cumsum([m * r for m, r in zip(counts, orow)])])
    out_b = torch.zeros(int(obase[-1]), dtype=torch.uint8, device="cuda")
    outs = [out_b.new_zeros((m, r)) for m, r in zip(counts, orow)]
    # descriptors, longest code first (the order CTAs claim frames in)
    ids, lo, oo = [], [], []
    for c in sorted(range(len(nk)), key=lambda c: -nk[c][0]):
        m = counts[c]
        ids.append(np.full(m, c, np.int32))
        lo.append(bases[c] + np.arange(m, dtype=np.int64) * nk[c][0])
        oo.append(obase[c] + np.arange(m, dtype=np.int64) * orow[c])
    d_ids, d_lo, d_oo = (torch.from_numpy(np.concatenate(x)).cuda() for x in (ids, lo, oo))
    dec = polar.polar_decode_i8

    def plain(_):
        for c in range(len(nk)):
            dec(codes[c], views[c], outs[c])

    stream = torch.cuda.current_stream()
    s2 = torch.cuda.Stream()
    s2.wait_stream(stream)
    with torch.cuda.stream(s2):
        polar.polar_batch_decode(batch, d_ids, d_lo, d_oo, flat, out_b, stream=s2)
    stream.wait_stream(s2)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        polar.polar_batch_decode(batch, d_ids, d_lo, d_oo, flat, out_b)
    out_b.zero_()
    plain(0)
    graph.replay()
    torch.cuda.synchronize()
    agree = bool(torch.equal(out_b, torch.cat([o.reshape(-1) for o in outs])))
    ferr = sum(int((outs[c] != infos[c]).any(dim=1).sum()) for c in range(len(nk)))
    with ClockSampler(0) as clk:
        plain_ms, _ = device_timed(torch, stream, plain, steps, warmup, 1)
        batched_ms, _ = device_timed(torch, stream, lambda i: graph.replay(), steps, warmup, 1)
    info_bits = sum(m * K for m, (N, K) in zip(counts, nk))
    return {
        "what": "one persistent launch over all frames, replayed from a CUDA graph (batched) "
                "vs one launch per code (plain), same device buffers",
        "frames": n, "codes": nk, "frames_per_code": counts, "llr": dtype,
        "design_db": synth.MIXED_DESIGN_DB, "ebn0_db": synth.MIXED_DESIGN_DB,
        "inputs": f"{flat.numel() * flat.element_size() / 2**20:.0f} MiB on the device (larger "
                  "than L2), generated by the library's Philox/encoder/AWGN chain, stored code by code",
        "batched": {"gbps": info_bits * steps / (batched_ms * 1e-3) / 1e9,
                    "step_ms": batched_ms / steps, "launches_per_step": 1, "cuda_graph": True,
                    "shape": dict(bshape, source=bsrc), "launch": polar.polar_batch_info(batch)},
        "plain": {"gbps": info_bits * steps / (plain_ms * 1e-3) / 1e9,
                  "step_ms": plain_ms / steps, "launches_per_step": len(nk),
                  "shapes": [dict(sh, source=src) for sh, src in shapes]},
        "batched_over_plain": plain_ms / batched_ms,
        "bits_agree": agree, "frame_errors": ferr, "compile_s": t_c, "steps": steps,
        "warmup": warmup, "clocks": clk.summary(),
    }


def serve_block(args, loads=(1, 10, 50, 200), seconds=0.5, max_frames=40_000):
    """Config-4 comparison for the default line: Poisson arrivals of float32
    frames of the mixed codes (Eb/N0 uniform in [2.0, 4.5] dB per frame) through
    the serving loop (continuous batching: overlapping launches, admission by
    device-memory budget) against a plain queue (one launch per code, one batch
    at a time), the request pool resident in HBM. One run per load; the full
    comparison with two runs per cell and a pinned-host pool is --mode serve."""
    import torch

    from paper_1504_00353_gb300 import autotune, polar
    nk = synth.MIXED_CODES
    P = 16384
    masks = [synth.frozen_mask(N, K, synth.MIXED_DESIGN_DB) for N, K in nk]
    codes = [polar.polar_code_create(N, K, m) for (N, K), m in zip(nk, masks)]
    cid = np.random.default_rng(4).integers(0, len(nk), P)
    _, views, infos, _ = device_mixed(torch, polar, codes, cid, "f32", seed=4,
                                      ebn0_range=(2.0, 4.5))
    counts = [int((cid == c).sum()) for c in range(len(nk))]
    orow = [code.out_row for code in codes]
    # the pool in arrival order, each request's frame right after the previous
    # one's (as a stream of requests arrives), so that the loop moves runs of
    # requests with one copy
    sizes = np.array([nk[c][0] for c in cid], np.int64)
    osz = np.array([orow[c] for c in cid], np.int64)
    lo = np.concatenate([[0], np.cumsum(sizes)[:-1]])
    oo = np.concatenate([[0], np.cumsum(osz)[:-1]])
    flat = torch.empty(int(sizes.sum()), dtype=torch.float32, device="cuda")
    rank = np.zeros(P, np.int64)
    seen = [0] * len(nk)
    for i, c in enumerate(cid):
        rank[i] = seen[c]
        seen[c] += 1
        flat[int(lo[i]): int(lo[i] + sizes[i])].copy_(views[c][rank[i]])
    reqs = np.zeros(P, polar.REQUEST_DTYPE)
    reqs["code_id"] = cid
    reqs["llr_off"] = lo * 4
    reqs["out_off"] = oo
    out_buf = torch.zeros(int(osz.sum()), dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    del views
    bshape, bsrc = autotune.batch_shape("f32")
    batch = polar.polar_batch_create(codes, False, bshape["threads"], bshape["smem_stage_max"],
                                     bshape["warp_stage_max"], bshape["ctas_per_sm"],
                                     bshape.get("flags", 0))
    budget = 4 << 30
    arms = {"served": dict(flags=0, slots=4, max_frames=4096),
            "plain": dict(flags=polar.SERVE_LAUNCH_PER_CODE, slots=1, max_frames=4096)}
    mean_coded = float(np.mean([N for N, K in nk]))
    mean_info = float(np.mean([K for N, K in nk]))
    gate = {}
    for name, a in arms.items():
        out_buf.zero_()
        serve_run(polar, batch, reqs, flat, out_buf, 2e6, P, a["flags"], a["slots"], budget,
                  a["max_frames"], seed=1)
        torch.cuda.synchronize()
        gate[name] = out_buf.clone()
    got = gate["served"].cpu().numpy()
    info_h = [x.cpu().numpy() for x in infos]
    row_err = sum(int(not np.array_equal(got[oo[i]: oo[i] + osz[i]], info_h[cid[i]][rank[i]]))
                  for i in range(P))
    rows = []
    with ClockSampler(0, interval_ms=1000) as clk:
        for load in loads:
            rate = load * 1e9 / mean_coded
            n_total = int(min(max_frames, max(1000, rate * seconds)))
            row = {"offered_coded_gbps": load, "frames": n_total}
            for name, a in arms.items():
                lat, wall, adm, launches = serve_run(
                    polar, batch, reqs, flat, out_buf, rate, n_total, a["flags"], a["slots"],
                    budget, a["max_frames"], seed=int(load * 7) + 11)
                us = lat * 1e-3
                row[name] = {"p50_us": float(np.percentile(us, 50)),
                             "p99_us": float(np.percentile(us, 99)),
                             "p999_us": float(np.percentile(us, 99.9)),
                             "info_gbps": n_total * mean_info / wall / 1e9,
                             "admissions": adm, "launches": launches}
            rows.append(row)
    return {
        "what": "served (continuous batching, 4 launch slots) vs plain (one launch per code, "
                "one batch at a time); latency = completion seen by the serving thread minus "
                "scheduled Poisson arrival",
        "pool": f"{P} float32 frames of the mixed codes in HBM, Eb/N0 uniform in [2.0, 4.5] dB "
                "per frame (library device chain, seeded)",
        "loads": rows, "bits_agree": bool(torch.equal(gate["served"], gate["plain"])),
        "frame_errors_in_pool": row_err, "pool_frames": P,
        "batch_shape": dict(bshape, source=bsrc), "clocks": clk.summary(),
    }


# ---------------------------------------------------------------- error rates

FER_POINTS = {
    "n1024_k512_2.5db": ([1.0, 1.5, 2.0, 2.5, 3.0], 400_000),
    "n32768_k29492_4.0db": ([3.75, 4.0, 4.25, 4.5, 4.75], 40_000),
}


def run_fer(args):
    """Frame and bit error rates over BPSK-AWGN, float32 against int8 LLRs (x8,
    +-127), every step on the GPU (Philox bits and noise, device encoder,
    specialised decoder, error count)."""
    import torch

    from paper_1504_00353_gb300 import polar
    torch.cuda.set_device(0)
    rows = []
    batch = 16384
    for wl_name, (points, frames) in FER_POINTS.items():
        wl = synth.WORKLOADS[wl_name]
        N, K = wl["N"], wl["K"]
        mask = synth.frozen_mask(N, K, wl["design_db"])
        for dtype in ("f32", "i8"):
            code = polar.polar_code_create(N, K, mask)
            shape, _ = tuned_or(N, K, mask, dtype)
            shape.setdefault("stage_channel", 2)
            compile_shape(code, dtype, shape, batch)
            polar.polar_fer_run(code, dtype == "i8", points[0], 0, batch, batch)  # warm-up
            for db in points:
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                fe, be = polar.polar_fer_run(code, dtype == "i8", db, 2024, frames, batch)
                dt = time.perf_counter() - t0
                rows.append({"workload": wl_name, "llr": dtype, "ebn0_db": db, "frames": frames,
                             "frame_errors": fe, "bit_errors": be, "fer": fe / frames,
                             "ber": be / (frames * K), "seconds": dt,
                             "chain_info_gbps": frames * K / dt / 1e9})
                print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
    line = {"metric": "frame / bit error rate, float32 vs int8 LLRs", "mode": "fer",
            "data": "synthetic", "config": {"workloads": list(FER_POINTS), "batch": batch,
                                            "channel": "BPSK-AWGN, Philox-4x32-10 + Box-Muller",
                                            "seed": 2024},
            "points": rows}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.mode == "fer":
        return run_fer(args)
    if args.mode == "mixed":
        return run_mixed(args)
    if args.mode == "serve":
        return run_serve(args)
    if args.mode == "latency":
        return run_latency(args)
    if args.impl == "reference":
        # the CPU oracle arm: rank 0 alone runs and prints, other ranks exit
        if int(os.environ.get("RANK", "0")) == 0:
            run_reference(args, 1, 0)
        return
    world, rank, local = dist_init(args)
    run_native(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
