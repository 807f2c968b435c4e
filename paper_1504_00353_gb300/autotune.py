"""Launch-shape autotuner for the specialised decoders.

For one code and LLR type it times candidate launch shapes on the GPU and keeps
the fastest: threads per CTA (threads per frame), the largest alpha stage held
in shared memory, the node size up to which warp 0 works alone (the tree depth
where work switches from CTA-wide to warp-level), and the cap on resident CTAs
(frames) per SM, which also sets the kernel's register budget. The search is
coordinate-wise (threads, then stage cap, then warp threshold, then CTAs per
SM); candidates of one round are compiled in parallel host threads (NVRTC) and
timed one after another with CUDA events on a batch that fills the GPU.

For a mixed batch the kernel has one block size for every code: the tuner picks
the block size that minimises the mix's expected time per frame, then the
per-code stage cap and warp threshold at that block size.

Results are kept in a JSON table (``tuned_shapes.json`` beside this file) keyed
by device name, code (N, K, hash of the frozen mask) and LLR type; ``lookup``
returns an entry for a code, falling back to any entry with the same N, K and
LLR type.
"""
from __future__ import annotations

import hashlib
import json
import os
import statistics
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

from . import polar

TABLE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned_shapes.json")
THREADS = (32, 64, 128, 256)
STAGES = (256, 512, 1024, 2048, 4096)
WARPS = (256, 512, 1024, 2048, 4096)
_lock = threading.Lock()


def mask_hash(mask) -> str:
    return hashlib.sha1(np.ascontiguousarray(np.asarray(mask, np.uint8)).tobytes()).hexdigest()[:12]


def code_key(N: int, K: int, mask, dtype: str, latency: bool = False) -> str:
    return f"{N}_{K}_{mask_hash(mask)}_{dtype}" + ("_lat" if latency else "")


def device_name() -> str:
    import torch
    return torch.cuda.get_device_name()


def load_table(path: str = TABLE) -> dict:
    if not os.path.exists(path):
        return {}
    with open(path) as fh:
        return json.load(fh)


def save_table(table: dict, path: str = TABLE):
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as fh:
        json.dump(table, fh, indent=1, sort_keys=True)
        fh.write("\n")
    os.replace(tmp, path)


def lookup(N: int, K: int, mask, dtype: str, table: dict | None = None, device: str | None = None,
           latency: bool = False):
    """Tuned shape for a code (batch-1 shape with latency=True), or None. Exact
    mask first, then the same (N, K, dtype)."""
    table = load_table() if table is None else table
    dev = table.get(device or device_name(), {})
    hit = dev.get(code_key(N, K, mask, dtype, latency))
    if hit:
        return hit
    want = 5 if latency else 4
    for k, v in sorted(dev.items()):
        parts = k.split("_")
        if (len(parts) == want and parts[0] == str(N) and parts[1] == str(K) and parts[3] == dtype
                and (not latency or parts[4] == "lat")):
            return v
    return None


def synthetic_llr(N: int, n_frames: int, dtype: str, ebn0_db: float, rate: float, seed: int = 0):
    """BPSK-AWGN LLRs of the all-zero codeword (a codeword of every polar code),
    generated on the device: the decoder's work does not depend on the values."""
    import torch
    g = torch.Generator(device="cuda").manual_seed(seed)
    s2 = 1.0 / (2.0 * rate * 10.0 ** (ebn0_db / 10.0))
    y = 1.0 + s2 ** 0.5 * torch.randn((n_frames, N), generator=g, device="cuda")
    llr = (2.0 / s2) * y
    if dtype == "i8":
        return torch.clamp(torch.round(8.0 * llr), -127, 127).to(torch.int8)
    return llr.float().contiguous()


def frames_for(N: int, sms: int) -> int:
    """Batch that keeps every SM busy with several waves of small CTAs."""
    return int(max(sms * 48, min(1 << 17, (1 << 26) // N)))


SHAPE_KEYS = ("threads", "smem_stage_max", "warp_stage_max", "ctas_per_sm", "stage_channel",
              "reg_subtree", "frames_per_cta", "local_leaves", "compile_form")
SHAPE_DEFAULTS = dict(ctas_per_sm=0, stage_channel=2, reg_subtree=256, frames_per_cta=1,
                      local_leaves=0, compile_form="auto")


def _shape_key(s: dict) -> tuple:
    return tuple(s.get(k, SHAPE_DEFAULTS.get(k, 0)) for k in SHAPE_KEYS)


def _shape(key: tuple) -> dict:
    return dict(zip(SHAPE_KEYS, key))


def apply_shape(code, dtype: str, shape: dict, n_frames: int):
    """Set a tuned shape on a code and compile its specialised decoder."""
    sh = dict(SHAPE_DEFAULTS, **shape)
    polar.polar_code_set_launch(code, dtype == "i8", threads=sh["threads"],
                                smem_stage_max=sh["smem_stage_max"],
                                warp_stage_max=sh["warp_stage_max"],
                                ctas_per_sm=sh["ctas_per_sm"], stage_channel=sh["stage_channel"])
    polar.polar_code_set_frames_per_cta(code, dtype == "i8", sh["frames_per_cta"])
    polar.polar_code_compile(code, dtype == "i8", n_frames, sh["reg_subtree"],
                             COMPILE_FORM[sh["compile_form"]] |
                             (polar.COMPILE_LOCAL_LEAVES if sh["local_leaves"] else 0))


def _compile(N, K, mask, dtype, shape, n_frames):
    code = polar.polar_code_create(N, K, mask)
    try:
        apply_shape(code, dtype, shape, n_frames)
    except polar.PolarError:
        return None
    return code


def _warm(fn, seconds=0.05):
    """Run fn until `seconds` of wall time have passed (at least 3 times), so
    that the GPU has left its idle clocks before a candidate is timed."""
    import time

    import torch
    t0, k = time.perf_counter(), 0
    while k < 3 or time.perf_counter() - t0 < seconds:
        fn()
        torch.cuda.synchronize()
        k += 1


def _time_latency(code, dtype, llr, out, reps=30) -> float:
    """Device time of a one-frame decode, queued behind a spin so that the host
    call overhead is not inside the events (median of reps)."""
    import torch
    dec = polar.polar_decode_i8 if dtype == "i8" else polar.polar_decode
    one_in, one_out = llr[:1], out[:1]
    _warm(lambda: dec(code, one_in, one_out), 0.02)
    ts = []
    for _ in range(reps):
        torch.cuda._sleep(200_000)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        dec(code, one_in, one_out)
        b.record()
        b.synchronize()
        ts.append(a.elapsed_time(b) * 1e-3)
    return statistics.median(ts)


def _time(code, dtype, llr, out, reps=5) -> float:
    import torch
    dec = polar.polar_decode_i8 if dtype == "i8" else polar.polar_decode
    _warm(lambda: dec(code, llr, out))
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        dec(code, llr, out)
        b.record()
        b.synchronize()
        ts.append(a.elapsed_time(b) * 1e-3)
    return statistics.median(ts)


class CodeTuner:
    """Times launch shapes of one code; remembers every shape it measured."""

    def __init__(self, N, K, mask, dtype, ebn0_db=3.0, n_frames=None, workers=8, log=None,
                 latency=False):
        import torch
        self.N, self.K, self.mask, self.dtype = N, K, np.asarray(mask, np.uint8), dtype
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        self.latency = latency
        self.n_frames = 1 if latency else (n_frames or frames_for(N, sms))
        self.llr = synthetic_llr(N, self.n_frames, dtype, ebn0_db, K / N)
        self.out = torch.empty((self.n_frames, (K + 7) // 8), dtype=torch.uint8, device="cuda")
        self.workers = workers
        self.seen: dict[tuple, float] = {}  # shape key -> seconds per frame
        self.log = log

    def clamp(self, s) -> dict:
        """The shape the library would use: stage cap at most N/2, warp threshold
        at most N, register subtree at most N (larger values change nothing)."""
        s = dict(SHAPE_DEFAULTS, **s)
        return dict(s, smem_stage_max=min(s["smem_stage_max"], max(self.N // 2, 64)),
                    warp_stage_max=min(s["warp_stage_max"], max(self.N, 256)),
                    reg_subtree=max(32, min(s["reg_subtree"], self.N)))

    def measure(self, shapes) -> None:
        todo = []
        for s in map(self.clamp, shapes):
            if _shape_key(s) not in self.seen and all(_shape_key(s) != _shape_key(x) for x in todo):
                todo.append(s)
        if not todo:
            return
        with ThreadPoolExecutor(max_workers=self.workers) as ex:
            codes = list(ex.map(lambda s: _compile(self.N, self.K, self.mask, self.dtype, s,
                                                   self.n_frames), todo))
        for s, code in zip(todo, codes):
            if code is None:
                self.seen[_shape_key(s)] = float("inf")
                continue
            launch = polar.polar_code_get_launch(code, self.dtype == "i8", self.n_frames)
            if not launch["unrolled"]:
                t = float("inf")
            elif self.latency:
                t = _time_latency(code, self.dtype, self.llr, self.out)
            else:
                t = _time(code, self.dtype, self.llr, self.out) / self.n_frames
            self.seen[_shape_key(s)] = t
            if self.log:
                what = (f"{t * 1e6:.1f} us" if self.latency else
                        f"{self.K / t / 1e9 if t < float('inf') else 0:.1f} Gbps")
                self.log(f"  ({self.N},{self.K}) {self.dtype} {_shape_key(s)}: {what}")
            del code

    def best(self, threads=None) -> tuple[dict, float]:
        cands = [(t, k) for k, t in self.seen.items() if threads is None or k[0] == threads]
        t, k = min(cands)
        return _shape(k), t

    def tune_latency(self) -> tuple[dict, float]:
        """Batch-1 shape: one CTA, every stage in shared memory when it fits
        (stage cap 0 = the library's choice), register subtrees up to 1024 leaves."""
        base = dict(smem_stage_max=0, warp_stage_max=1024, ctas_per_sm=0, stage_channel=1,
                    reg_subtree=256)
        self.measure([dict(base, threads=t) for t in (128, 256, 512, 1024)])
        cur, _ = self.best()
        self.measure([dict(cur, warp_stage_max=w) for w in (256, 512, 1024, 2048, 4096)])
        cur, _ = self.best()
        self.measure([dict(cur, reg_subtree=r) for r in (256, 512, 1024)])
        cur, _ = self.best()
        self.measure([dict(cur, stage_channel=c) for c in (1, 2)])
        cur, _ = self.best()
        self.measure([dict(cur, local_leaves=v) for v in (0, 1)])
        return self.best()

    def tune(self, threads_options=THREADS, fixed_threads=None, tune_ctas=True) -> tuple[dict, float]:
        def default(t):
            return dict(threads=t, smem_stage_max=512 if t == 32 else 2048, warp_stage_max=2048,
                        ctas_per_sm=0)
        if fixed_threads is None:
            self.measure([default(t) for t in threads_options])
            # one warp per frame, several frames per CTA, at two stage caps
            if tune_ctas:
                self.measure([dict(default(32), frames_per_cta=f, smem_stage_max=s)
                              for f in (2, 4) for s in (512, 1024)])
            cur, _ = self.best()
        else:
            self.measure([default(fixed_threads)])
            cur, _ = self.best(fixed_threads)
        T = cur["threads"]
        self.measure([dict(cur, smem_stage_max=s) for s in STAGES])
        cur, _ = self.best(T)
        if T > 32:
            self.measure([dict(cur, warp_stage_max=w) for w in WARPS])
            cur, _ = self.best(T)
        if tune_ctas:  # fewer resident frames per SM, more registers per thread
            top = min(32, 2048 // T)
            self.measure([dict(cur, ctas_per_sm=c) for c in (8, 12, 16, 20, 24, 28) if c < top])
            cur, _ = self.best(T)
            if T == 32:  # several frames per CTA, one per warp (ctas_per_sm counts CTAs)
                self.measure([dict(cur, frames_per_cta=f,
                                   ctas_per_sm=(cur["ctas_per_sm"] + f - 1) // f if cur["ctas_per_sm"] else 0)
                              for f in (2, 4)])
            cur, _ = self.best(T)
            # the inlined decoder against one with shared code for equal subtrees
            self.measure([dict(cur, compile_form=f) for f in ("auto", "subtrees")])
            cur, _ = self.best(T)
            # register-resident subtree size: the depth below which a frame's
            # tree is decoded in registers instead of through memory stages
            self.measure([dict(cur, reg_subtree=r) for r in (256, 512)])
        return self.best(T)


def tune_code(N, K, mask, dtype, table=None, save=True, tuner=None, **kw) -> dict:
    """Tune one code (throughput, or batch-1 with latency=True); store and return
    its entry."""
    tuner = tuner or CodeTuner(N, K, mask, dtype, **kw)
    if tuner.latency:
        shape, t = tuner.tune_latency()
        entry = dict(shape, latency_us=t * 1e6, n_frames=1)
    else:
        shape, t = tuner.tune()
        entry = dict(shape, gbps=K / t / 1e9, n_frames=tuner.n_frames)
    with _lock:
        tab = load_table() if table is None else table
        tab.setdefault(device_name(), {})[code_key(N, K, mask, dtype, tuner.latency)] = entry
        if save:
            save_table(tab)
    return entry


def mixed_sample(tuners, n_frames, seed=0):
    """A device-resident mixed batch for timing: frames of the tuners' codes in
    equal expected shares, stored code by code, descriptors longest code first
    (the order a batch is claimed in). Returns (code_id, llr_off, out_off, llr,
    out) tensors."""
    import torch
    rng = np.random.default_rng(seed)
    counts = np.bincount(rng.integers(0, len(tuners), n_frames), minlength=len(tuners))
    parts, ids, lo, oo = [], [], [], []
    pos = opos = 0
    for c in sorted(range(len(tuners)), key=lambda c: -tuners[c].N):
        tu, m = tuners[c], int(counts[c])
        idx = torch.arange(m, device="cuda") % tu.n_frames
        parts.append(tu.llr[idx].reshape(-1))
        ids += [c] * m
        lo += [pos + j * tu.N for j in range(m)]
        oo += [opos + j * ((tu.K + 7) // 8) for j in range(m)]
        pos += m * tu.N
        opos += m * ((tu.K + 7) // 8)
    dev = lambda a, t: torch.tensor(a, dtype=t, device="cuda")
    out = torch.empty(opos, dtype=torch.uint8, device="cuda")
    return (dev(ids, torch.int32), dev(lo, torch.int64), dev(oo, torch.int64), torch.cat(parts), out)


def time_batch(batch, sample, reps=5) -> float:
    import torch
    ids, lo, oo, llr, out = sample
    _warm(lambda: polar.polar_batch_decode(batch, ids, lo, oo, llr, out))
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        polar.polar_batch_decode(batch, ids, lo, oo, llr, out)
        b.record()
        b.synchronize()
        ts.append(a.elapsed_time(b) * 1e-3)
    return statistics.median(ts)


def tune_batch(tuners, weights=None, sample_frames=16384, workers=6, log=None) -> dict:
    """Shape of a mixed-batch decoder over the tuners' codes. (1) One block size
    for all codes: least expected time per frame of the mix, each code at its
    default stage cap and warp threshold in its own kernel. (2) Per-code stage
    cap and warp threshold tuned at that block size. (3) The batch kernel
    itself, timed on a mixed sample: one kernel's shared memory (the largest
    code's) and register budget bound every code's resident frames, so caps on
    the stage size and on resident CTAs per SM are tried jointly. Returns
    dict(threads, smem_stage_max[], warp_stage_max[], ctas_per_sm, gbps, ...)."""
    w = np.ones(len(tuners)) / len(tuners) if weights is None else np.asarray(weights, float)
    for tu in tuners:
        tu.measure([dict(threads=t, smem_stage_max=512 if t == 32 else 2048, warp_stage_max=2048,
                         ctas_per_sm=0) for t in THREADS])
    cost = {t: float(sum(wi * tu.best(t)[1] for wi, tu in zip(w, tuners))) for t in THREADS}
    T = min(cost, key=cost.get)
    shapes = [tu.tune(fixed_threads=T, tune_ctas=False)[0] for tu in tuners]
    S0 = [s["smem_stage_max"] for s in shapes]
    W0 = [s["warp_stage_max"] for s in shapes]
    codes = [polar.polar_code_create(tu.N, tu.K, tu.mask) for tu in tuners]
    cands = []
    for cap in (None, 2048, 1024, 512, 256):
        S = [min(x, cap) if cap else x for x in S0]
        for cps in ((0, 28, 24) if T == 32 else (0,)):
            c = (tuple(S), cps)
            if c not in [x for x in cands]:
                cands.append(c)

    def build(c):
        try:
            return polar.polar_batch_create(codes, tuners[0].dtype == "i8", T, list(c[0]), W0, c[1])
        except polar.PolarError:
            return None

    with ThreadPoolExecutor(max_workers=workers) as ex:
        batches = list(ex.map(build, cands))
    sample = mixed_sample(tuners, sample_frames)
    ids = sample[0].cpu().numpy()
    bits = float(sum(tuners[c].K for c in ids))
    results = []
    for c, b in zip(cands, batches):
        if b is None:
            continue
        t = time_batch(b, sample)
        results.append((t, c, polar.polar_batch_info(b)))
        if log:
            log(f"  batch T={T} S={list(c[0])} cps={c[1]}: {bits / t / 1e9:.1f} Gbps "
                f"(grid {results[-1][2]['grid']})")
        del b
    t, (S, cps), info = min(results, key=lambda r: r[0])
    flags, threads = 0, T
    # the same stage caps with subtree functions shared by all bodies, and (one
    # warp per frame) with two or four frames per CTA
    trials = [(T, polar.COMPILE_OUTLINE_SUBTREES, cps)]
    if T == 32:
        trials += [(32 * f, polar.BATCH_FRAME_PER_WARP, (cps + f - 1) // f if cps else 0)
                   for f in (2, 4)]
    for tt, fl, cc in trials:
        try:
            b = polar.polar_batch_create(codes, tuners[0].dtype == "i8", tt, list(S), W0, cc, fl)
        except polar.PolarError:
            continue
        t2 = time_batch(b, sample)
        if log:
            log(f"  batch T={tt} S={list(S)} cps={cc} flags={fl}: {bits / t2 / 1e9:.1f} Gbps")
        if t2 < t:
            t, flags, threads, cps = t2, fl, tt, cc
            info = polar.polar_batch_info(b)
        del b
    return dict(threads=threads, smem_stage_max=list(S), warp_stage_max=W0, ctas_per_sm=cps,
                flags=flags,
                gbps=bits / t / 1e9, grid=info["grid"], sample_frames=sample_frames,
                per_code_gbps=[tu.K / tu.best(T)[1] / 1e9 for tu in tuners],
                expected_s_per_frame={str(k): v for k, v in cost.items()})


def main(argv=None):
    import argparse

    import torch

    from . import synth
    p = argparse.ArgumentParser(description="tune launch shapes on the current GPU")
    p.add_argument("--workload", action="append", default=[],
                   help="a named workload of synth.WORKLOADS (repeatable)")
    p.add_argument("--mixed", action="store_true", help="the mixed-length code set")
    p.add_argument("--dtype", action="append", default=[], choices=["f32", "i8"])
    p.add_argument("--latency", action="store_true",
                   help="tune the batch-1 (latency) shape of the named workloads instead")
    p.add_argument("--out", default=TABLE)
    a = p.parse_args(argv)
    torch.cuda.set_device(0)
    table = load_table(a.out)
    # (N, K, mask, design dB, frames: the workload's batch, else enough to fill the GPU)
    codes = [(w["N"], w["K"], synth.frozen_mask(w["N"], w["K"], w["design_db"]), w["design_db"],
              w["n_frames"]) for w in (synth.WORKLOADS[n] for n in a.workload)]
    if a.mixed:
        codes += [(N, K, synth.frozen_mask(N, K, synth.MIXED_DESIGN_DB), synth.MIXED_DESIGN_DB,
                   None) for N, K in synth.MIXED_CODES]
    for dtype in a.dtype or ["i8"]:
        tuners = []
        for N, K, mask, db, nf in codes:
            tu = CodeTuner(N, K, mask, dtype, ebn0_db=db, n_frames=nf, log=print,
                           latency=a.latency)
            e = tune_code(N, K, mask, dtype, table=table, save=False, tuner=tu)
            print(f"({N},{K}) {dtype}: {e}", flush=True)
            save_table(table, a.out)
            tuners.append((db, tu))
        if a.mixed and not a.latency:
            mixed = [tu for db, tu in tuners if db == synth.MIXED_DESIGN_DB and
                     (tu.N, tu.K) in synth.MIXED_CODES][-len(synth.MIXED_CODES):]
            b = tune_batch(mixed, log=print)
            table.setdefault(device_name(), {})[f"mixed_{dtype}"] = b
            print(f"mixed {dtype}: {b}", flush=True)
            save_table(table, a.out)
        del tuners



# ---------------------------------------------------------------- shapes in use

# Launch shapes used when the table holds no entry for a code on this device
# (chosen by measurement on GB300): threads per CTA, largest shared-memory alpha
# stage, warp-run threshold, channel read in place (stage_channel 2).
FALLBACK = {
    (32768, 29492, "f32"): dict(threads=128, smem_stage_max=2048, warp_stage_max=2048,
                                stage_channel=2),
    (32768, 29492, "i8"): dict(threads=32, smem_stage_max=512, stage_channel=2),
    (1024, 512, "f32"): dict(threads=32, stage_channel=2),
    (1024, 512, "i8"): dict(threads=32, stage_channel=2),
}
# Batch-1 (latency) shapes: one CTA, every stage in shared memory.
FALLBACK_LATENCY = {(32768, 29492): dict(threads=256, warp_stage_max=1024)}
COMPILE_FORM = {"auto": 0, "subtrees": 1, "memory": 2, "compact": 3, "full": 4}


def shape_for(N: int, K: int, mask, dtype: str, latency: bool = False, default=None):
    """The launch shape a decode of this code uses: the table's entry for this
    device (batch-1 entry with latency=True), else the measured fallback, else
    `default` (or the library's own choice). Returns (shape dict, source)."""
    try:
        e = lookup(N, K, mask, dtype, latency=latency)
    except Exception:  # no table, or no device to name
        e = None
    if e:
        return {k: e[k] for k in SHAPE_KEYS if k in e}, "tuned"
    fb = FALLBACK_LATENCY.get((N, K)) if latency else FALLBACK.get((N, K, dtype))
    if fb is None:
        fb = default or {}
    return dict(fb), "default"


def configure(code, dtype: str, shape: dict, n_frames: int, interpreter: bool = False,
              form: str = "auto"):
    """Set a launch shape (polar_code_set_launch arguments plus reg_subtree and
    frames_per_cta) on a code and compile its specialised decoder for decodes of
    n_frames frames (unless timing the interpreter)."""
    sh = dict(shape)
    reg = sh.pop("reg_subtree", 0)
    fpc = sh.pop("frames_per_cta", 1)
    local = polar.COMPILE_LOCAL_LEAVES if sh.pop("local_leaves", 0) else 0
    tuned_form = sh.pop("compile_form", "auto")
    if form == "auto":  # an explicit form from the caller wins over the table's
        form = tuned_form
    polar.polar_code_set_launch(code, dtype == "i8", **sh)
    polar.polar_code_set_frames_per_cta(code, dtype == "i8", fpc)
    if not interpreter:
        polar.polar_code_compile(code, dtype == "i8", n_frames, reg, COMPILE_FORM[form] | local)


def batch_shape(dtype: str):
    """Shape of the mixed-batch decoder over the mixed code set: the table's
    entry for this device, else one warp per frame with the library's per-code
    choices. Returns (dict of polar_batch_create arguments, source)."""
    try:
        e = load_table().get(device_name(), {}).get(f"mixed_{dtype}")
    except Exception:
        e = None
    if e:
        return dict(threads=e["threads"], smem_stage_max=e["smem_stage_max"],
                    warp_stage_max=e["warp_stage_max"], ctas_per_sm=e.get("ctas_per_sm", 0),
                    flags=e.get("flags", 0)), "tuned"
    return dict(threads=32, smem_stage_max=None, warp_stage_max=None, ctas_per_sm=0,
                flags=0), "default"


if __name__ == "__main__":
    main()
