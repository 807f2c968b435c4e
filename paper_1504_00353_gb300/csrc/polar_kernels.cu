// Fast-SSC decoding kernels for sm_103a (GB300).
//
// Method: Giard et al., "Low-Latency Software Polar Decoders" (arXiv 1504.00353),
// Sec. II-C/II-D. One CTA decodes one frame at a time and loops over frames
// (persistent grid sized to the resident-CTA count). The frame's operation list
// (the depth-first Fast-SSC call list of Listing 1, built on the host) is
// interpreted in order, at three granularities:
//   - wide operations (node size N_v > warp_stage_max) use every thread of the
//     CTA, loads issued ahead of use, one __syncthreads after each;
//   - narrower operations run on warp 0 alone with __syncwarp between them while
//     the other warps jump past the run (the host stores the run's end);
//   - subtrees of at most 32 leaves run entirely in registers of warp 0: every
//     alpha stage of size 1..16 lives in one register (stage n, element j at
//     lane n + j), stage 32 in a second one (element j at lane j), and the
//     subtree's 32 bit estimates in one warp-uniform word. F and G are two
//     shuffles and one operation, Rate-1 and SPC a ballot (SPC adds a warp min
//     reduction), Combine is arithmetic on the uniform word.
// Memory layout (Sec. III-B): the alpha stage for node size n occupies elements
// [n, 2n) of a per-CTA array, in shared memory for n <= smem_stage_max and in
// per-CTA device scratch above that; beta is one N-bit array in shared memory
// (node (off, n) owns bits [off, off+n), Combine rewrites only the left half).
// The channel LLRs are read in place from device memory with 16-byte vector
// loads, or (stage_channel) copied to shared memory with cp.async.bulk under an
// mbarrier, double buffered so the next frame's copy overlaps this frame.
// float32: F is an exact min with the XOR of the sign bits (beta in {+0,-0},
// Sec. III-B), G adds alpha_v[i] with its sign flipped by beta_l (Listing 3),
// one IEEE add. int8: G is a saturating add then max(-127) (Listing 4).
// Both agree bit for bit with a scalar evaluation in the same order.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <set>
#include <utility>

#include "polar_internal.h"

namespace polar {
namespace {

template <typename T, class Grp>
__device__ __forceinline__ void trace_store(uint32_t kind, uint32_t n, uint32_t trace_off,
                                            const Frame<T> &fr, float *trace_row) {
    if (kind > OP_G0R) return;
    const uint32_t h = n >> 1;
    const T *src = fr.stage(h);
    for (uint32_t i = Grp::rank(); i < h; i += Grp::size())
        trace_row[trace_off + i] = static_cast<float>(src[i]);
}

// ---------------------------------------------------------------- register subtrees

// A subtree of at most 32 leaves decoded by warp 0 in registers. Stage n <= 16
// element j is register A on lane n + j; stage 32 element j is register B on
// lane j; bits[j] of the uniform word `bits` is the estimate of leaf o0 + j.
template <typename T>
struct RegTree {
    using Acc = typename Llr<T>::Acc;
    Acc A, B;
    uint32_t bits, o0, n0;

    __device__ __forceinline__ void enter(const T *src, uint32_t n, uint32_t o, uint32_t lane) {
        n0 = n;
        o0 = o;
        bits = 0;
        if (n == 32) {
            B = static_cast<Acc>(src[lane]);
        } else {
            A = (lane >= n && lane < 2 * n) ? static_cast<Acc>(src[lane - n]) : Acc(0);
        }
    }

    __device__ __forceinline__ void set_field(uint32_t p, uint32_t n, uint32_t v) {
        const uint32_t fm = low_mask(n) << p;
        bits = (bits & ~fm) | ((v << p) & fm);
    }

    // Execute one operation of the subtree.
    __device__ __forceinline__ void exec(uint32_t kind, uint32_t n, uint32_t o, uint32_t lane) {
        const uint32_t p = o - o0;
        const Acc src = n == 32 ? B : A;
        const uint32_t base = n == 32 ? 0u : n;
        switch (kind) {
        case OP_F:
        case OP_G:
        case OP_G0R: {
            const uint32_t h = n >> 1;
            const uint32_t i = lane - h;  // output element of this lane (lanes [h, 2h))
            const Acc x = __shfl_sync(kFull, src, (base + i) & 31u);
            const Acc y = __shfl_sync(kFull, src, (base + i + h) & 31u);
            Acc r;
            if (kind == OP_F) r = op_f(x, y);
            else if (kind == OP_G) r = op_g(x, y, (bits >> ((p + i) & 31u)) & 1u);
            else r = op_add(x, y);
            if (lane >= h && lane < 2 * h) A = r;
            break;
        }
        case OP_C:
        case OP_C0R: {
            const uint32_t h = n >> 1, m = low_mask(h);
            const uint32_t l = (bits >> p) & m, r = (bits >> (p + h)) & m;
            set_field(p, h, kind == OP_C ? (l ^ r) : r);
            break;
        }
        case OP_R0: set_field(p, n, 0u); break;
        case OP_R1: {
            const bool in = lane >= base && lane < base + n;
            const uint32_t bal = __ballot_sync(kFull, in && src < Acc(0));
            set_field(p, n, bal >> base);
            break;
        }
        case OP_REP: {
            Acc t = src;
            for (uint32_t m = n >> 1; m > 0; m >>= 1) {
                const Acc y = __shfl_down_sync(kFull, t, m);
                if (lane >= base && lane < base + m) t = op_add(t, y);
            }
            const Acc s = __shfl_sync(kFull, t, base);
            set_field(p, n, s < Acc(0) ? kFull : 0u);
            break;
        }
        default: {  // SPC
            const bool in = lane >= base && lane < base + n;
            const uint32_t hd = __ballot_sync(kFull, in && src < Acc(0)) >> base;
            const uint32_t mag = in ? mag_bits(src) : kFull;
            const uint32_t mn = __reduce_min_sync(kFull, mag);
            const uint32_t first = __ffs(__ballot_sync(kFull, in && mag == mn)) - 1u - base;
            set_field(p, n, hd ^ ((__popc(hd) & 1u) << first));
            break;
        }
        }
    }

    __device__ __forceinline__ void trace(uint32_t n, uint32_t trace_off, uint32_t lane,
                                          float *row) const {
        const uint32_t h = n >> 1;
        if (lane >= h && lane < 2 * h) row[trace_off + lane - h] = static_cast<float>(A);
    }
};

// The operation list as one warp sees it: a 32-op window in registers (op
// base + l on lane l) and the following window already requested, so an op is
// one shuffle away and device-memory latency is hidden 32 ops ahead. Indices
// passed to get() never decrease.
struct OpWindow {
    const uint32_t *ops;
    uint32_t n, base, cur, nxt, lane;

    __device__ __forceinline__ uint32_t fetch(uint32_t i) const {
        return i < n ? __ldg(ops + i) : 0u;
    }
    __device__ __forceinline__ void start(const uint32_t *p, uint32_t count, uint32_t l) {
        ops = p;
        n = count;
        lane = l;
        base = 0;
        cur = fetch(l);
        nxt = fetch(32 + l);
    }
    __device__ __forceinline__ void advance() {
        base += 32;
        cur = nxt;
        nxt = fetch(base + 32 + lane);
    }
    __device__ __forceinline__ uint32_t get(uint32_t j) {
        while (j - base >= 32) advance();
        return __shfl_sync(kFull, cur, j - base);
    }
    // First index >= i whose node is wider than 2^log2W (n if none).
    __device__ __forceinline__ uint32_t skip_narrow(uint32_t i, uint32_t log2W) {
        for (;;) {
            while (i - base >= 32) advance();
            const bool stop = lane >= i - base && base + lane < n && op_log2n(cur) > log2W;
            const uint32_t b = __ballot_sync(kFull, stop);
            if (b) return base + __ffs(b) - 1;
            if (base + 32 >= n) return n;
            i = base + 32;
        }
    }
};

// ---------------------------------------------------------------- interpreter body

// Runs the operation list of one frame: narrow runs on warp 0 (register
// subtrees or memory ops), wide ops on the whole CTA.
template <typename T, bool TRACE>
struct InterpBody {
    const KernelArgs &a;
    __device__ __forceinline__ void operator()(const Frame<T> &fr, float *trace_row) const {
        const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
        OpWindow win;
        win.start(a.ops, a.n_ops, lane);
        uint32_t i = 0;
        while (i < a.n_ops) {
            uint32_t w = win.get(i);
            if (op_log2n(w) <= a.log2W) {
                // a run of narrow ops: warp 0 executes it, the other warps skip it
                if (warp == 0) {
                    RegTree<T> rt;
                    uint32_t j = i;
                    for (;;) {
                        const uint32_t kind = op_kind(w), n = 1u << op_log2n(w), o = op_off(w);
                        const uint32_t jn = j + 1;
                        const uint32_t wn = jn < a.n_ops ? win.get(jn) : 0u;
                        if (w & OPW_REG) {
                            if (w & OPW_REG_ENTER) rt.enter(fr.stage_in(n), n, o, lane);
                            rt.exec(kind, n, o, lane);
                            if (TRACE && kind <= OP_G0R)
                                rt.trace(n, __ldg(a.trace_offs + j), lane, trace_row);
                            if (w & OPW_REG_EXIT) {
                                if (lane == 0) write_field(fr.beta, rt.o0, rt.n0, rt.bits);
                                __syncwarp();
                            }
                        } else {
                            exec_op<T, WarpGrp>(kind, n, o, fr);
                            __syncwarp();
                            if (TRACE) {
                                trace_store<T, WarpGrp>(kind, n, __ldg(a.trace_offs + j), fr, trace_row);
                                __syncwarp();
                            }
                        }
                        j = jn;
                        if (j >= a.n_ops || op_log2n(wn) > a.log2W) break;
                        w = wn;
                    }
                    i = j;
                } else {
                    i = win.skip_narrow(i, a.log2W);
                }
                __syncthreads();
            } else {
                const uint32_t kind = op_kind(w), n = 1u << op_log2n(w);
                exec_op<T, CtaGrp>(kind, n, op_off(w), fr);
                __syncthreads();
                if (TRACE) trace_store<T, CtaGrp>(kind, n, __ldg(a.trace_offs + i), fr, trace_row);
                ++i;
            }
        }
    }
};

template <typename T, bool TRACE, bool STAGE>
__global__ void __launch_bounds__(1024) fastssc_decode_kernel(const KernelArgs a) {
    run_frames<T, TRACE, STAGE>(a, InterpBody<T, TRACE>{a});
}

template <typename T, bool TRACE, bool STAGE>
const void *kernel_ptr() {
    return reinterpret_cast<const void *>(&fastssc_decode_kernel<T, TRACE, STAGE>);
}

const void *select_kernel(bool is_i8, bool trace, bool stage) {
    if (is_i8) {
        if (trace) return stage ? kernel_ptr<int8_t, true, true>() : kernel_ptr<int8_t, true, false>();
        return stage ? kernel_ptr<int8_t, false, true>() : kernel_ptr<int8_t, false, false>();
    }
    if (trace) return stage ? kernel_ptr<float, true, true>() : kernel_ptr<float, true, false>();
    return stage ? kernel_ptr<float, false, true>() : kernel_ptr<float, false, false>();
}


}  // namespace

// Raise a kernel variant's dynamic shared-memory limit to the device's opt-in
// maximum, once per (variant, device). It is never lowered afterwards, so any
// shape the host selects can launch.
cudaError_t ensure_smem_limit(const void *k) {
    static std::mutex mu;
    static std::set<std::pair<const void *, int>> done;
    int device = 0;
    cudaError_t e = cudaGetDevice(&device);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> g(mu);
    if (done.count({k, device})) return cudaSuccess;
    int optin = 0;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    if (e == cudaSuccess) done.insert({k, device});
    return e;
}


// Fixed device scratch for polar_decode_noalloc: the alpha stages above the
// shared-memory cap of every resident CTA live here instead of in memory taken
// with cudaMallocAsync. Every GPU that loads this library holds the array until
// the process exits; all calls on a device share it.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

cudaError_t noalloc_scratch(void **ptr) {
    static std::mutex mu;
    static void *addr[kMaxDevices] = {};
    int device = 0;
    cudaError_t e = cudaGetDevice(&device);
    if (e != cudaSuccess) return e;
    if (device < 0 || static_cast<size_t>(device) >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> g(mu);
    if (!addr[device]) {
        // Host code only knows a stand-in for the array; its device address is
        // looked up once per device, with that device current.
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        addr[device] = p;
    }
    *ptr = addr[device];
    return cudaSuccess;
}

size_t kernel_smem_bytes(uint32_t N, uint32_t S, uint32_t threads, bool is_i8, bool stage) {
    (void)threads;
    return SmemLayout(N, S, is_i8 ? 1u : 4u, stage).total;
}

int kernel_max_ctas_per_sm(bool is_i8, bool stage, uint32_t threads, size_t smem_bytes) {
    const void *k = select_kernel(is_i8, false, stage);
    if (ensure_smem_limit(k) != cudaSuccess) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, static_cast<int>(threads),
                                                      smem_bytes) != cudaSuccess)
        return 0;
    return n;
}

// Self-test of the bounded wait: an mbarrier that expects one arrival which
// never comes; the wait gives up after limit_ns, exactly as the channel-staging
// wait does, and reports through the status word. No copy is in flight, so the
// CTA can leave at once.
__global__ void bounded_wait_selftest_kernel(int *status, unsigned long long limit_ns) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        if (!mbar_wait(&bar, 0u, limit_ns)) atomicOr(status, 1);
    }
}

cudaError_t launch_bounded_wait_selftest(int *status, unsigned long long limit_ns,
                                         cudaStream_t stream) {
    bounded_wait_selftest_kernel<<<1, 32, 0, stream>>>(status, limit_ns);
    return cudaGetLastError();
}

cudaError_t launch_decode(bool is_i8, bool trace, bool stage, const LaunchShape &shape,
                          const KernelArgs &args, cudaStream_t stream) {
    const void *k = select_kernel(is_i8, trace, stage);
    cudaError_t e = ensure_smem_limit(k);
    if (e != cudaSuccess) return e;
    void *params[] = {const_cast<KernelArgs *>(&args)};
    return cudaLaunchKernel(k, dim3(shape.grid), dim3(shape.threads), params, shape.smem_bytes,
                            stream);
}

}  // namespace polar
