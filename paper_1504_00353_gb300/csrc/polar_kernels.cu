// Fast-SSC decoding kernels for sm_103a (GB300).
//
// Method: Giard et al., "Low-Latency Software Polar Decoders" (arXiv 1504.00353),
// Sec. II-C/II-D. One CTA decodes one frame at a time and loops over frames
// (persistent grid sized to the resident-CTA count). The frame's operation list
// (the depth-first Fast-SSC call list of Listing 1, built on the host) is
// interpreted in order:
//   - wide operations (node size N_v > warp_stage_max) use every thread of the
//     CTA, with one __syncthreads after each;
//   - runs of narrow operations (N_v <= warp_stage_max) are executed by warp 0
//     alone with __syncwarp between them, the other warps jump past the run
//     (the host stores the run's end in each operation);
//   - alpha (LLR) stages follow the paper's single-buffer-per-stage layout
//     (Sec. III-B "Improved Layout of the alpha-memory"): the stage for node
//     size n occupies elements [n, 2n) of a per-CTA array, in shared memory for
//     n <= smem_stage_max and in per-CTA device scratch above that;
//   - beta is one N-bit array (Sec. III-B "Eliminating Superfluous Operations on
//     beta-Values"): node (off, n) owns bits [off, off+n), Combine rewrites only
//     the left half; bits are packed 32 per word in shared memory;
//   - the channel LLRs are read in place from device memory with 16-byte
//     vector loads, or (stage_channel) copied to shared memory with
//     cp.async.bulk under an mbarrier, double buffered so the next frame's copy
//     overlaps this frame's decode.
// float32: F is an exact min with the XOR of the sign bits (Sec. III-B, beta in
// {+0,-0}), G adds alpha_v[i] with its sign bit flipped by beta_l (Listing 3),
// one IEEE add. int8: packed byte SIMD, G is a saturating byte add followed by
// max(-127) (Listing 4). Both match a scalar evaluation bit for bit.
#include <cuda_runtime.h>

#include <cstdint>

#include "polar_internal.h"

namespace polar {
namespace {

constexpr unsigned long long kWaitNs = 2000000000ull;  // bounded mbarrier wait: 2 s
constexpr uint32_t kWaitPolls = 1u << 28;              // and at most this many polls

__host__ __device__ constexpr size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Shared-memory carve-up, computed identically on host and device.
struct SmemLayout {
    size_t alpha, beta, rkey, rpar, chan0, chan1, mbar, total;
    __host__ __device__ SmemLayout(uint32_t N, uint32_t S, uint32_t threads, uint32_t es,
                                   bool stage) {
        const uint32_t Se = S < N / 2 ? S : N / 2;
        const uint32_t NW = N >= 32 ? N / 32 : 1;
        size_t o = 0;
        alpha = o;
        o = align_up(o + size_t(2) * Se * es, 128);
        beta = o;
        o = align_up(o + size_t(NW) * 4, 16);
        rkey = o;
        o += 32 * 8;
        rpar = o;
        o = align_up(o + 32 * 4, 128);
        chan0 = chan1 = o;
        if (stage) {
            chan0 = o;
            o = align_up(o + size_t(N) * es, 128);
            chan1 = o;
            o = align_up(o + size_t(N) * es, 128);
        }
        mbar = o;
        o += 16;
        total = align_up(o, 16);
        (void)threads;
    }
};

// ---------------------------------------------------------------- element ops

__device__ __forceinline__ float f_f32(float a, float b) {
    const float m = fminf(fabsf(a), fabsf(b));
    return __uint_as_float(__float_as_uint(m) |
                           ((__float_as_uint(a) ^ __float_as_uint(b)) & 0x80000000u));
}
// Eq. 2 with beta_l as the sign bit of alpha_v[i] (Listing 3): one IEEE add.
__device__ __forceinline__ float g_f32(float a, float b, uint32_t bit) {
    return b + __uint_as_float(__float_as_uint(a) ^ (bit << 31));
}

__device__ __forceinline__ int f_i8s(int a, int b) {
    const int m = min(abs(a), abs(b));
    return (a ^ b) < 0 ? -m : m;
}
__device__ __forceinline__ int sat127(int v) { return max(-127, min(127, v)); }
__device__ __forceinline__ int g_i8s(int a, int b, uint32_t bit) {
    return sat127(bit ? b - a : b + a);
}

// Four int8 lanes per 32-bit word.
__device__ __forceinline__ uint32_t bytes_from_bits4(uint32_t bits4) {
    // bit k of bits4 -> byte k = 0xFF
    return ((bits4 * 0x00204081u) & 0x01010101u) * 0xFFu;
}
__device__ __forceinline__ uint32_t f_i8x4(uint32_t a, uint32_t b) {
    const uint32_t m = __vminu4(__vabsss4(a), __vabsss4(b));
    const uint32_t sel = (((a ^ b) & 0x80808080u) >> 7) * 0xFFu;
    return (m & ~sel) | (__vneg4(m) & sel);
}
__device__ __forceinline__ uint32_t g_i8x4(uint32_t a, uint32_t b, uint32_t bits4) {
    const uint32_t sel = bytes_from_bits4(bits4);
    const uint32_t an = (a & ~sel) | (__vneg4(a) & sel);
    return __vmaxs4(__vaddss4(b, an), 0x81818181u);
}
__device__ __forceinline__ uint32_t g0r_i8x4(uint32_t a, uint32_t b) {
    return __vmaxs4(__vaddss4(b, a), 0x81818181u);
}

__device__ __forceinline__ bool is_neg(float a) { return a < 0.0f; }
__device__ __forceinline__ bool is_neg(int8_t a) { return a < 0; }

// SPC key: |alpha| in the high word, index in the low word; the minimum key is
// the least magnitude at the lowest index (Listing 2 returns the first lane).
__device__ __forceinline__ unsigned long long spc_key(float a, uint32_t idx) {
    return (static_cast<unsigned long long>(__float_as_uint(fabsf(a))) << 32) | idx;
}
__device__ __forceinline__ unsigned long long spc_key(int8_t a, uint32_t idx) {
    return (static_cast<unsigned long long>(abs(static_cast<int>(a))) << 32) | idx;
}

__device__ __forceinline__ float add_fold(float a, float b) { return a + b; }
__device__ __forceinline__ int add_fold(int a, int b) { return sat127(a + b); }

template <typename T> struct Llr;
template <> struct Llr<float> {
    static constexpr uint32_t V = 4;  // elements per 16-byte vector
    using Acc = float;
};
template <> struct Llr<int8_t> {
    static constexpr uint32_t V = 16;
    using Acc = int;
};

// ---------------------------------------------------------------- groups

struct WarpGrp {
    static constexpr bool kCta = false;
    __device__ static uint32_t rank() { return threadIdx.x & 31u; }
    __device__ static uint32_t size() { return 32u; }
    __device__ static void sync() { __syncwarp(); }
};
struct CtaGrp {
    static constexpr bool kCta = true;
    __device__ static uint32_t rank() { return threadIdx.x; }
    __device__ static uint32_t size() { return blockDim.x; }
    __device__ static void sync() { __syncthreads(); }
};

// ---------------------------------------------------------------- beta helpers

// Replace bits [off, off+n) (n < 32, inside one word) with the low n bits of v.
__device__ __forceinline__ void write_field(uint32_t *beta, uint32_t off, uint32_t n,
                                            uint32_t v) {
    const uint32_t p = off & 31u;
    const uint32_t fm = ((1u << n) - 1u) << p;
    uint32_t w = beta[off >> 5];
    w = (w & ~fm) | ((v << p) & fm);
    beta[off >> 5] = w;
}

__device__ __forceinline__ uint32_t bits_at(const uint32_t *beta, uint32_t pos, uint32_t nbits) {
    const uint32_t w = beta[pos >> 5] >> (pos & 31u);
    return nbits >= 32 ? w : (w & ((1u << nbits) - 1u));
}

// ---------------------------------------------------------------- F / G / G_0R

template <uint32_t KIND>
__device__ __forceinline__ void fg_vec(const float *in, float *out, uint32_t h, uint32_t e,
                                       const uint32_t *beta, uint32_t o) {
    const float4 a = *reinterpret_cast<const float4 *>(in + e);
    const float4 b = *reinterpret_cast<const float4 *>(in + h + e);
    float4 r;
    if (KIND == OP_F) {
        r.x = f_f32(a.x, b.x);
        r.y = f_f32(a.y, b.y);
        r.z = f_f32(a.z, b.z);
        r.w = f_f32(a.w, b.w);
    } else if (KIND == OP_G) {
        const uint32_t bits = bits_at(beta, o + e, 4);
        r.x = g_f32(a.x, b.x, bits & 1u);
        r.y = g_f32(a.y, b.y, (bits >> 1) & 1u);
        r.z = g_f32(a.z, b.z, (bits >> 2) & 1u);
        r.w = g_f32(a.w, b.w, (bits >> 3) & 1u);
    } else {
        r.x = b.x + a.x;
        r.y = b.y + a.y;
        r.z = b.z + a.z;
        r.w = b.w + a.w;
    }
    *reinterpret_cast<float4 *>(out + e) = r;
}

template <uint32_t KIND>
__device__ __forceinline__ void fg_vec(const int8_t *in, int8_t *out, uint32_t h, uint32_t e,
                                       const uint32_t *beta, uint32_t o) {
    const uint4 a = *reinterpret_cast<const uint4 *>(in + e);
    const uint4 b = *reinterpret_cast<const uint4 *>(in + h + e);
    uint4 r;
    if (KIND == OP_F) {
        r.x = f_i8x4(a.x, b.x);
        r.y = f_i8x4(a.y, b.y);
        r.z = f_i8x4(a.z, b.z);
        r.w = f_i8x4(a.w, b.w);
    } else if (KIND == OP_G) {
        const uint32_t bits = bits_at(beta, o + e, 16);
        r.x = g_i8x4(a.x, b.x, bits & 0xFu);
        r.y = g_i8x4(a.y, b.y, (bits >> 4) & 0xFu);
        r.z = g_i8x4(a.z, b.z, (bits >> 8) & 0xFu);
        r.w = g_i8x4(a.w, b.w, (bits >> 12) & 0xFu);
    } else {
        r.x = g0r_i8x4(a.x, b.x);
        r.y = g0r_i8x4(a.y, b.y);
        r.z = g0r_i8x4(a.z, b.z);
        r.w = g0r_i8x4(a.w, b.w);
    }
    *reinterpret_cast<uint4 *>(out + e) = r;
}

template <uint32_t KIND>
__device__ __forceinline__ float fg_scalar(float a, float b, uint32_t bit) {
    return KIND == OP_F ? f_f32(a, b) : (KIND == OP_G ? g_f32(a, b, bit) : b + a);
}
template <uint32_t KIND>
__device__ __forceinline__ int8_t fg_scalar(int8_t a, int8_t b, uint32_t bit) {
    return static_cast<int8_t>(KIND == OP_F ? f_i8s(a, b)
                                            : (KIND == OP_G ? g_i8s(a, b, bit) : sat127(b + a)));
}

// out[i] = op(in[i], in[i + h]) for i < h (in = alpha_v of a node of size 2h).
template <typename T, class Grp, uint32_t KIND>
__device__ __forceinline__ void op_fg(const T *in, T *out, uint32_t h, const uint32_t *beta,
                                      uint32_t o) {
    constexpr uint32_t V = Llr<T>::V;
    if (h >= V) {
        for (uint32_t e = Grp::rank() * V; e < h; e += Grp::size() * V)
            fg_vec<KIND>(in, out, h, e, beta, o);
    } else {
        for (uint32_t i = Grp::rank(); i < h; i += Grp::size()) {
            const uint32_t bit = KIND == OP_G ? bits_at(beta, o + i, 1) : 0u;
            out[i] = fg_scalar<KIND>(in[i], in[i + h], bit);
        }
    }
}

// ---------------------------------------------------------------- Combine / Rate-0

template <class Grp>
__device__ __forceinline__ void op_combine(uint32_t *beta, uint32_t n, uint32_t o, bool copy) {
    const uint32_t h = n >> 1;
    if (h >= 32) {
        const uint32_t wl = o >> 5, wr = (o + h) >> 5, nw = h >> 5;
        for (uint32_t j = Grp::rank(); j < nw; j += Grp::size()) {
            const uint32_t r = beta[wr + j];
            beta[wl + j] = copy ? r : (beta[wl + j] ^ r);
        }
    } else if (Grp::rank() == 0) {
        const uint32_t p = o & 31u, fm = (1u << h) - 1u;
        uint32_t w = beta[o >> 5];
        const uint32_t r = (w >> (p + h)) & fm;
        const uint32_t l = copy ? r : (((w >> p) & fm) ^ r);
        w = (w & ~(fm << p)) | (l << p);
        beta[o >> 5] = w;
    }
}

template <class Grp>
__device__ __forceinline__ void op_r0(uint32_t *beta, uint32_t n, uint32_t o) {
    if (n >= 32) {
        for (uint32_t j = Grp::rank(); j < (n >> 5); j += Grp::size()) beta[(o >> 5) + j] = 0u;
    } else if (Grp::rank() == 0) {
        write_field(beta, o, n, 0u);
    }
}

// ---------------------------------------------------------------- node decoders

// Rate-1 (Eq. 4): one ballot per 32 consecutive elements.
template <typename T, class Grp>
__device__ __forceinline__ void op_r1(const T *in, uint32_t *beta, uint32_t n, uint32_t o) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t w0 = Grp::kCta ? (threadIdx.x >> 5) : 0u;
    const uint32_t ws = Grp::kCta ? (blockDim.x >> 5) : 1u;
    const uint32_t nch = (n + 31u) >> 5;
    for (uint32_t c = w0; c < nch; c += ws) {
        const uint32_t idx = (c << 5) + lane;
        const bool neg = idx < n && is_neg(in[idx]);
        const uint32_t bal = __ballot_sync(0xffffffffu, neg);
        if (lane == 0) {
            if (n >= 32) beta[(o >> 5) + c] = bal;
            else write_field(beta, o, n, bal);
        }
    }
}

// SPC: hard decisions, parity of them, flip the least-|alpha| (lowest index)
// decision when the parity is odd.
template <typename T, class Grp>
__device__ __forceinline__ void op_spc(const T *in, uint32_t *beta, uint32_t n, uint32_t o,
                                       unsigned long long *rkey, uint32_t *rpar) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t w0 = Grp::kCta ? (threadIdx.x >> 5) : 0u;
    const uint32_t ws = Grp::kCta ? (blockDim.x >> 5) : 1u;
    const uint32_t nch = (n + 31u) >> 5;
    unsigned long long kmin = ~0ull;
    uint32_t par = 0;
    for (uint32_t c = w0; c < nch; c += ws) {
        const uint32_t idx = (c << 5) + lane;
        const bool valid = idx < n;
        const T a = valid ? in[idx] : T(0);
        const uint32_t bal = __ballot_sync(0xffffffffu, valid && is_neg(a));
        par ^= __popc(bal) & 1u;
        if (lane == 0) {
            if (n >= 32) beta[(o >> 5) + c] = bal;
            else write_field(beta, o, n, bal);
        }
        if (valid) {
            const unsigned long long k = spc_key(a, idx);
            kmin = k < kmin ? k : kmin;
        }
    }
#pragma unroll
    for (uint32_t s = 16; s > 0; s >>= 1) {
        const unsigned long long t = __shfl_xor_sync(0xffffffffu, kmin, s);
        kmin = t < kmin ? t : kmin;
    }
    if (Grp::kCta) {
        const uint32_t w = threadIdx.x >> 5;
        if (lane == 0) {
            rkey[w] = kmin;
            rpar[w] = par;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t p = 0;
            for (uint32_t i = 0; i < ws; ++i) {
                kmin = rkey[i] < kmin ? rkey[i] : kmin;
                p ^= rpar[i];
            }
            if (p) {
                const uint32_t pos = o + static_cast<uint32_t>(kmin & 0xffffffffull);
                beta[pos >> 5] ^= 1u << (pos & 31u);
            }
        }
    } else if (lane == 0 && par) {
        const uint32_t pos = o + static_cast<uint32_t>(kmin & 0xffffffffull);
        beta[pos >> 5] ^= 1u << (pos & 31u);
    }
}

// tmp[i] = in[i] + in[i + m] for i < m (saturating for int8); tmp may alias in.
template <typename T, class Grp>
__device__ __forceinline__ void fold_level(const T *in, T *tmp, uint32_t m) {
    constexpr uint32_t V = Llr<T>::V;
    if (m >= V) {
        for (uint32_t e = Grp::rank() * V; e < m; e += Grp::size() * V)
            fg_vec<OP_G0R>(in, tmp, m, e, nullptr, 0);
    } else {
        for (uint32_t i = Grp::rank(); i < m; i += Grp::size())
            tmp[i] = fg_scalar<OP_G0R>(in[i], in[i + m], 0u);
    }
}

// Repetition: the sum of alpha_v folded as t[i] <- t[i] + t[i + m],
// m = n/2, n/4, ..., 1 (the G_0R chain SC would compute on this node); the
// bit is (sum < 0), replicated over the node.
template <typename T, class Grp>
__device__ __forceinline__ void op_rep(const T *in, T *tmp, uint32_t *beta, uint32_t n,
                                       uint32_t o) {
    using Acc = typename Llr<T>::Acc;
    uint32_t len = n;
    const T *src = in;
    while (len > 64) {
        const uint32_t m = len >> 1;
        fold_level<T, Grp>(src, tmp, m);
        Grp::sync();
        src = tmp;
        len = m;
    }
    if (threadIdx.x < 32) {
        const uint32_t lane = threadIdx.x;
        Acc x;
        uint32_t cur;
        if (len == 64) {
            x = add_fold(static_cast<Acc>(src[lane]), static_cast<Acc>(src[lane + 32]));
            cur = 32;
        } else {
            x = lane < len ? static_cast<Acc>(src[lane]) : Acc(0);
            cur = len;
        }
        while (cur > 1) {
            cur >>= 1;
            const Acc y = __shfl_down_sync(0xffffffffu, x, cur);
            if (lane < cur) x = add_fold(x, y);
        }
        const Acc s = __shfl_sync(0xffffffffu, x, 0);
        const uint32_t word = s < Acc(0) ? 0xffffffffu : 0u;
        if (n >= 32) {
            for (uint32_t j = lane; j < (n >> 5); j += 32) beta[(o >> 5) + j] = word;
        } else if (lane == 0) {
            write_field(beta, o, n, word);
        }
    }
}

// ---------------------------------------------------------------- dispatch

template <typename T>
struct Frame {
    const T *chan;     // channel LLRs of the frame (shared or device memory)
    T *s_alpha;        // shared alpha array (stage n at [n, 2n), n <= S)
    T *g_alpha;        // device scratch (stage n at [n - 2S, 2n - 2S), n > S)
    uint32_t *beta;    // shared beta bits
    unsigned long long *rkey;
    uint32_t *rpar;
    uint32_t N, S;
    __device__ __forceinline__ const T *stage_in(uint32_t n) const {
        return n == N ? chan : (n <= S ? s_alpha + n : g_alpha + (n - 2 * S));
    }
    __device__ __forceinline__ T *stage(uint32_t n) const {
        return n <= S ? s_alpha + n : g_alpha + (n - 2 * S);
    }
};

template <typename T, class Grp>
__device__ __forceinline__ void exec_op(uint32_t meta, uint32_t o, const Frame<T> &fr) {
    const uint32_t kind = meta & 0xffu;
    const uint32_t n = 1u << ((meta >> 8) & 0xffu);
    switch (kind) {
    case OP_F:
        op_fg<T, Grp, OP_F>(fr.stage_in(n), fr.stage(n >> 1), n >> 1, fr.beta, o);
        break;
    case OP_G:
        op_fg<T, Grp, OP_G>(fr.stage_in(n), fr.stage(n >> 1), n >> 1, fr.beta, o);
        break;
    case OP_G0R:
        op_fg<T, Grp, OP_G0R>(fr.stage_in(n), fr.stage(n >> 1), n >> 1, fr.beta, o);
        break;
    case OP_C:
        op_combine<Grp>(fr.beta, n, o, false);
        break;
    case OP_C0R:
        op_combine<Grp>(fr.beta, n, o, true);
        break;
    case OP_R0:
        op_r0<Grp>(fr.beta, n, o);
        break;
    case OP_R1:
        op_r1<T, Grp>(fr.stage_in(n), fr.beta, n, o);
        break;
    case OP_REP:
        op_rep<T, Grp>(fr.stage_in(n), fr.stage(n >> 1), fr.beta, n, o);
        break;
    default:
        op_spc<T, Grp>(fr.stage_in(n), fr.beta, n, o, fr.rkey, fr.rpar);
        break;
    }
}

template <typename T, class Grp>
__device__ __forceinline__ void trace_store(uint32_t meta, const DevOp &op, const Frame<T> &fr,
                                            float *trace_row) {
    const uint32_t kind = meta & 0xffu;
    if (kind > OP_G0R) return;
    const uint32_t h = 1u << (((meta >> 8) & 0xffu) - 1u);
    const T *src = fr.stage(h);
    for (uint32_t i = Grp::rank(); i < h; i += Grp::size())
        trace_row[op.trace_off + i] = static_cast<float>(src[i]);
}

__device__ __forceinline__ DevOp load_op(const DevOp *ops, uint32_t i) {
    const uint4 v = __ldg(reinterpret_cast<const uint4 *>(ops) + i);
    return DevOp{v.x, v.y, v.z, v.w};
}

// Software bit extract: the bits of x selected by m, packed to the bottom.
__device__ __forceinline__ uint32_t pext32(uint32_t x, uint32_t m) {
    if (m == 0xffffffffu) return x;
    uint32_t r = 0, k = 0;
    while (m) {
        const uint32_t b = m & (0u - m);
        r |= ((x & b) ? 1u : 0u) << k;
        ++k;
        m ^= b;
    }
    return r;
}

// ---------------------------------------------------------------- bulk copy

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint64_t *bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes,
                                          uint64_t *bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}
// Bounded wait for the phase with the given parity; false after kWaitNs.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    const unsigned long long t0 = globaltimer();
    for (uint32_t i = 0; i < kWaitPolls; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
        if (ok) return true;
        if ((i & 63u) == 63u && globaltimer() - t0 > kWaitNs) return false;
    }
    return false;
}

// ---------------------------------------------------------------- kernel

template <typename T, bool TRACE, bool STAGE>
__global__ void __launch_bounds__(1024) fastssc_decode_kernel(const KernelArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    const SmemLayout L(a.N, a.S, blockDim.x, sizeof(T), STAGE);
    const uint32_t tid = threadIdx.x, warp = tid >> 5;

    Frame<T> fr;
    fr.s_alpha = reinterpret_cast<T *>(smem + L.alpha);
    fr.g_alpha = a.gscratch ? static_cast<T *>(a.gscratch) + size_t(blockIdx.x) * a.gstride
                            : nullptr;
    fr.beta = reinterpret_cast<uint32_t *>(smem + L.beta);
    fr.rkey = reinterpret_cast<unsigned long long *>(smem + L.rkey);
    fr.rpar = reinterpret_cast<uint32_t *>(smem + L.rpar);
    fr.N = a.N;
    fr.S = a.S;

    T *chanbuf[2] = {reinterpret_cast<T *>(smem + L.chan0), reinterpret_cast<T *>(smem + L.chan1)};
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + L.mbar);
    const uint32_t chan_bytes = a.N * static_cast<uint32_t>(sizeof(T));
    const T *llr = static_cast<const T *>(a.llr);
    const size_t G = gridDim.x;

    if (STAGE) {
        if (tid == 0) {
            mbar_init(&mbar[0]);
            mbar_init(&mbar[1]);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            for (size_t k = 0; k < 2; ++k) {
                const size_t f = blockIdx.x + k * G;
                if (f < a.n_frames) bulk_load(chanbuf[k], llr + f * a.N, chan_bytes, &mbar[k]);
            }
        }
        __syncthreads();
    }

    uint32_t it = 0;
    for (size_t f = blockIdx.x; f < a.n_frames; f += G, ++it) {
        if (STAGE) {
            const uint32_t b = it & 1u;
            const bool bad = !mbar_wait(&mbar[b], (it >> 1) & 1u);
            if (__syncthreads_or(bad)) {
                if (tid == 0) atomicOr(a.status, 1);
                // let any copy still in flight land before the CTA's shared memory is released
                mbar_wait(&mbar[b], (it >> 1) & 1u);
                if (f + G < a.n_frames) mbar_wait(&mbar[b ^ 1u], ((it + 1) >> 1) & 1u);
                return;
            }
            fr.chan = chanbuf[b];
        } else {
            fr.chan = llr + f * a.N;
        }
        float *trace_row = TRACE ? a.trace + f * a.trace_stride : nullptr;

        uint32_t i = 0;
        while (i < a.n_ops) {
            const DevOp op = load_op(a.ops, i);
            if (op.meta & OPF_WARP) {
                if (warp == 0) {
                    DevOp cur = op;
                    for (uint32_t j = i;;) {
                        const bool more = j + 1 < op.next;
                        const DevOp nxt = more ? load_op(a.ops, j + 1) : cur;
                        exec_op<T, WarpGrp>(cur.meta, cur.off, fr);
                        __syncwarp();
                        if (TRACE) {
                            trace_store<T, WarpGrp>(cur.meta, cur, fr, trace_row);
                            __syncwarp();
                        }
                        if (!more) break;
                        ++j;
                        cur = nxt;
                    }
                }
                i = op.next;
                __syncthreads();
            } else {
                exec_op<T, CtaGrp>(op.meta, op.off, fr);
                __syncthreads();
                if (TRACE) trace_store<T, CtaGrp>(op.meta, op, fr, trace_row);
                ++i;
            }
        }

        // Pack x_hat restricted to A, LSB first (output word u = info bits [32u, 32u+32)).
        uint8_t *out = a.out + f * a.out_row;
        for (uint32_t u = tid; u < a.KW; u += blockDim.x) {
            const uint32_t lo = u << 5;
            const uint32_t hi = min(lo + 32u, a.K);
            uint32_t acc = 0;
            for (uint32_t w = __ldg(a.ext_wstart + u); w < a.NW; ++w) {
                const uint32_t pre = __ldg(a.ext_pre + w);
                if (pre >= hi) break;
                const uint32_t m = __ldg(a.ext_mask + w);
                if (!m) continue;
                const uint32_t e = pext32(fr.beta[w], m);
                const int pos = static_cast<int>(pre) - static_cast<int>(lo);
                acc |= pos >= 0 ? (e << pos) : (e >> (-pos));
            }
            if (hi - lo < 32) acc &= (1u << (hi - lo)) - 1u;
            const uint32_t nb = min(4u, a.out_row - 4u * u);
            uint8_t *dst = out + 4u * u;
            if (nb == 4 && (reinterpret_cast<uintptr_t>(dst) & 3u) == 0) {
                *reinterpret_cast<uint32_t *>(dst) = acc;
            } else {
                for (uint32_t b = 0; b < nb; ++b) dst[b] = static_cast<uint8_t>(acc >> (8 * b));
            }
        }
        __syncthreads();

        if (STAGE && tid == 0 && f + 2 * G < a.n_frames) {
            // every thread is done reading this buffer (barrier above); order those
            // generic-proxy reads before the async-proxy write of the next frame
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            bulk_load(chanbuf[it & 1u], llr + (f + 2 * G) * a.N, chan_bytes, &mbar[it & 1u]);
        }
    }
}

template <typename T, bool TRACE, bool STAGE>
void *kernel_ptr() {
    return reinterpret_cast<void *>(&fastssc_decode_kernel<T, TRACE, STAGE>);
}

void *select_kernel(bool is_i8, bool trace, bool stage) {
    if (is_i8) {
        if (trace) return stage ? kernel_ptr<int8_t, true, true>() : kernel_ptr<int8_t, true, false>();
        return stage ? kernel_ptr<int8_t, false, true>() : kernel_ptr<int8_t, false, false>();
    }
    if (trace) return stage ? kernel_ptr<float, true, true>() : kernel_ptr<float, true, false>();
    return stage ? kernel_ptr<float, false, true>() : kernel_ptr<float, false, false>();
}

}  // namespace

size_t kernel_smem_bytes(uint32_t N, uint32_t S, uint32_t threads, bool is_i8, bool stage) {
    return SmemLayout(N, S, threads, is_i8 ? 1u : 4u, stage).total;
}

int kernel_max_ctas_per_sm(bool is_i8, bool stage, uint32_t threads, size_t smem_bytes) {
    void *k = select_kernel(is_i8, false, stage);
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(smem_bytes)) != cudaSuccess)
        return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, static_cast<int>(threads),
                                                      smem_bytes) != cudaSuccess)
        return 0;
    return n;
}

cudaError_t launch_decode(bool is_i8, bool trace, bool stage, const LaunchShape &shape,
                          const KernelArgs &args, cudaStream_t stream) {
    void *k = select_kernel(is_i8, trace, stage);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(shape.smem_bytes));
    if (e != cudaSuccess) return e;
    void *params[] = {const_cast<KernelArgs *>(&args)};
    return cudaLaunchKernel(k, dim3(shape.grid), dim3(shape.threads), params, shape.smem_bytes,
                            stream);
}

}  // namespace polar
