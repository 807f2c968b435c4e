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

constexpr unsigned long long kWaitNs = 2000000000ull;  // bounded mbarrier wait: 2 s
constexpr uint32_t kWaitPolls = 1u << 28;              // and at most this many polls
constexpr uint32_t kFull = 0xffffffffu;

__host__ __device__ constexpr size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Shared-memory carve-up, computed identically on host and device.
struct SmemLayout {
    size_t alpha, beta, rkey, rpar, chan0, chan1, mbar, total;
    __host__ __device__ SmemLayout(uint32_t N, uint32_t S, uint32_t es, bool stage) {
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
__device__ __forceinline__ int sat127(int v) { return max(-127, min(127, v)); }
__device__ __forceinline__ int f_i8s(int a, int b) {
    const int m = min(abs(a), abs(b));
    return (a ^ b) < 0 ? -m : m;
}
__device__ __forceinline__ int g_i8s(int a, int b, uint32_t bit) {
    return sat127(bit ? b - a : b + a);
}

// Element op on the accumulator type (float, or int holding an int8 value).
__device__ __forceinline__ float op_f(float a, float b) { return f_f32(a, b); }
__device__ __forceinline__ int op_f(int a, int b) { return f_i8s(a, b); }
__device__ __forceinline__ float op_g(float a, float b, uint32_t bit) { return g_f32(a, b, bit); }
__device__ __forceinline__ int op_g(int a, int b, uint32_t bit) { return g_i8s(a, b, bit); }
__device__ __forceinline__ float op_add(float a, float b) { return a + b; }
__device__ __forceinline__ int op_add(int a, int b) { return sat127(a + b); }
__device__ __forceinline__ uint32_t mag_bits(float a) { return __float_as_uint(fabsf(a)); }
__device__ __forceinline__ uint32_t mag_bits(int a) { return static_cast<uint32_t>(abs(a)); }

// Four int8 lanes per 32-bit word.
__device__ __forceinline__ uint32_t bytes_from_bits4(uint32_t bits4) {
    return ((bits4 * 0x00204081u) & 0x01010101u) * 0xFFu;  // bit k -> byte k = 0xFF
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

__device__ __forceinline__ unsigned long long spc_key(float a, uint32_t idx) {
    return (static_cast<unsigned long long>(__float_as_uint(fabsf(a))) << 32) | idx;
}
__device__ __forceinline__ unsigned long long spc_key(int8_t a, uint32_t idx) {
    return (static_cast<unsigned long long>(abs(static_cast<int>(a))) << 32) | idx;
}

template <typename T> struct Llr;
template <> struct Llr<float> {
    static constexpr uint32_t V = 4;  // elements per 16-byte vector
    using Acc = float;
    using Vec = float4;
};
template <> struct Llr<int8_t> {
    static constexpr uint32_t V = 16;
    using Acc = int;
    using Vec = uint4;
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

__device__ __forceinline__ uint32_t low_mask(uint32_t n) { return n >= 32 ? kFull : ((1u << n) - 1u); }

// Replace bits [off, off+n) (n <= 32, inside one word) with the low n bits of v.
__device__ __forceinline__ void write_field(uint32_t *beta, uint32_t off, uint32_t n, uint32_t v) {
    if (n >= 32) {
        beta[off >> 5] = v;
        return;
    }
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

// ---------------------------------------------------------------- F / G / G_0R in memory

template <uint32_t KIND>
__device__ __forceinline__ float4 fg4(float4 a, float4 b, uint32_t bits) {
    float4 r;
    if (KIND == OP_F) {
        r.x = f_f32(a.x, b.x); r.y = f_f32(a.y, b.y); r.z = f_f32(a.z, b.z); r.w = f_f32(a.w, b.w);
    } else if (KIND == OP_G) {
        r.x = g_f32(a.x, b.x, bits & 1u);
        r.y = g_f32(a.y, b.y, (bits >> 1) & 1u);
        r.z = g_f32(a.z, b.z, (bits >> 2) & 1u);
        r.w = g_f32(a.w, b.w, (bits >> 3) & 1u);
    } else {
        r.x = b.x + a.x; r.y = b.y + a.y; r.z = b.z + a.z; r.w = b.w + a.w;
    }
    return r;
}
template <uint32_t KIND>
__device__ __forceinline__ uint4 fg4(uint4 a, uint4 b, uint32_t bits) {
    uint4 r;
    if (KIND == OP_F) {
        r.x = f_i8x4(a.x, b.x); r.y = f_i8x4(a.y, b.y); r.z = f_i8x4(a.z, b.z); r.w = f_i8x4(a.w, b.w);
    } else if (KIND == OP_G) {
        r.x = g_i8x4(a.x, b.x, bits & 0xFu);
        r.y = g_i8x4(a.y, b.y, (bits >> 4) & 0xFu);
        r.z = g_i8x4(a.z, b.z, (bits >> 8) & 0xFu);
        r.w = g_i8x4(a.w, b.w, (bits >> 12) & 0xFu);
    } else {
        r.x = g0r_i8x4(a.x, b.x); r.y = g0r_i8x4(a.y, b.y); r.z = g0r_i8x4(a.z, b.z); r.w = g0r_i8x4(a.w, b.w);
    }
    return r;
}

template <uint32_t KIND, typename T>
__device__ __forceinline__ T fg_scalar(T a, T b, uint32_t bit) {
    using Acc = typename Llr<T>::Acc;
    const Acc x = a, y = b;
    return static_cast<T>(KIND == OP_F ? op_f(x, y) : (KIND == OP_G ? op_g(x, y, bit) : op_add(x, y)));
}

// out[i] = op(in[i], in[i + h]) for i < h; in and out never overlap. Four vectors
// per thread are loaded before any is used, so device-memory operands (the
// channel at the root, scratch stages) overlap their latency.
template <typename T, class Grp, uint32_t KIND>
__device__ __forceinline__ void op_fg(const T *__restrict__ in, T *__restrict__ out, uint32_t h,
                                      const uint32_t *beta, uint32_t o) {
    using Vec = typename Llr<T>::Vec;
    constexpr uint32_t V = Llr<T>::V;
    if (h >= V) {
        const uint32_t nv = h / V, G = Grp::size();
        const Vec *va = reinterpret_cast<const Vec *>(in);
        const Vec *vb = reinterpret_cast<const Vec *>(in + h);
        Vec *vo = reinterpret_cast<Vec *>(out);
        uint32_t v = Grp::rank();
        for (; v + 3 * G < nv; v += 4 * G) {
            Vec a[4], b[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                a[k] = va[v + k * G];
                b[k] = vb[v + k * G];
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint32_t bits = KIND == OP_G ? bits_at(beta, o + (v + k * G) * V, V) : 0u;
                vo[v + k * G] = fg4<KIND>(a[k], b[k], bits);
            }
        }
        for (; v < nv; v += G) {
            const uint32_t bits = KIND == OP_G ? bits_at(beta, o + v * V, V) : 0u;
            vo[v] = fg4<KIND>(va[v], vb[v], bits);
        }
    } else {
        for (uint32_t i = Grp::rank(); i < h; i += Grp::size()) {
            const uint32_t bit = KIND == OP_G ? bits_at(beta, o + i, 1) : 0u;
            out[i] = fg_scalar<KIND, T>(in[i], in[i + h], bit);
        }
    }
}

// ---------------------------------------------------------------- Combine / Rate-0 in memory

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
        beta[o >> 5] = (w & ~(fm << p)) | (l << p);
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

// ---------------------------------------------------------------- node decoders in memory

// Rate-1 (Eq. 4): one ballot per 32 consecutive elements; four chunks loaded ahead.
template <typename T, class Grp>
__device__ __forceinline__ void op_r1(const T *__restrict__ in, uint32_t *beta, uint32_t n,
                                      uint32_t o) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t w0 = Grp::kCta ? (threadIdx.x >> 5) : 0u;
    const uint32_t ws = Grp::kCta ? (blockDim.x >> 5) : 1u;
    const uint32_t nch = (n + 31u) >> 5;
    uint32_t c = w0;
    for (; c + 3 * ws < nch; c += 4 * ws) {
        T a[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) a[k] = in[((c + k * ws) << 5) + lane];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint32_t bal = __ballot_sync(kFull, is_neg(a[k]));
            if (lane == 0) beta[(o >> 5) + c + k * ws] = bal;
        }
    }
    for (; c < nch; c += ws) {
        const uint32_t idx = (c << 5) + lane;
        const bool neg = idx < n && is_neg(in[idx]);
        const uint32_t bal = __ballot_sync(kFull, neg);
        if (lane == 0) write_field(beta, o + (c << 5), n < 32 ? n : 32, bal);
    }
}

// SPC: hard decisions, their parity, flip the least-|alpha| (lowest index)
// decision when the parity is odd.
template <typename T, class Grp>
__device__ __forceinline__ void op_spc(const T *__restrict__ in, uint32_t *beta, uint32_t n,
                                       uint32_t o, unsigned long long *rkey, uint32_t *rpar) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t w0 = Grp::kCta ? (threadIdx.x >> 5) : 0u;
    const uint32_t ws = Grp::kCta ? (blockDim.x >> 5) : 1u;
    const uint32_t nch = (n + 31u) >> 5;
    unsigned long long kmin = ~0ull;
    uint32_t par = 0;
    uint32_t c = w0;
    for (; c + 3 * ws < nch; c += 4 * ws) {
        T a[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) a[k] = in[((c + k * ws) << 5) + lane];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint32_t bal = __ballot_sync(kFull, is_neg(a[k]));
            par ^= __popc(bal) & 1u;
            if (lane == 0) beta[(o >> 5) + c + k * ws] = bal;
            const unsigned long long key = spc_key(a[k], ((c + k * ws) << 5) + lane);
            kmin = key < kmin ? key : kmin;
        }
    }
    for (; c < nch; c += ws) {
        const uint32_t idx = (c << 5) + lane;
        const bool valid = idx < n;
        const T a = valid ? in[idx] : T(0);
        const uint32_t bal = __ballot_sync(kFull, valid && is_neg(a));
        par ^= __popc(bal) & 1u;
        if (lane == 0) write_field(beta, o + (c << 5), n < 32 ? n : 32, bal);
        if (valid) {
            const unsigned long long key = spc_key(a, idx);
            kmin = key < kmin ? key : kmin;
        }
    }
#pragma unroll
    for (uint32_t s = 16; s > 0; s >>= 1) {
        const unsigned long long t = __shfl_xor_sync(kFull, kmin, s);
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

// Repetition: the sum of alpha_v folded as t[i] <- t[i] + t[i + m],
// m = n/2, n/4, ..., 1 (the G_0R chain SC computes on this node); the bit is
// (sum < 0), replicated. Folds above 64 values run in memory (tmp = the free
// stage n/2), the last ones as warp shuffles with the same pairing.
template <typename T, class Grp>
__device__ __forceinline__ void op_rep(const T *in, T *tmp, uint32_t *beta, uint32_t n,
                                       uint32_t o) {
    using Acc = typename Llr<T>::Acc;
    uint32_t len = n;
    const T *src = in;
    while (len > 64) {
        const uint32_t m = len >> 1;
        if (src == tmp) {
            for (uint32_t i = Grp::rank(); i < m; i += Grp::size())
                tmp[i] = fg_scalar<OP_G0R, T>(tmp[i], tmp[i + m], 0u);
        } else {
            op_fg<T, Grp, OP_G0R>(src, tmp, m, nullptr, 0);
        }
        Grp::sync();
        src = tmp;
        len = m;
    }
    if (threadIdx.x < 32) {
        const uint32_t lane = threadIdx.x;
        Acc x;
        uint32_t cur;
        if (len == 64) {
            x = op_add(static_cast<Acc>(src[lane]), static_cast<Acc>(src[lane + 32]));
            cur = 32;
        } else {
            x = lane < len ? static_cast<Acc>(src[lane]) : Acc(0);
            cur = len;
        }
        while (cur > 1) {
            cur >>= 1;
            const Acc y = __shfl_down_sync(kFull, x, cur);
            if (lane < cur) x = op_add(x, y);
        }
        const Acc s = __shfl_sync(kFull, x, 0);
        const uint32_t word = s < Acc(0) ? kFull : 0u;
        if (n >= 32) {
            for (uint32_t j = lane; j < (n >> 5); j += 32) beta[(o >> 5) + j] = word;
        } else if (lane == 0) {
            write_field(beta, o, n, word);
        }
    }
}

// ---------------------------------------------------------------- frame state

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
__device__ __forceinline__ void exec_op(uint32_t kind, uint32_t n, uint32_t o, const Frame<T> &fr) {
    switch (kind) {
    case OP_F: op_fg<T, Grp, OP_F>(fr.stage_in(n), fr.stage(n >> 1), n >> 1, fr.beta, o); break;
    case OP_G: op_fg<T, Grp, OP_G>(fr.stage_in(n), fr.stage(n >> 1), n >> 1, fr.beta, o); break;
    case OP_G0R: op_fg<T, Grp, OP_G0R>(fr.stage_in(n), fr.stage(n >> 1), n >> 1, fr.beta, o); break;
    case OP_C: op_combine<Grp>(fr.beta, n, o, false); break;
    case OP_C0R: op_combine<Grp>(fr.beta, n, o, true); break;
    case OP_R0: op_r0<Grp>(fr.beta, n, o); break;
    case OP_R1: op_r1<T, Grp>(fr.stage_in(n), fr.beta, n, o); break;
    case OP_REP: op_rep<T, Grp>(fr.stage_in(n), fr.stage(n >> 1), fr.beta, n, o); break;
    default: op_spc<T, Grp>(fr.stage_in(n), fr.beta, n, o, fr.rkey, fr.rpar); break;
    }
}

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

// Software bit extract: the bits of x selected by m, packed to the bottom.
__device__ __forceinline__ uint32_t pext32(uint32_t x, uint32_t m) {
    if (m == kFull) return x;
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
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
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
    const SmemLayout L(a.N, a.S, sizeof(T), STAGE);
    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31u;

    Frame<T> fr;
    fr.s_alpha = reinterpret_cast<T *>(smem + L.alpha);
    fr.g_alpha = a.gscratch ? static_cast<T *>(a.gscratch) + size_t(blockIdx.x) * a.gstride
                            : nullptr;
    fr.beta = reinterpret_cast<uint32_t *>(smem + L.beta);
    fr.rkey = reinterpret_cast<unsigned long long *>(smem + L.rkey);
    fr.rpar = reinterpret_cast<uint32_t *>(smem + L.rpar);
    fr.N = a.N;
    fr.S = a.S;

    T *const chan0 = reinterpret_cast<T *>(smem + L.chan0);
    T *const chan1 = reinterpret_cast<T *>(smem + L.chan1);
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + L.mbar);
    const uint32_t chan_bytes = a.N * static_cast<uint32_t>(sizeof(T));
    const T *llr = static_cast<const T *>(a.llr);
    const size_t G = gridDim.x;

    if (STAGE) {
        if (tid == 0) {
            mbar_init(&mbar[0]);
            mbar_init(&mbar[1]);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            if (blockIdx.x < a.n_frames)
                bulk_load(chan0, llr + size_t(blockIdx.x) * a.N, chan_bytes, &mbar[0]);
            if (blockIdx.x + G < a.n_frames)
                bulk_load(chan1, llr + (blockIdx.x + G) * a.N, chan_bytes, &mbar[1]);
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
            fr.chan = b ? chan1 : chan0;
        } else {
            fr.chan = llr + f * a.N;
        }
        float *trace_row = TRACE ? a.trace + f * a.trace_stride : nullptr;

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
            bulk_load((it & 1u) ? chan1 : chan0, llr + (f + 2 * G) * a.N, chan_bytes,
                      &mbar[it & 1u]);
        }
    }
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

}  // namespace

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
