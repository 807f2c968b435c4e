// Device building blocks of the Fast-SSC decoder (sm_103a), shared by the
// operation-list interpreter (polar_kernels.cu, compiled by nvcc) and by the
// per-code specialised decoders that polar_codegen.cpp emits and compiles at
// run time with NVRTC. The file therefore includes no host header when
// __CUDACC_RTC__ is defined.
//
// Method: Giard et al., "Low-Latency Software Polar Decoders" (arXiv 1504.00353),
// Sec. II-C/II-D: min-sum F (Eq. 1), G (Eq. 2) and G_0R, Combine (Eq. 3) and
// Combine_0R, Rate-0, Rate-1 (Eq. 4), Repetition and SPC nodes.
//
// Memory layout (Sec. III-B): the alpha stage of node size n occupies elements
// [n, 2n) of a per-CTA array, in shared memory for n <= S and in per-CTA
// device scratch above that; beta is one N-bit array (node (off, n) owns bits
// [off, off+n), Combine rewrites only the left half), bit-packed in shared
// memory. float32: F is an exact min with the XOR of the sign bits (beta in
// {+0,-0}), G adds alpha_v[i] with its sign flipped by beta_l (Listing 3): one
// IEEE add. int8: G is a saturating add followed by max(-127) (Listing 4);
// in memory-level operations the int8 values are computed as f16 pairs, which
// is exact for them (see op_i8x4). Every operation agrees bit for bit with a
// scalar evaluation in the same order.
#pragma once

#ifdef __CUDACC_RTC__
typedef unsigned int uint32_t;
typedef int int32_t;
typedef unsigned long long uint64_t;
typedef signed char int8_t;
typedef unsigned char uint8_t;
typedef unsigned long size_t;
typedef unsigned long uintptr_t;
#else
#include <cstddef>
#include <cstdint>
#endif

namespace polar {

// Operation kinds of the depth-first Fast-SSC list (Sec. II-D, Listing 1).
enum OpKind : uint32_t {
    OP_F = 0,     // alpha_l = f(alpha_v[i], alpha_v[i + N_v/2])          (Eq. 1)
    OP_G = 1,     // alpha_r = g(alpha_v[i], alpha_v[i + N_v/2], beta_l)  (Eq. 2)
    OP_G0R = 2,   // G with an all-zero beta_l (left child Rate-0)
    OP_C = 3,     // beta_v[i] ^= beta_v[i + N_v/2], i < N_v/2            (Eq. 3)
    OP_C0R = 4,   // beta_v[i] = beta_v[i + N_v/2] (left child Rate-0)
    OP_R0 = 5,    // beta_v = 0 (Rate-0 right child, or a Rate-0 root)
    OP_R1 = 6,    // beta_v[i] = alpha_v[i] < 0                           (Eq. 4)
    OP_REP = 7,   // Repetition: threshold of the folded sum, replicated
    OP_SPC = 8,   // SPC: hard decisions, flip least-|alpha| bit on odd parity
};

// How an operation reads its input stage: RD_NORMAL; RD_STREAM, an L2
// evict-first policy (the channel LLRs, read far apart in time); RD_LAST, the
// last read of a scratch stage before it is rewritten: evict-first, and the
// generated code then discards the lines (discard_l2) so that the dead data is
// never written back to DRAM. Hints only: the values read are the same.
enum : uint32_t { RD_NORMAL = 0, RD_STREAM = 1, RD_LAST = 2 };

// One operation as the interpreter reads it: a 32-bit word
//   bits 0-3   kind (OpKind)
//   bits 4-8   log2(N_v)
//   bit  9     inside a register-resident subtree (N_v <= kRegSubtree)
//   bit  10    first op of such a subtree: (N_v, off) is the subtree root
//   bit  11    last op of such a subtree: store its bits to beta
//   bits 12-31 off >> log2(N_v), off = index of the node's first leaf
enum : uint32_t {
    OPW_REG = 1u << 9,
    OPW_REG_ENTER = 1u << 10,
    OPW_REG_EXIT = 1u << 11,
};

__host__ __device__ inline uint32_t op_kind(uint32_t w) { return w & 0xFu; }
__host__ __device__ inline uint32_t op_log2n(uint32_t w) { return (w >> 4) & 0x1Fu; }
__host__ __device__ inline uint32_t op_off(uint32_t w) { return (w >> 12) << op_log2n(w); }

// Largest subtree the interpreter decodes in the registers of one warp.
constexpr uint32_t kRegSubtree = 32;

// Kernel parameters (identical layout for the interpreter and the generated
// decoders).
struct KernelArgs {
    const uint32_t *ops;           // n_ops packed operation words
    const uint32_t *trace_offs;    // per op: offset of its F/G/G_0R outputs in a trace row
    const uint32_t *ext_mask;      // info mask of each beta word (NW words)
    const uint32_t *ext_pre;       // info bits before beta word w (NW words)
    const uint32_t *ext_wstart;    // first beta word feeding output word u (KW words)
    int *status;                   // error flags (bit 0: a bounded wait expired)
    const void *llr;
    uint8_t *out;
    float *trace;
    void *gscratch;
    size_t n_frames;
    size_t trace_stride;           // floats per frame
    size_t gstride;                // scratch elements per CTA
    uint32_t n_ops;
    uint32_t N, log2N, K;
    uint32_t S;                    // smem_stage_max (already clipped to N/2)
    uint32_t log2W;                // ops with log2(N_v) <= log2W run on warp 0 alone
    uint32_t NW;                   // beta words (max(1, N/32))
    uint32_t KW;                   // output 32-bit words (ceil(K/32))
    uint32_t out_row;              // bytes per output row (ceil(K/8))
};

__host__ __device__ constexpr size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// One code of a mixed batch, as the batch kernel sees it.
struct CodeDesc {
    const uint32_t *ext_mask;      // as in KernelArgs
    const uint32_t *ext_pre;
    const uint32_t *ext_wstart;
    uint32_t N, K, NW, KW, out_row;
    uint32_t S;                    // smem_stage_max of this code (clipped to N/2)
};

// Parameters of the mixed-batch kernel: frame i belongs to code code_id[i],
// its LLRs start at element llr_off[i] of llr, its packed bits at byte
// out_off[i] of out. CTAs claim frames with an atomic counter.
struct BatchArgs {
    const CodeDesc *codes;
    const uint32_t *code_id;
    const unsigned long long *llr_off;
    const unsigned long long *out_off;
    const void *llr;
    uint8_t *out;
    unsigned int *counter;         // next unclaimed frame; zero before the launch
    void *gscratch;
    size_t gstride;                // scratch elements per frame slot (max over codes)
    size_t n_frames;
    uint32_t smem_alpha_elems;     // alpha region: max over codes of 2 * S
    uint32_t smem_beta_words;      // beta region: max over codes of NW
};

// Shared-memory bytes of one frame slot of the batch kernel (alpha, beta,
// reduction slots), computed identically on host and device.
__host__ __device__ inline size_t batch_slot_bytes(uint32_t alpha_elems, uint32_t beta_words,
                                                   uint32_t es) {
    return align_up(align_up(size_t(alpha_elems) * es, 128) + align_up(size_t(beta_words) * 4, 16) +
                        32 * 8 + 32 * 4,
                    128);
}


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

#if defined(__CUDACC__)

constexpr unsigned long long kWaitNs = 2000000000ull;  // bounded mbarrier wait: 2 s
constexpr uint32_t kWaitPolls = 1u << 28;              // and at most this many polls
constexpr uint32_t kFull = 0xffffffffu;

// ---------------------------------------------------------------- element ops

// Eq. 1: min(|a|, |b|) carrying the XOR of the two signs, one instruction.
__device__ __forceinline__ float f_f32(float a, float b) {
    float r;
    asm("min.xorsign.abs.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
    return r;
}
// Eq. 2 with beta_l as the sign bit of alpha_v[i] (Listing 3): one IEEE add.
__device__ __forceinline__ float g_f32(float a, float b, uint32_t bit) {
    return b + __uint_as_float(__float_as_uint(a) ^ (bit << 31));
}
__device__ __forceinline__ int sat127(int v) { return max(-127, min(127, v)); }
// Eq. 1 on integers: max(min(a, b), -max(a, b)) equals sgn(a) sgn(b) min(|a|, |b|)
// (both positive: min(a, b); both negative: -max(a, b) = min(|a|, |b|); mixed
// signs: the negative one of min(a, b) and -max(a, b) with the smaller magnitude).
__device__ __forceinline__ int f_i8s(int a, int b) { return max(min(a, b), -max(a, b)); }
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

// Four int8 lanes per 32-bit word, computed as two f16x2 pairs. Every int8
// value and every sum of two of them is an integer of magnitude <= 254, exact
// in f16, so F (one min.xorsign.abs, Eq. 1), G and G_0R (one IEEE add, Eq. 2,
// then the clamp to [-127, 127] that the saturating byte add followed by
// max(-127) gives) are exact: the results are the byte results bit for bit.
// The arithmetic runs on the FP16 units instead of byte-wise integer sequences.
__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel) {
    uint32_t r;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(sel));
    return r;
}
__device__ __forceinline__ uint32_t hadd2(uint32_t a, uint32_t b) {
    uint32_t r;
    asm("add.rn.f16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
    return r;
}
__device__ __forceinline__ uint32_t hmin2(uint32_t a, uint32_t b) {
    uint32_t r;
    asm("min.f16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
    return r;
}
__device__ __forceinline__ uint32_t hmax2(uint32_t a, uint32_t b) {
    uint32_t r;
    asm("max.f16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
    return r;
}
// Eq. 1 on two f16 lanes: min(|a|, |b|) carrying the XOR of the signs.
__device__ __forceinline__ uint32_t hf2(uint32_t a, uint32_t b) {
    uint32_t r;
    asm("min.xorsign.abs.f16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
    return r;
}
// Clamp both f16 lanes to [-127, 127] (0xD7F0 = -127, 0x57F0 = 127).
__device__ __forceinline__ uint32_t hsat2(uint32_t v) {
    return hmin2(hmax2(v, 0xD7F0D7F0u), 0x57F057F0u);
}

// Four int8 LLRs as two f16x2 words: bytes 0, 1 in lo, bytes 2, 3 in hi.
struct H4 {
    uint32_t lo, hi;
};
// Byte x (in [-127, 127]) flipped to x + 128 = x ^ 0x80 under the exponent
// byte 0x64 is the f16 1024 + x + 128 (f16 steps by 1 in [1024, 2048)); adding
// -1152 (0xE480) leaves x exactly.
__device__ __forceinline__ H4 h4_unpack(uint32_t w) {
    const uint32_t u = w ^ 0x80808080u;
    return {hadd2(prmt(u, 0x64646464u, 0x4140u), 0xE480E480u),
            hadd2(prmt(u, 0x64646464u, 0x4342u), 0xE480E480u)};
}
// Back to bytes: for an integer x in [-254, 254], 1280 + x (0x6500 = 1280) lies
// in [1024, 2048), so its mantissa is 256 + x, whose low byte is x mod 256: the
// two's-complement byte. (-0 maps to 0.)
__device__ __forceinline__ uint32_t h4_pack(H4 v) {
    return prmt(hadd2(v.lo, 0x65006500u), hadd2(v.hi, 0x65006500u), 0x6420u);
}
// F / G / G_0R on four LLRs; bits4 = beta_l of the four (bit k for element k).
// G flips the sign of alpha_v[i] where beta_l is 1 (Listing 3's sign XOR): the
// sign bits of elements 0..3 sit at bits 15, 31 of lo and of hi, and bit k of
// bits4 reaches them by one multiply (the partial products land on disjoint
// bits, so nothing carries).
template <uint32_t KIND>
__device__ __forceinline__ H4 h4_op(H4 a, H4 b, uint32_t bits4) {
    if constexpr (KIND == OP_F) {
        return {hf2(a.lo, b.lo), hf2(a.hi, b.hi)};
    } else if constexpr (KIND == OP_G) {
        const uint32_t ml = (bits4 * 0x40008000u) & 0x80008000u;
        const uint32_t mh = (bits4 * 0x10002000u) & 0x80008000u;
        return {hsat2(hadd2(b.lo, a.lo ^ ml)), hsat2(hadd2(b.hi, a.hi ^ mh))};
    } else {
        return {hsat2(hadd2(b.lo, a.lo)), hsat2(hadd2(b.hi, a.hi))};
    }
}
template <uint32_t KIND>
__device__ __forceinline__ uint32_t op_i8x4(uint32_t a, uint32_t b, uint32_t bits4) {
    return h4_pack(h4_op<KIND>(h4_unpack(a), h4_unpack(b), bits4));
}

// 32-bit word j of a 16-byte vector (j a constant after unrolling).
__device__ __forceinline__ uint32_t vword(const uint4 &v, uint32_t j) {
    return j == 0 ? v.x : (j == 1 ? v.y : (j == 2 ? v.z : v.w));
}
__device__ __forceinline__ void set_vword(uint4 &v, uint32_t j, uint32_t w) {
    if (j == 0) v.x = w;
    else if (j == 1) v.y = w;
    else if (j == 2) v.z = w;
    else v.w = w;
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

// ---------------------------------------------------------------- hinted device-memory reads

__device__ __forceinline__ unsigned long long evict_first_policy() {
    unsigned long long p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
template <uint32_t RD>
__device__ __forceinline__ uint4 ldv(const uint4 *p, unsigned long long pol) {
    if constexpr (RD == RD_NORMAL) {
        return *p;
    } else {
        uint4 r;
        asm volatile("ld.global.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
                     : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w) : "l"(p), "l"(pol) : "memory");
        return r;
    }
}
template <uint32_t RD>
__device__ __forceinline__ float4 ldv(const float4 *p, unsigned long long pol) {
    if constexpr (RD == RD_NORMAL) {
        return *p;
    } else {
        float4 r;
        asm volatile("ld.global.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
                     : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w) : "l"(p), "l"(pol) : "memory");
        return r;
    }
}
__device__ __forceinline__ unsigned long long policy_for(uint32_t rd) {
    return rd == RD_NORMAL ? 0ull : evict_first_policy();
}

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

// Drop [p, p + bytes) of a scratch stage from L2 without writing it back
// (discard.global.L2: afterwards the bytes are undefined until written again).
// Call after a group barrier that follows the stage's last read; p 128-byte
// aligned, bytes a multiple of 128.
template <class Grp>
__device__ __forceinline__ void discard_l2(const void *p, uint32_t bytes) {
    for (uint32_t off = Grp::rank() * 128u; off < bytes; off += Grp::size() * 128u)
        asm volatile("discard.global.L2 [%0], 128;" ::"l"(static_cast<const char *>(p) + off)
                     : "memory");
}

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
    r.x = op_i8x4<KIND>(a.x, b.x, bits & 0xFu);
    r.y = op_i8x4<KIND>(a.y, b.y, (bits >> 4) & 0xFu);
    r.z = op_i8x4<KIND>(a.z, b.z, (bits >> 8) & 0xFu);
    r.w = op_i8x4<KIND>(a.w, b.w, (bits >> 12) & 0xFu);
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
template <typename T, class Grp, uint32_t KIND, uint32_t RD = RD_NORMAL>
__device__ __forceinline__ void op_fg(const T *__restrict__ in, T *__restrict__ out, uint32_t h,
                                      const uint32_t *beta, uint32_t o) {
    using Vec = typename Llr<T>::Vec;
    constexpr uint32_t V = Llr<T>::V;
    if (h >= V) {
        const uint32_t nv = h / V, G = Grp::size();
        const Vec *va = reinterpret_cast<const Vec *>(in);
        const Vec *vb = reinterpret_cast<const Vec *>(in + h);
        Vec *vo = reinterpret_cast<Vec *>(out);
        const unsigned long long pol = policy_for(RD);
        uint32_t v = Grp::rank();
        for (; v + 3 * G < nv; v += 4 * G) {
            Vec a[4], b[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                a[k] = ldv<RD>(va + v + k * G, pol);
                b[k] = ldv<RD>(vb + v + k * G, pol);
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint32_t bits = KIND == OP_G ? bits_at(beta, o + (v + k * G) * V, V) : 0u;
                vo[v + k * G] = fg4<KIND>(a[k], b[k], bits);
            }
        }
        for (; v < nv; v += G) {
            const uint32_t bits = KIND == OP_G ? bits_at(beta, o + v * V, V) : 0u;
            vo[v] = fg4<KIND>(ldv<RD>(va + v, pol), ldv<RD>(vb + v, pol), bits);
        }
    } else {
        for (uint32_t i = Grp::rank(); i < h; i += Grp::size()) {
            const uint32_t bit = KIND == OP_G ? bits_at(beta, o + i, 1) : 0u;
            out[i] = fg_scalar<KIND, T>(in[i], in[i + h], bit);
        }
    }
}

// A chain of L = 2 or 3 operations down the tree, fused: K0 on node (o, n)
// (F, G or G_0R), then K1 and K2 (F or G_0R) on the node of the next stage
// that the previous operation produced the LLRs of. In list order these are
// consecutive operations, each reading the stage the one before it just
// wrote. Here every thread loads the 2^L inputs of one column of outputs
// (elements j + m n / 2^L of stage n) once, keeps the intermediate values in
// registers and stores each intermediate stage as well (a later operation
// reads it again) and the last one. Element by element this is the same
// arithmetic as the L operations one after another. stage1/2/3 = stages n/2,
// n/4, n/8; (n >> L) must be a multiple of the vector width.
// STORE: bit 0 stores stage n/2, bit 1 stage n/4 (for L = 3; the last stage
// is always stored): an intermediate stage that no later operation reads is
// not written at all. RD: how the input stage is read (see RD_LAST).
template <typename T, class Grp, uint32_t L, uint32_t K0, uint32_t K1, uint32_t K2,
          uint32_t STORE = 3u, uint32_t RD = RD_NORMAL>
__device__ __forceinline__ void op_chain(const T *__restrict__ in, T *__restrict__ stage1,
                                         T *__restrict__ stage2, T *__restrict__ stage3,
                                         uint32_t n, const uint32_t *beta, uint32_t o) {
    using Vec = typename Llr<T>::Vec;
    constexpr uint32_t V = Llr<T>::V, M = 1u << L;
    const uint32_t nvc = (n >> L) / V;  // vector columns of the last stage
    const Vec *vi = reinterpret_cast<const Vec *>(in);
    Vec *v1 = reinterpret_cast<Vec *>(stage1);
    Vec *v2 = reinterpret_cast<Vec *>(stage2);
    Vec *v3 = reinterpret_cast<Vec *>(stage3);
    const unsigned long long pol = policy_for(RD);
    for (uint32_t c = Grp::rank(); c < nvc; c += Grp::size()) {
        Vec x[M];
#pragma unroll
        for (uint32_t m = 0; m < M; ++m) x[m] = ldv<RD>(vi + c + m * nvc, pol);
        if constexpr (sizeof(T) == 1) {
            // int8: word by word in f16 pairs; intermediate stages are packed
            // back to bytes only where they are stored
            uint32_t gb[M / 2];
#pragma unroll
            for (uint32_t m = 0; m < M / 2; ++m)
                gb[m] = K0 == OP_G ? bits_at(beta, o + (c + m * nvc) * V, V) : 0u;
            Vec y[M / 2], z[M / 4], w;
#pragma unroll
            for (uint32_t j = 0; j < 4; ++j) {
                H4 xh[M], yh[M / 2], zh[M / 4];
#pragma unroll
                for (uint32_t m = 0; m < M; ++m) xh[m] = h4_unpack(vword(x[m], j));
#pragma unroll
                for (uint32_t m = 0; m < M / 2; ++m) {
                    yh[m] = h4_op<K0>(xh[m], xh[m + M / 2], (gb[m] >> (4 * j)) & 0xFu);
                    if (STORE & 1u) set_vword(y[m], j, h4_pack(yh[m]));
                }
#pragma unroll
                for (uint32_t m = 0; m < M / 4; ++m) {
                    zh[m] = h4_op<K1>(yh[m], yh[m + M / 4], 0u);
                    if (L == 2 || (STORE & 2u)) set_vword(z[m], j, h4_pack(zh[m]));
                }
                if constexpr (L == 3) set_vword(w, j, h4_pack(h4_op<K2>(zh[0], zh[1], 0u)));
            }
#pragma unroll
            for (uint32_t m = 0; m < M / 2; ++m)
                if (STORE & 1u) v1[c + m * nvc] = y[m];
#pragma unroll
            for (uint32_t m = 0; m < M / 4; ++m)
                if (L == 2 || (STORE & 2u)) v2[c + m * nvc] = z[m];
            if constexpr (L == 3) v3[c] = w;
        } else {
            Vec y[M / 2];
#pragma unroll
            for (uint32_t m = 0; m < M / 2; ++m) {
                const uint32_t bits = K0 == OP_G ? bits_at(beta, o + (c + m * nvc) * V, V) : 0u;
                y[m] = fg4<K0>(x[m], x[m + M / 2], bits);
                if (STORE & 1u) v1[c + m * nvc] = y[m];
            }
            Vec z[M / 4];
#pragma unroll
            for (uint32_t m = 0; m < M / 4; ++m) {
                z[m] = fg4<K1>(y[m], y[m + M / 4], 0u);
                if (L == 2 || (STORE & 2u)) v2[c + m * nvc] = z[m];
            }
            if constexpr (L == 3) v3[c] = fg4<K2>(z[0], z[1], 0u);
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

// Sign bits of the 16 int8 values of v, value k at bit k. Per word the sign
// bits 7, 15, 23, 31 are moved to bits 28..31 by one multiply (the partial
// products of 0x00204081 land on distinct bits, so nothing carries).
__device__ __forceinline__ uint32_t sign_bits16(uint4 v) {
    const uint32_t m0 = ((v.x & 0x80808080u) * 0x00204081u) >> 28;
    const uint32_t m1 = ((v.y & 0x80808080u) * 0x00204081u) >> 28;
    const uint32_t m2 = ((v.z & 0x80808080u) * 0x00204081u) >> 28;
    const uint32_t m3 = ((v.w & 0x80808080u) * 0x00204081u) >> 28;
    return m0 | (m1 << 4) | (m2 << 8) | (m3 << 12);
}

// Rate-1 (Eq. 4) on int8 LLRs, n >= 32: 16 values per lane per 16-byte load;
// lanes 2j and 2j + 1 of a warp hold the two halves of one beta word. Four
// loads per lane are in flight before the first is used.
template <class Grp>
__device__ __forceinline__ void op_r1_i8v(const int8_t *__restrict__ in, uint32_t *beta,
                                          uint32_t n, uint32_t o) {
    const uint4 *v = reinterpret_cast<const uint4 *>(in);
    const uint32_t nv = n >> 4, lane = threadIdx.x & 31u;
    const uint32_t w0 = Grp::kCta ? (threadIdx.x & ~31u) : 0u;
    const uint32_t step = Grp::kCta ? blockDim.x : 32u;
    for (uint32_t base = w0; base < nv; base += 4 * step) {
        uint32_t m[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint32_t i = base + k * step + lane;
            m[k] = i < nv ? sign_bits16(v[i]) : 0u;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint32_t i = base + k * step + lane;
            const uint32_t hi = __shfl_down_sync(kFull, m[k], 1);
            if (i < nv && !(lane & 1u)) beta[(o >> 5) + (i >> 1)] = m[k] | (hi << 16);
        }
    }
}

// Rate-1 (Eq. 4) on float32 LLRs, n >= 128: four values per lane per 16-byte
// load; the eight lanes 8w..8w+7 of a warp hold the 32 values of one beta word
// and OR their 4-bit pieces together with three shuffles. Four loads per lane
// are in flight before the first is used.
template <class Grp>
__device__ __forceinline__ void op_r1_f32v(const float *__restrict__ in, uint32_t *beta,
                                           uint32_t n, uint32_t o) {
    const float4 *v = reinterpret_cast<const float4 *>(in);
    const uint32_t nv = n >> 2, lane = threadIdx.x & 31u;
    const uint32_t w0 = Grp::kCta ? (threadIdx.x & ~31u) : 0u;
    const uint32_t step = Grp::kCta ? blockDim.x : 32u;
    for (uint32_t base = w0; base < nv; base += 4 * step) {
        uint32_t m[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint32_t i = base + k * step + lane;
            uint32_t b = 0;
            if (i < nv) {
                const float4 x = v[i];
                b = (__float_as_uint(x.x) >> 31) | ((__float_as_uint(x.y) >> 30) & 2u) |
                    ((__float_as_uint(x.z) >> 29) & 4u) | ((__float_as_uint(x.w) >> 28) & 8u);
            }
            m[k] = b << (4u * (lane & 7u));
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint32_t i = base + k * step + lane;
            uint32_t w = m[k];
            w |= __shfl_xor_sync(kFull, w, 1);
            w |= __shfl_xor_sync(kFull, w, 2);
            w |= __shfl_xor_sync(kFull, w, 4);
            if (i < nv && !(lane & 7u)) beta[(o >> 5) + (i >> 3)] = w;
        }
    }
}

// Rate-1 (Eq. 4): one ballot per 32 consecutive elements; four chunks loaded ahead.
template <typename T, class Grp>
__device__ __forceinline__ void op_r1(const T *__restrict__ in, uint32_t *beta, uint32_t n,
                                      uint32_t o) {
    if constexpr (sizeof(T) == 1) {
        if (n >= 32) {
            op_r1_i8v<Grp>(reinterpret_cast<const int8_t *>(in), beta, n, o);
            return;
        }
    } else {
        if (n >= 128) {
            op_r1_f32v<Grp>(reinterpret_cast<const float *>(in), beta, n, o);
            return;
        }
    }
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
// decision when the parity is odd (Listing 2 returns the first lane equal to
// the minimum).
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
    // the last folds: warp 0 of the CTA (CTA group), or the calling warp
    if (!Grp::kCta || threadIdx.x < 32) {
        const uint32_t lane = threadIdx.x & 31u;
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

// ---------------------------------------------------------------- L2 prefetch

// Ask L2 to fetch [p, p + bytes) ahead of use (cp.async.bulk.prefetch: a hint
// with nothing to wait for). Called by a whole warp; lane k issues the k-th
// 4 KiB slice. p 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void prefetch_l2(const void *p, uint32_t bytes) {
    for (uint32_t off = (threadIdx.x & 31u) * 4096u; off < bytes; off += 32u * 4096u) {
        const uint32_t n = bytes - off < 4096u ? bytes - off : 4096u;
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;"
                     ::"l"(static_cast<const char *>(p) + off), "r"(n) : "memory");
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
// Bounded wait for the phase with the given parity; false after limit_ns (or
// kWaitPolls polls).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity,
                                          unsigned long long limit_ns = kWaitNs) {
    const unsigned long long t0 = globaltimer();
    for (uint32_t i = 0; i < kWaitPolls; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
        if (ok) return true;
        if ((i & 63u) == 63u && globaltimer() - t0 > limit_ns) return false;
    }
    return false;
}

// ---------------------------------------------------------------- frame loop

// Persistent loop over the frames of a launch: frame f goes to CTA f % grid.
// For each frame `body(fr, trace_row)` runs the operation list; afterwards the
// estimate x_hat restricted to A is packed LSB first (output word u = info bits
// [32u, 32u+32)). With STAGE the frame's LLRs are brought into shared memory
// by cp.async.bulk, two frames ahead of use.
template <typename T, bool TRACE, bool STAGE, class Body>
__device__ __forceinline__ void run_frames(const KernelArgs &a, const Body &body) {
    extern __shared__ __align__(128) unsigned char smem[];
    const SmemLayout L(a.N, a.S, sizeof(T), STAGE);
    const uint32_t tid = threadIdx.x;

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

        body(fr, trace_row);

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

// Persistent loop with several frames per CTA, one per warp: the CTA's
// F = blockDim.x / 32 warps decode F frames side by side, each with its own
// shared-memory region and scratch, running the same straight-line decoder
// (every group operation of the body is warp-level). Barriers in the body keep
// the warps in step, so that they share the instructions they fetch. In the
// last group, warps without a frame decode frame 0 again and store nothing, so
// that every warp passes the same barriers.
template <typename T, class Body>
__device__ __forceinline__ void run_warp_frames(const KernelArgs &a, const Body &body) {
    extern __shared__ __align__(128) unsigned char smem[];
    const SmemLayout L(a.N, a.S, sizeof(T), false);
    const size_t per_frame = align_up(L.total, 128);
    const uint32_t lane = threadIdx.x & 31u, w = threadIdx.x >> 5, F = blockDim.x >> 5;
    unsigned char *base = smem + size_t(w) * per_frame;
    Frame<T> fr;
    fr.s_alpha = reinterpret_cast<T *>(base + L.alpha);
    fr.beta = reinterpret_cast<uint32_t *>(base + L.beta);
    fr.rkey = reinterpret_cast<unsigned long long *>(base + L.rkey);
    fr.rpar = reinterpret_cast<uint32_t *>(base + L.rpar);
    fr.g_alpha = a.gscratch
                     ? static_cast<T *>(a.gscratch) + (size_t(blockIdx.x) * F + w) * a.gstride
                     : nullptr;
    fr.N = a.N;
    fr.S = a.S;
    const T *llr = static_cast<const T *>(a.llr);
    const size_t groups = (a.n_frames + F - 1) / F;
    for (size_t g = blockIdx.x; g < groups; g += gridDim.x) {
        const size_t f = g * F + w;
        const bool valid = f < a.n_frames;
        fr.chan = llr + (valid ? f : 0) * a.N;
        body(fr, nullptr);
        if (valid) {
            uint8_t *out = a.out + f * a.out_row;
            for (uint32_t u = lane; u < a.KW; u += 32u) {
                const uint32_t lo = u << 5;
                const uint32_t hi = min(lo + 32u, a.K);
                uint32_t acc = 0;
                for (uint32_t wd = __ldg(a.ext_wstart + u); wd < a.NW; ++wd) {
                    const uint32_t pre = __ldg(a.ext_pre + wd);
                    if (pre >= hi) break;
                    const uint32_t m = __ldg(a.ext_mask + wd);
                    if (!m) continue;
                    const uint32_t e = pext32(fr.beta[wd], m);
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
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- out-of-line forms

// The memory-resident operations as real calls with run-time sizes: the compact
// form of a generated decoder uses them so that code size grows with the number
// of distinct subtrees, not with the length of the operation list.
template <typename T, class Grp, uint32_t KIND, uint32_t RD = RD_NORMAL>
__device__ __noinline__ void mem_fg(const T *in, T *out, uint32_t h, const uint32_t *beta,
                                    uint32_t o) {
    op_fg<T, Grp, KIND, RD>(in, out, h, beta, o);
}
template <typename T, class Grp, uint32_t L, uint32_t K0, uint32_t K1, uint32_t K2,
          uint32_t STORE = 3u, uint32_t RD = RD_NORMAL>
__device__ __noinline__ void mem_chain(const T *in, T *stage1, T *stage2, T *stage3, uint32_t n,
                                       const uint32_t *beta, uint32_t o) {
    op_chain<T, Grp, L, K0, K1, K2, STORE, RD>(in, stage1, stage2, stage3, n, beta, o);
}
template <class Grp>
__device__ __noinline__ void mem_combine(uint32_t *beta, uint32_t n, uint32_t o, bool copy) {
    op_combine<Grp>(beta, n, o, copy);
}
template <class Grp>
__device__ __noinline__ void mem_r0(uint32_t *beta, uint32_t n, uint32_t o) {
    op_r0<Grp>(beta, n, o);
}
template <typename T, class Grp>
__device__ __noinline__ void mem_r1(const T *in, uint32_t *beta, uint32_t n, uint32_t o) {
    op_r1<T, Grp>(in, beta, n, o);
}
template <typename T, class Grp>
__device__ __noinline__ void mem_rep(const T *in, T *tmp, uint32_t *beta, uint32_t n, uint32_t o) {
    op_rep<T, Grp>(in, tmp, beta, n, o);
}
template <typename T, class Grp>
__device__ __noinline__ void mem_spc(const T *in, uint32_t *beta, uint32_t n, uint32_t o,
                                     unsigned long long *rkey, uint32_t *rpar) {
    op_spc<T, Grp>(in, beta, n, o, rkey, rpar);
}

// ---------------------------------------------------------------- mixed batches

// Persistent loop of the mixed-batch kernel: each CTA claims the next frame,
// points its Frame at the frame's code (shared base pointers, per-code N and
// S), runs `body(code_id, fr)` and packs the frame's information bits.
template <typename T, class Body>
__device__ __forceinline__ void run_batch(const BatchArgs &a, const Body &body) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ unsigned int s_item;
    const uint32_t tid = threadIdx.x;
    const size_t alpha_bytes = align_up(size_t(a.smem_alpha_elems) * sizeof(T), 128);
    const size_t beta_bytes = align_up(size_t(a.smem_beta_words) * 4, 16);
    Frame<T> fr;
    fr.s_alpha = reinterpret_cast<T *>(smem);
    fr.beta = reinterpret_cast<uint32_t *>(smem + alpha_bytes);
    fr.rkey = reinterpret_cast<unsigned long long *>(smem + alpha_bytes + beta_bytes);
    fr.rpar = reinterpret_cast<uint32_t *>(smem + alpha_bytes + beta_bytes + 32 * 8);
    fr.g_alpha = a.gscratch ? static_cast<T *>(a.gscratch) + size_t(blockIdx.x) * a.gstride : nullptr;
    const T *llr = static_cast<const T *>(a.llr);
    for (;;) {
        if (tid == 0) s_item = atomicAdd(a.counter, 1u);
        __syncthreads();
        const size_t item = s_item;
        __syncthreads();  // every thread has read s_item before it is overwritten
        if (item >= a.n_frames) break;
        const uint32_t cid = __ldg(a.code_id + item);
        const CodeDesc d = a.codes[cid];
        fr.N = d.N;
        fr.S = d.S;
        fr.chan = llr + __ldg(a.llr_off + item);
        body(cid, fr);
        uint8_t *out = a.out + __ldg(a.out_off + item);
        for (uint32_t u = tid; u < d.KW; u += blockDim.x) {
            const uint32_t lo = u << 5;
            const uint32_t hi = min(lo + 32u, d.K);
            uint32_t acc = 0;
            for (uint32_t w = __ldg(d.ext_wstart + u); w < d.NW; ++w) {
                const uint32_t pre = __ldg(d.ext_pre + w);
                if (pre >= hi) break;
                const uint32_t m = __ldg(d.ext_mask + w);
                if (!m) continue;
                const uint32_t e = pext32(fr.beta[w], m);
                const int pos = static_cast<int>(pre) - static_cast<int>(lo);
                acc |= pos >= 0 ? (e << pos) : (e >> (-pos));
            }
            if (hi - lo < 32) acc &= (1u << (hi - lo)) - 1u;
            const uint32_t nb = min(4u, d.out_row - 4u * u);
            for (uint32_t b = 0; b < nb; ++b) out[4u * u + b] = static_cast<uint8_t>(acc >> (8 * b));
        }
        __syncthreads();
    }
}

// Persistent loop of the mixed-batch kernel with several frames per CTA, one
// per warp: the CTA claims F = blockDim.x / 32 consecutive frames of the list
// (listed longest code first, so they are almost always frames of one code)
// and its warps run that code's body side by side, each on its own frame,
// shared-memory slot and scratch slot, meeting at the CTA barriers the
// warp-level bodies place after each register subtree. When the F frames
// belong to several codes, the CTA runs the body of each of those codes in
// turn; in a turn, a warp whose frame is of another code decodes a copy of the
// turn's first frame of that code and stores nothing, so that every warp passes
// the same barriers. The same holds for the warps past the end of the list.
template <typename T, class Body>
__device__ __forceinline__ void run_batch_warps(const BatchArgs &a, const Body &body) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ unsigned int s_base;
    __shared__ uint32_t s_cid[32];
    const uint32_t lane = threadIdx.x & 31u, w = threadIdx.x >> 5, F = blockDim.x >> 5;
    const size_t slot = batch_slot_bytes(a.smem_alpha_elems, a.smem_beta_words, sizeof(T));
    unsigned char *base = smem + size_t(w) * slot;
    const size_t alpha_bytes = align_up(size_t(a.smem_alpha_elems) * sizeof(T), 128);
    const size_t beta_bytes = align_up(size_t(a.smem_beta_words) * 4, 16);
    Frame<T> fr;
    fr.s_alpha = reinterpret_cast<T *>(base);
    fr.beta = reinterpret_cast<uint32_t *>(base + alpha_bytes);
    fr.rkey = reinterpret_cast<unsigned long long *>(base + alpha_bytes + beta_bytes);
    fr.rpar = reinterpret_cast<uint32_t *>(base + alpha_bytes + beta_bytes + 32 * 8);
    fr.g_alpha = a.gscratch ? static_cast<T *>(a.gscratch) + (size_t(blockIdx.x) * F + w) * a.gstride
                            : nullptr;
    const T *llr = static_cast<const T *>(a.llr);
    for (;;) {
        if (threadIdx.x == 0) s_base = atomicAdd(a.counter, F);
        __syncthreads();
        const size_t first = s_base;
        if (first >= a.n_frames) break;
        const size_t item = first + w;
        if (lane == 0) s_cid[w] = __ldg(a.code_id + (item < a.n_frames ? item : first));
        __syncthreads();
        const uint32_t mine = s_cid[w];
        for (uint32_t k = 0; k < F; ++k) {
            const uint32_t cid = s_cid[k];
            bool seen = false;
            for (uint32_t j = 0; j < k; ++j) seen |= s_cid[j] == cid;
            if (seen) continue;  // this code's turn has been run
            const bool own = mine == cid && item < a.n_frames;
            const size_t src = own ? item : first + k;
            const CodeDesc d = a.codes[cid];
            fr.N = d.N;
            fr.S = d.S;
            fr.chan = llr + __ldg(a.llr_off + src);
            body(cid, fr);
            if (own) {
                uint8_t *out = a.out + __ldg(a.out_off + item);
                for (uint32_t u = lane; u < d.KW; u += 32u) {
                    const uint32_t lo = u << 5;
                    const uint32_t hi = min(lo + 32u, d.K);
                    uint32_t acc = 0;
                    for (uint32_t wd = __ldg(d.ext_wstart + u); wd < d.NW; ++wd) {
                        const uint32_t pre = __ldg(d.ext_pre + wd);
                        if (pre >= hi) break;
                        const uint32_t m = __ldg(d.ext_mask + wd);
                        if (!m) continue;
                        const uint32_t e = pext32(fr.beta[wd], m);
                        const int pos = static_cast<int>(pre) - static_cast<int>(lo);
                        acc |= pos >= 0 ? (e << pos) : (e >> (-pos));
                    }
                    if (hi - lo < 32) acc &= (1u << (hi - lo)) - 1u;
                    const uint32_t nb = min(4u, d.out_row - 4u * u);
                    for (uint32_t b = 0; b < nb; ++b) out[4u * u + b] = static_cast<uint8_t>(acc >> (8 * b));
                }
            }
            __syncthreads();
        }
    }
}

// ---------------------------------------------------------------- specialised subtrees

// Compile-time loop: f(UC<I>{}) for I in [B, E). Indices reach the body as
// template constants, so arrays indexed by them stay in registers.
template <uint32_t V> struct UC {
    static constexpr uint32_t value = V;
};
template <uint32_t B, uint32_t E, class F>
__device__ __forceinline__ void static_for(F &&f) {
    if constexpr (B < E) {
        f(UC<B>{});
        static_for<B + 1, E>(f);
    }
}

// Register-subtree arithmetic. Both LLR types are held in float registers:
// int8 LLRs are integers in [-127, 127], exact in float, and every sum of two
// of them is exact too. int8 keeps its saturation: each G and each Repetition
// fold is clamped to [-127, 127], which is what the saturating byte add
// followed by max(-127) gives. F is one min.xorsign.abs for both types.
template <typename T>
__device__ __forceinline__ float sat_reg(float v) {
    if constexpr (sizeof(T) == 1) return fminf(fmaxf(v, -127.0f), 127.0f);
    else return v;
}
template <typename T>
__device__ __forceinline__ float rop_f(float a, float b) { return f_f32(a, b); }
template <typename T>
__device__ __forceinline__ float rop_g(float a, float b, uint32_t bit) { return sat_reg<T>(g_f32(a, b, bit)); }
template <typename T>
__device__ __forceinline__ float rop_add(float a, float b) { return sat_reg<T>(a + b); }

// Subtree of at most R leaves decoded by warp 0 with compile-time node sizes and
// offsets (the generated decoders): stage m >= 32 is m/32 registers per lane
// (element j + 32k in register k of lane j), stages 1..16 share register A
// (stage m element j on lane m + j), and the subtree's bits are R/32 words held
// identically by every lane (word k = leaves [32k, 32k + 32) of the subtree).
// F and G above 32 leaves are lane-local; at 32 and below they are shuffles.
template <typename T, uint32_t R>
struct RegSub {
    using Acc = float;  // both LLR types (see rop_f)
    static constexpr uint32_t NWORD = R >= 32 ? R / 32 : 1;
    Acc s1024[32], s512[16], s256[8], s128[4], s64[2], s32, A;
    Acc l16[16], l8[8], l4[4], l2[2], l1;  // the per-lane form of nodes of <= 16 leaves
    uint32_t bw[NWORD];
    uint32_t lane;

    template <uint32_t m, uint32_t k>
    __device__ __forceinline__ Acc &reg() {
        if constexpr (m == 1024) return s1024[k];
        else if constexpr (m == 512) return s512[k];
        else if constexpr (m == 256) return s256[k];
        else if constexpr (m == 128) return s128[k];
        else if constexpr (m == 64) return s64[k];
        else return s32;
    }

    // Load the subtree root's LLRs (stage n0) from memory.
    template <uint32_t n0>
    __device__ __forceinline__ void enter(const T *src) {
        if constexpr (n0 >= 32) {
            static_for<0, n0 / 32>([&](auto kc) {
                constexpr uint32_t k = decltype(kc)::value;
                reg<n0, k>() = static_cast<Acc>(src[32 * k + lane]);
            });
        } else {
            A = (lane >= n0 && lane < 2 * n0) ? static_cast<Acc>(src[(lane - n0) & 31u]) : Acc(0);
        }
    }

    // Store the subtree's n0 bits at leaf offset o0 of beta. The words are the
    // same on every lane, so lane 0 stores them, 16 bytes at a time (o0 is a
    // multiple of n0, so the words are 16-byte aligned from 128 leaves up).
    template <uint32_t n0>
    __device__ __forceinline__ void exit(uint32_t *beta, uint32_t o0) {
        if constexpr (n0 >= 128) {
            if (lane == 0) {
                static_for<0, n0 / 128>([&](auto kc) {
                    constexpr uint32_t k = decltype(kc)::value;
                    uint4 q;
                    q.x = bw[4 * k];
                    q.y = bw[4 * k + 1];
                    q.z = bw[4 * k + 2];
                    q.w = bw[4 * k + 3];
                    *reinterpret_cast<uint4 *>(beta + (o0 >> 5) + 4 * k) = q;
                });
            }
        } else if constexpr (n0 >= 32) {
            if (lane == 0) {
                static_for<0, n0 / 32>([&](auto kc) {
                    constexpr uint32_t k = decltype(kc)::value;
                    beta[(o0 >> 5) + k] = bw[k];
                });
            }
        } else {
            if (lane == 0) write_field(beta, o0, n0, bw[0]);
        }
    }

    template <uint32_t w, uint32_t q, uint32_t width>
    __device__ __forceinline__ void set_field(uint32_t v) {
        if constexpr (width >= 32) {
            bw[w] = v;
        } else {
            constexpr uint32_t fm = ((1u << width) - 1u) << q;
            bw[w] = (bw[w] & ~fm) | ((v << q) & fm);
        }
    }

    // F / G / G_0R of a node of n leaves at subtree offset p.
    template <uint32_t KIND, uint32_t n, uint32_t p>
    __device__ __forceinline__ void fg() {
        if constexpr (n >= 64) {
            constexpr uint32_t K = n / 64;
            static_for<0, K>([&](auto kc) {
                constexpr uint32_t k = decltype(kc)::value;
                const Acc x = reg<n, k>(), y = reg<n, k + K>();
                Acc r;
                if constexpr (KIND == OP_F) r = rop_f<T>(x, y);
                else if constexpr (KIND == OP_G) r = rop_g<T>(x, y, (bw[p / 32 + k] >> lane) & 1u);
                else r = rop_add<T>(x, y);
                reg<n / 2, k>() = r;
            });
        } else if constexpr (n == 32) {
            // output element i = lane - 16 (lanes 16..31) from s32 of lanes i and i + 16
            const Acc x = __shfl_up_sync(kFull, s32, 16);
            const Acc y = s32;
            Acc r;
            if constexpr (KIND == OP_F) r = rop_f<T>(x, y);
            else if constexpr (KIND == OP_G) r = rop_g<T>(x, y, (bw[p / 32] >> ((lane - 16) & 31u)) & 1u);
            else r = rop_add<T>(x, y);
            if (lane >= 16) A = r;
        } else {
            constexpr uint32_t h = n / 2, q = p % 32;
            // output element i = lane - h (lanes [h, 2h)) from lanes n + i and n + i + h
            const Acc x = __shfl_down_sync(kFull, A, h);
            const Acc y = __shfl_down_sync(kFull, A, n);
            Acc r;
            if constexpr (KIND == OP_F) r = rop_f<T>(x, y);
            else if constexpr (KIND == OP_G) r = rop_g<T>(x, y, (bw[p / 32] >> ((q + lane - h) & 31u)) & 1u);
            else r = rop_add<T>(x, y);
            if (lane >= h && lane < 2 * h) A = r;
        }
    }

    // Combine (copy = false) / Combine_0R (copy = true) of a node of n leaves at p.
    template <uint32_t n, uint32_t p, bool copy>
    __device__ __forceinline__ void combine() {
        constexpr uint32_t h = n / 2;
        if constexpr (h >= 32) {
            static_for<0, h / 32>([&](auto kc) {
                constexpr uint32_t k = decltype(kc)::value;
                const uint32_t r = bw[(p + h) / 32 + k];
                bw[p / 32 + k] = copy ? r : (bw[p / 32 + k] ^ r);
            });
        } else {
            constexpr uint32_t w = p / 32, q = p % 32, m = (1u << h) - 1u;
            const uint32_t l = (bw[w] >> q) & m, r = (bw[w] >> (q + h)) & m;
            set_field<w, q, h>(copy ? r : (l ^ r));
        }
    }

    template <uint32_t n, uint32_t p>
    __device__ __forceinline__ void r0() {
        if constexpr (n >= 32) {
            static_for<0, n / 32>([&](auto kc) { bw[p / 32 + decltype(kc)::value] = 0u; });
        } else {
            set_field<p / 32, p % 32, n>(0u);
        }
    }

    template <uint32_t n, uint32_t p>
    __device__ __forceinline__ void r1() {
        if constexpr (n >= 32) {
            static_for<0, n / 32>([&](auto kc) {
                constexpr uint32_t k = decltype(kc)::value;
                bw[p / 32 + k] = __ballot_sync(kFull, reg<n, k>() < Acc(0));
            });
        } else {
            const bool in = lane >= n && lane < 2 * n;
            set_field<p / 32, p % 32, n>(__ballot_sync(kFull, in && A < Acc(0)) >> n);
        }
    }

    // Folds t[k] <- t[k] + t[k + m] for m = K/2, ..., 1 over K lane-local values.
    template <uint32_t K>
    __device__ __forceinline__ void fold_local(Acc (&t)[K]) {
        if constexpr (K > 1) {
            static_for<0, K / 2>([&](auto kc) {
                constexpr uint32_t k = decltype(kc)::value;
                t[k] = rop_add<T>(t[k], t[k + K / 2]);
            });
            fold_local<K / 2>(reinterpret_cast<Acc(&)[K / 2]>(t));
        }
    }

    template <uint32_t n, uint32_t p>
    __device__ __forceinline__ void rep() {
        Acc x;
        if constexpr (n >= 32) {
            constexpr uint32_t K = n / 32;
            Acc t[K];
            static_for<0, K>([&](auto kc) {
                constexpr uint32_t k = decltype(kc)::value;
                t[k] = reg<n, k>();
            });
            // lane-local folds t[e] += t[e + m] for m = n/2 .. 32 (e = lane + 32k)
            fold_local<K>(t);
            x = t[0];
#pragma unroll
            for (uint32_t m = 16; m >= 1; m /= 2) {
                const Acc y = __shfl_down_sync(kFull, x, m);
                if (lane < m) x = rop_add<T>(x, y);
            }
            x = __shfl_sync(kFull, x, 0);
            const uint32_t word = x < Acc(0) ? kFull : 0u;
            static_for<0, n / 32>([&](auto kc) { bw[p / 32 + decltype(kc)::value] = word; });
        } else {
            x = A;
#pragma unroll
            for (uint32_t m = n / 2; m >= 1; m /= 2) {
                const Acc y = __shfl_down_sync(kFull, x, m);
                if (lane >= n && lane < n + m) x = rop_add<T>(x, y);
            }
            x = __shfl_sync(kFull, x, n);
            set_field<p / 32, p % 32, n>(x < Acc(0) ? kFull : 0u);
        }
    }

    // ---- Per-lane form of a node of at most 16 leaves: every lane copies the
    // node's LLRs and decodes the whole node on its own, with no shuffles. Each
    // operation is the same arithmetic in the same order as its shuffle form
    // (F, G, the Repetition fold t[i] + t[i + m], the lowest-index SPC flip),
    // and the bits land in the same warp-uniform words. Fewer dependent steps
    // per operation than the shuffle form, more instructions: for one frame
    // in flight (latency), not for many.
    template <uint32_t m, uint32_t k>
    __device__ __forceinline__ Acc &loc() {
        if constexpr (m == 16) return l16[k];
        else if constexpr (m == 8) return l8[k];
        else if constexpr (m == 4) return l4[k];
        else if constexpr (m == 2) return l2[k];
        else return l1;
    }

    // Stage n0 (register A, lanes [n0, 2 n0)) to every lane.
    template <uint32_t n0>
    __device__ __forceinline__ void lenter() {
        static_for<0, n0>([&](auto kc) {
            constexpr uint32_t k = decltype(kc)::value;
            loc<n0, k>() = __shfl_sync(kFull, A, n0 + k);
        });
    }

    template <uint32_t KIND, uint32_t n, uint32_t p>
    __device__ __forceinline__ void lfg() {
        constexpr uint32_t h = n / 2;
        static_for<0, h>([&](auto kc) {
            constexpr uint32_t k = decltype(kc)::value;
            const Acc x = loc<n, k>(), y = loc<n, k + h>();
            Acc r;
            if constexpr (KIND == OP_F) r = rop_f<T>(x, y);
            else if constexpr (KIND == OP_G) r = rop_g<T>(x, y, (bw[p / 32] >> ((p % 32) + k)) & 1u);
            else r = rop_add<T>(x, y);
            loc<h, k>() = r;
        });
    }

    template <uint32_t n, uint32_t p>
    __device__ __forceinline__ uint32_t lhard() {
        uint32_t b = 0;
        static_for<0, n>([&](auto kc) {
            constexpr uint32_t k = decltype(kc)::value;
            b |= (loc<n, k>() < Acc(0) ? 1u : 0u) << k;
        });
        return b;
    }

    template <uint32_t n, uint32_t p>
    __device__ __forceinline__ void lr1() { set_field<p / 32, p % 32, n>(lhard<n, p>()); }

    template <uint32_t n, uint32_t p>
    __device__ __forceinline__ void lrep() {
        Acc t[n];
        static_for<0, n>([&](auto kc) { t[decltype(kc)::value] = loc<n, decltype(kc)::value>(); });
        fold_local<n>(t);
        set_field<p / 32, p % 32, n>(t[0] < Acc(0) ? kFull : 0u);
    }

    template <uint32_t n, uint32_t p>
    __device__ __forceinline__ void lspc() {
        const uint32_t hd = lhard<n, p>();
        uint32_t best = mag_bits(loc<n, 0>()), at = 0;
        static_for<1, n>([&](auto kc) {
            constexpr uint32_t k = decltype(kc)::value;
            const uint32_t mg = mag_bits(loc<n, k>());
            at = mg < best ? k : at;  // strictly smaller: the lowest index keeps a tie
            best = mg < best ? mg : best;
        });
        set_field<p / 32, p % 32, n>(hd ^ ((__popc(hd) & 1u) << at));
    }

    // Repetition-SPC node of n leaves (8 or 16) at subtree offset p, decoded
    // speculatively (Sec. II-D): F feeds the Repetition child while G for a
    // left estimate of all zeros and for one of all ones feed two SPC decodes;
    // the Repetition decision selects one SPC estimate and Eq. 3 joins the
    // halves. Bit-identical to F, rep, G, spc, combine in that order (the fold
    // order of the sum and the SPC tie rule are the ones rep<> and spc<> use).
    template <uint32_t n, uint32_t p>
    __device__ __forceinline__ void repspc() {
        static_assert(n == 8 || n == 16, "Repetition-SPC node in the shuffle layout");
        constexpr uint32_t h = n / 2;
        const bool act = lane < h;
        const Acc x = __shfl_sync(kFull, A, (n + lane) & 31u);      // alpha_v[i], i = lane
        const Acc y = __shfl_sync(kFull, A, (n + h + lane) & 31u);  // alpha_v[i + h]
        Acc s = rop_f<T>(x, y);
#pragma unroll
        for (uint32_t m = h / 2; m >= 1; m /= 2) {
            const Acc t = __shfl_down_sync(kFull, s, m);
            if (lane < m) s = rop_add<T>(s, t);
        }
        const bool one = __shfl_sync(kFull, s, 0) < Acc(0);
        const Acc g0 = rop_g<T>(x, y, 0u), g1 = rop_g<T>(x, y, 1u);
        const uint32_t hd0 = __ballot_sync(kFull, act && g0 < Acc(0));
        const uint32_t hd1 = __ballot_sync(kFull, act && g1 < Acc(0));
        const uint32_t m0 = act ? mag_bits(g0) : kFull, m1 = act ? mag_bits(g1) : kFull;
        const uint32_t mn0 = __reduce_min_sync(kFull, m0), mn1 = __reduce_min_sync(kFull, m1);
        const uint32_t f0 = __ffs(__ballot_sync(kFull, act && m0 == mn0)) - 1u;
        const uint32_t f1 = __ffs(__ballot_sync(kFull, act && m1 == mn1)) - 1u;
        const uint32_t r0 = hd0 ^ ((__popc(hd0) & 1u) << f0);
        const uint32_t r1 = hd1 ^ ((__popc(hd1) & 1u) << f1);
        const uint32_t right = one ? r1 : r0;
        const uint32_t left = (one ? (1u << h) - 1u : 0u) ^ right;
        set_field<p / 32, p % 32, n>(left | (right << h));
    }

    template <uint32_t n, uint32_t p>
    __device__ __forceinline__ void spc() {
        if constexpr (n >= 32) {
            constexpr uint32_t K = n / 32;
            uint32_t par = 0, mk = kFull;
            static_for<0, K>([&](auto kc) {
                constexpr uint32_t k = decltype(kc)::value;
                const uint32_t hd = __ballot_sync(kFull, reg<n, k>() < Acc(0));
                bw[p / 32 + k] = hd;
                par ^= __popc(hd);
                const uint32_t mg = mag_bits(reg<n, k>());
                mk = mg < mk ? mg : mk;
            });
            const uint32_t mn = __reduce_min_sync(kFull, mk);
            uint32_t e = kFull;  // lowest element index of this lane with |alpha| == mn
            static_for<0, K>([&](auto kc) {
                constexpr uint32_t k = K - 1 - decltype(kc)::value;
                if (mag_bits(reg<n, k>()) == mn) e = 32 * k + lane;
            });
            e = __reduce_min_sync(kFull, e);
            if (par & 1u) {
                static_for<0, K>([&](auto kc) {
                    constexpr uint32_t k = decltype(kc)::value;
                    if ((e >> 5) == k) bw[p / 32 + k] ^= 1u << (e & 31u);
                });
            }
        } else {
            const bool in = lane >= n && lane < 2 * n;
            const uint32_t hd = __ballot_sync(kFull, in && A < Acc(0)) >> n;
            const uint32_t mag = in ? mag_bits(A) : kFull;
            const uint32_t mn = __reduce_min_sync(kFull, mag);
            const uint32_t first = (__ffs(__ballot_sync(kFull, in && mag == mn)) - 1u - n) & 31u;
            set_field<p / 32, p % 32, n>(hd ^ ((__popc(hd) & 1u) << first));
        }
    }
};

// Pointer to stage n of a generated decoder with compile-time N and S.
template <typename T, uint32_t N, uint32_t S, uint32_t n>
__device__ __forceinline__ const T *gen_in(const Frame<T> &fr) {
    if constexpr (n == N) return fr.chan;
    else if constexpr (n <= S) return fr.s_alpha + n;
    else return fr.g_alpha + (n - 2 * S);
}
template <typename T, uint32_t S, uint32_t n>
__device__ __forceinline__ T *gen_out(const Frame<T> &fr) {
    if constexpr (n <= S) return fr.s_alpha + n;
    else return fr.g_alpha + (n - 2 * S);
}

#endif  // __CUDACC__

}  // namespace polar
