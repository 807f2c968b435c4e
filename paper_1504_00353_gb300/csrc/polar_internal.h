// Internal types shared by the host side (polar_host.cpp) and the CUDA kernels
// (polar_kernels.cu) of libpolar_gb300. Not part of the public ABI.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

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

// One operation as the kernel reads it: a 32-bit word
//   bits 0-3   kind (OpKind)
//   bits 4-8   log2(N_v)
//   bit  9     inside a register-resident subtree (N_v <= kRegSubtree)
//   bit  10    first op of such a subtree: (N_v, off) is the subtree root
//   bit  11    last op of such a subtree: store its bits to beta
//   bits 12-31 off >> log2(N_v), off = index of the node's first leaf
// Whether an op runs on one warp or on the whole CTA is decided at run time
// from N_v and the launch's warp_stage_max.
enum : uint32_t {
    OPW_REG = 1u << 9,
    OPW_REG_ENTER = 1u << 10,
    OPW_REG_EXIT = 1u << 11,
};

__host__ __device__ inline uint32_t op_kind(uint32_t w) { return w & 0xFu; }
__host__ __device__ inline uint32_t op_log2n(uint32_t w) { return (w >> 4) & 0x1Fu; }
__host__ __device__ inline uint32_t op_off(uint32_t w) { return (w >> 12) << op_log2n(w); }

// Largest subtree a warp decodes with its LLRs and bits held in registers.
constexpr uint32_t kRegSubtree = 32;

struct HostOp {
    uint32_t kind, log2n, off, flags;
};

// Launch shape of one decode.
struct LaunchShape {
    uint32_t threads;
    uint32_t smem_stage_max;  // S: stages of size <= S in shared memory
    uint32_t warp_stage_max;  // W: ops with N_v <= W run on warp 0 alone
    uint32_t ctas_per_sm;
    uint32_t stage_channel;   // 1 = bulk-copy the frame's LLRs to shared memory
    uint32_t grid;
    size_t smem_bytes;
    size_t scratch_elems_per_cta;  // device alpha scratch per CTA (elements)
};

struct KernelArgs {
    const uint32_t *ops;           // n_ops packed operation words
    const uint32_t *trace_offs;    // per op: offset of its F/G/G_0R outputs in a trace row
    const uint32_t *ext_mask;
    const uint32_t *ext_pre;
    const uint32_t *ext_wstart;
    int *status;
    const void *llr;
    uint8_t *out;
    float *trace;
    void *gscratch;
    size_t n_frames;
    size_t trace_stride;       // floats per frame
    size_t gstride;            // scratch elements per CTA
    uint32_t n_ops;
    uint32_t N, log2N, K;
    uint32_t S;                // smem_stage_max (already clipped to N/2)
    uint32_t log2W;            // ops with log2(N_v) <= log2W run on warp 0 alone
    uint32_t NW;               // beta words (max(1, N/32))
    uint32_t KW;               // output 32-bit words (ceil(K/32))
    uint32_t out_row;          // bytes per output row (ceil(K/8))
};

// Shared-memory bytes the kernel needs for a shape (alpha, beta, reduction
// slots, channel buffers and barriers), aligned pieces included.
size_t kernel_smem_bytes(uint32_t N, uint32_t S, uint32_t threads, bool is_i8,
                         bool stage_channel);

// Maximum resident CTAs per SM for the kernel variant and shape (occupancy API).
int kernel_max_ctas_per_sm(bool is_i8, bool stage_channel, uint32_t threads,
                           size_t smem_bytes);

// Launch the decode kernel. Returns the CUDA error of the launch.
cudaError_t launch_decode(bool is_i8, bool trace, bool stage_channel,
                          const LaunchShape &shape, const KernelArgs &args,
                          cudaStream_t stream);

}  // namespace polar
