// Internal types shared by the host side (polar_host.cpp, polar_codegen.cpp) and
// the CUDA kernels (polar_kernels.cu) of libpolar_gb300. Not part of the public ABI.
// Device-visible types (op words, KernelArgs, SmemLayout) live in polar_ops.cuh.
#pragma once

#include <cstddef>
#include <cstdint>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include <cuda_runtime.h>

#include "polar_gb300.h"
#include "polar_ops.cuh"

namespace polar {

constexpr uint32_t kMaxN = 1u << 20;
constexpr size_t kMaxDevices = 64;
// Operation lists longer than this are compiled in the compact form by default.
constexpr size_t kCompactOps = 4096;

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
    size_t scratch_elems_per_cta;  // device alpha scratch per frame slot (elements)
    uint32_t frames_per_cta;       // > 1: one frame per warp, `threads` = 32 x this
};

struct DeviceState {
    bool ready = false;
    int *status = nullptr;
    uint32_t *tables = nullptr;  // ops | trace_offs | ext_mask | ext_pre | ext_wstart
};

struct UserLaunch {
    uint32_t threads = 0, smem_stage_max = 0, warp_stage_max = 0, ctas_per_sm = 0,
             stage_channel = 0, frames_per_cta = 0;
};

// A decoder specialised to one code and launch shape (generated CUDA source
// compiled with NVRTC): key = (is_i8, threads, S, W, stage_channel, frames per CTA).
using CompiledKey = std::tuple<bool, uint32_t, uint32_t, uint32_t, uint32_t, uint32_t>;
struct CompiledKernel {
    cudaLibrary_t lib = nullptr;
    cudaKernel_t kernel = nullptr;
    uint32_t reg_subtree = 0;
    uint32_t outline = 0;  // kOutlineSubtrees | kOutlineMemory
    std::map<int, int> occupancy;  // device -> resident CTAs per SM
    std::map<int, void *> func;    // device -> CUfunction of `kernel` in its primary context
};

inline int log2u(uint32_t v) {
    int l = 0;
    while ((1u << l) < v) ++l;
    return l;
}

inline bool is_pow2(uint32_t v) { return v && !(v & (v - 1)); }

// Shared-memory bytes the kernel needs for a shape (alpha, beta, reduction
// slots, channel buffers and barriers), aligned pieces included.
size_t kernel_smem_bytes(uint32_t N, uint32_t S, uint32_t threads, bool is_i8,
                         bool stage_channel);

// Maximum resident CTAs per SM for the interpreter variant and shape.
int kernel_max_ctas_per_sm(bool is_i8, bool stage_channel, uint32_t threads,
                           size_t smem_bytes);

// Raise a kernel's dynamic shared-memory limit to the device maximum (once).
cudaError_t ensure_smem_limit(const void *k);

// Size of the static device scratch used by polar_decode_noalloc (per device).
constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;

// Device address of that scratch on the current device; the first call on a
// device looks it up with cudaGetSymbolAddress (no allocation).
cudaError_t noalloc_scratch(void **ptr);

// Launch the bounded-wait self-test: a wait that nothing completes gives up
// after limit_ns and sets bit 0 of *status (device memory).
cudaError_t launch_bounded_wait_selftest(int *status, unsigned long long limit_ns,
                                         cudaStream_t stream);

// Launch the interpreter kernel. Returns the CUDA error of the launch.
cudaError_t launch_decode(bool is_i8, bool trace, bool stage_channel,
                          const LaunchShape &shape, const KernelArgs &args,
                          cudaStream_t stream);

}  // namespace polar

// The code handle behind polar_code_t.
struct polar_code {
    enum NodeType { NT_R0, NT_R1, NT_REP, NT_SPC, NT_SPLIT };

    uint32_t N = 0, K = 0, log2N = 0, max_rep = UINT32_MAX, max_spc = UINT32_MAX;
    std::vector<uint8_t> frozen;
    std::vector<uint32_t> frozen_prefix;  // frozen count in [0, i)
    std::vector<uint32_t> info_idx;       // A in increasing order
    std::vector<polar::HostOp> ops;       // interpreter list (register subtrees <= 32)
    std::vector<uint32_t> trace_off;      // per op (F/G/G_0R), floats
    size_t trace_len = 0;
    uint32_t NW = 1, KW = 0;
    std::vector<uint32_t> ext_mask, ext_pre, ext_wstart;
    polar::UserLaunch user[2];
    std::mutex mu;
    // One slot per device ordinal, sized once so pointers into it stay valid.
    std::vector<polar::DeviceState> dev = std::vector<polar::DeviceState>(polar::kMaxDevices);
    std::map<polar::CompiledKey, polar::CompiledKernel> compiled;
    std::string compile_log;
    bool systematic_checked = false, systematic_valid = false;  // device encoder check

    // Node type from its leaves, in this order: all frozen -> Rate-0, none
    // frozen -> Rate-1, only the last leaf information -> Repetition, only the
    // first leaf frozen -> SPC (Sec. II-D), otherwise split. A size-2 node
    // [frozen, info] is therefore a Repetition node.
    NodeType classify(uint32_t off, uint32_t n) const {
        const uint32_t nf = frozen_prefix[off + n] - frozen_prefix[off];
        if (nf == n) return NT_R0;
        if (nf == 0) return NT_R1;
        if (nf == n - 1 && !frozen[off + n - 1] && n <= max_rep) return NT_REP;
        if (nf == 1 && frozen[off] && n <= max_spc) return NT_SPC;
        return NT_SPLIT;
    }

    // Depth-first operation list of Listing 1. A node with a Rate-0 left child
    // is G_0R, right subtree, Combine_0R; otherwise F, left subtree, then either
    // a Rate-0 fill of the right half (no G; Combine leaves beta_l as is) or G,
    // right subtree, Combine. Every maximal subtree of at most reg_max leaves is
    // marked as one register-resident subtree (first/last op flagged).
    std::vector<polar::HostOp> build_ops(uint32_t reg_max) const {
        std::vector<polar::HostOp> out;
        build_top(0, N, reg_max, out);
        return out;
    }

    void build_top(uint32_t off, uint32_t n, uint32_t reg_max,
                   std::vector<polar::HostOp> &out) const {
        if (n > reg_max) {
            build(off, n, reg_max, true, out);
            return;
        }
        const size_t first = out.size();
        build(off, n, reg_max, false, out);
        for (size_t i = first; i < out.size(); ++i) out[i].flags |= polar::OPW_REG;
        out[first].flags |= polar::OPW_REG_ENTER;
        out.back().flags |= polar::OPW_REG_EXIT;
    }

    void build(uint32_t off, uint32_t n, uint32_t reg_max, bool top,
               std::vector<polar::HostOp> &out) const {
        auto emit = [&](uint32_t kind, uint32_t size, uint32_t o) {
            out.push_back(polar::HostOp{kind, static_cast<uint32_t>(polar::log2u(size)), o, 0u});
        };
        switch (classify(off, n)) {
        case NT_R0: emit(polar::OP_R0, n, off); return;
        case NT_R1: emit(polar::OP_R1, n, off); return;
        case NT_REP: emit(polar::OP_REP, n, off); return;
        case NT_SPC: emit(polar::OP_SPC, n, off); return;
        default: break;
        }
        const uint32_t h = n / 2;
        auto child = [&](uint32_t o) {
            if (top) build_top(o, h, reg_max, out);
            else build(o, h, reg_max, false, out);
        };
        if (classify(off, h) == NT_R0) {
            emit(polar::OP_G0R, n, off);
            child(off + h);
            emit(polar::OP_C0R, n, off);
            return;
        }
        emit(polar::OP_F, n, off);
        child(off);
        if (classify(off + h, h) == NT_R0) {
            emit(polar::OP_R0, h, off + h);
            return;
        }
        emit(polar::OP_G, n, off);
        child(off + h);
        emit(polar::OP_C, n, off);
    }

    void build_tables() {
        frozen_prefix.assign(N + 1, 0);
        for (uint32_t i = 0; i < N; ++i) frozen_prefix[i + 1] = frozen_prefix[i] + frozen[i];
        info_idx.clear();
        for (uint32_t i = 0; i < N; ++i)
            if (!frozen[i]) info_idx.push_back(i);
        ops = build_ops(polar::kRegSubtree);
        trace_off.assign(ops.size(), 0);
        size_t t = 0;
        for (size_t i = 0; i < ops.size(); ++i) {
            trace_off[i] = static_cast<uint32_t>(t);
            if (ops[i].kind <= polar::OP_G0R) t += size_t(1) << (ops[i].log2n - 1);
        }
        trace_len = t;
        // Output packing: beta word w holds leaves [32w, 32w+32).
        NW = N >= 32 ? N / 32 : 1;
        KW = (K + 31) / 32;
        ext_mask.assign(NW, 0);
        ext_pre.assign(NW, 0);
        for (uint32_t i = 0; i < N; ++i)
            if (!frozen[i]) ext_mask[i >> 5] |= 1u << (i & 31);
        uint32_t pre = 0;
        for (uint32_t w = 0; w < NW; ++w) {
            ext_pre[w] = pre;
            pre += static_cast<uint32_t>(__builtin_popcount(ext_mask[w]));
        }
        ext_wstart.assign(KW, 0);
        uint32_t w = 0;
        for (uint32_t u = 0; u < KW; ++u) {
            const uint32_t lo = 32 * u;
            while (w < NW && ext_pre[w] + static_cast<uint32_t>(__builtin_popcount(ext_mask[w])) <= lo)
                ++w;
            ext_wstart[u] = w;
        }
    }

    // Packed operation words of the interpreter list (see polar_ops.cuh).
    std::vector<uint32_t> device_ops() const {
        std::vector<uint32_t> d(ops.size());
        for (size_t r = 0; r < ops.size(); ++r) {
            const polar::HostOp &o = ops[r];
            d[r] = o.kind | (o.log2n << 4) | o.flags | ((o.off >> o.log2n) << 12);
        }
        return d;
    }

    ~polar_code();
};

// The mixed-batch decoder behind polar_batch_t.
struct polar_batch {
    bool is_i8 = false;
    int device = -1;
    uint32_t threads = 32;
    std::vector<polar_code *> codes;
    std::vector<uint32_t> S, W, R;
    polar::CompiledKernel ck;
    polar::LaunchShape shape{};
    polar::CodeDesc *d_codes = nullptr;
    unsigned int *d_counter = nullptr;
    void *scratch = nullptr;
    size_t gstride = 0;  // scratch elements per frame slot
    uint32_t alpha_elems = 0, beta_words = 0;
    uint32_t frames_per_cta = 1;  // > 1: one frame per warp (POLAR_BATCH_FRAME_PER_WARP)
    std::string log;

    size_t elem_bytes() const { return is_i8 ? 1 : 4; }
    // CTAs one launch over n_frames frames uses.
    size_t grid_for(size_t n_frames) const {
        const size_t groups = (n_frames + frames_per_cta - 1) / frames_per_cta;
        return groups < shape.grid ? groups : shape.grid;
    }
    // Scratch bytes one launch over n_frames frames needs.
    size_t scratch_bytes(size_t n_frames) const {
        return grid_for(n_frames) * frames_per_cta * gstride * elem_bytes();
    }
    ~polar_batch();
};

namespace polar {
// Source text of the decoder specialised to `code` for one launch shape.
// outline: kOutlineSubtrees makes every register subtree a call to one
// out-of-line function per distinct frozen pattern; kOutlineMemory makes the
// memory-resident operations out-of-line calls with run-time sizes. Both keep
// very long operation lists (N = 2^20) compilable.
constexpr uint32_t kOutlineSubtrees = 1u, kOutlineMemory = 2u;
// Split nodes of 4 to 16 leaves inside register subtrees in the per-lane form
// (every lane decodes the node alone; see RegSub::lenter): shorter dependent
// chains for one frame in flight.
constexpr uint32_t kLocalLeaves = 4u;
std::string generate_source(const polar_code &code, bool is_i8, const LaunchShape &shape,
                            uint32_t reg_subtree, uint32_t outline = 0);
// Source of the mixed-batch decoder: one specialised body per code (per-code
// shared-memory stage cap S, warp threshold W, register subtree R); outline as
// for generate_source, with the subtree functions shared by all bodies.
std::string generate_batch_source(const std::vector<const polar_code *> &codes, bool is_i8,
                                  const std::vector<uint32_t> &S, const std::vector<uint32_t> &W,
                                  const std::vector<uint32_t> &R, uint32_t threads,
                                  uint32_t min_blocks, uint32_t outline = 0,
                                  bool warp_frames = false);
// Compile generated source with NVRTC for the current device's architecture and
// load `kernel_name` from it. Returns cudaSuccess and fills *out, or an error
// (log in *log).
cudaError_t compile_source(const std::string &src, CompiledKernel *out, std::string *log,
                           const char *kernel_name = "polar_unrolled");
// Resident CTAs per SM of a compiled decoder on the current device (0 on error);
// also raises its dynamic shared-memory limit to the device maximum.
int compiled_max_ctas(CompiledKernel *ck, uint32_t threads, size_t smem_bytes);
// Launch a compiled decoder on the current device.
cudaError_t launch_compiled(CompiledKernel *ck, const LaunchShape &shape, const void *args,
                            cudaStream_t stream);
// The library's stream-ordered memory pool on `device` (created on first use):
// freed blocks stay cached in it, so per-call scratch does not go back to the
// driver at every synchronisation (the default pool releases at a threshold of
// zero). Returns nullptr if the pool cannot be created.
cudaMemPool_t device_pool(int device);
// cudaMallocAsync from that pool (falls back to the default pool).
cudaError_t pool_alloc(void **p, size_t bytes, int device, cudaStream_t s);
// The code's tables on `device` (uploaded on first use): op words, trace
// offsets and the info-bit packing tables (see DeviceState).
polar_status code_device_state(polar_code *c, int device, DeviceState **out);
// Launch the batch decoder over n_frames frames with the given work counter and
// alpha scratch (grid = min(resident CTAs, n_frames)); zeroes the counter on
// the stream first. polar_batch_decode passes the batch's own workspace, the
// serving loop one workspace per in-flight launch.
cudaError_t batch_launch(polar_batch *b, const uint32_t *code_id, const uint64_t *llr_off,
                         const uint64_t *out_off, const void *llr, uint8_t *out, size_t n_frames,
                         unsigned int *counter, void *scratch, cudaStream_t stream);
}  // namespace polar
