// Mixed-code batches: one persistent kernel decodes frames of several polar
// codes from a work queue, each frame with the decoder body specialised to its
// code (polar_codegen.cpp). Everything the launch needs (descriptor table,
// work counter, alpha scratch for the resident CTAs) is allocated when the
// batch decoder is created, so a decode call allocates nothing and a stream
// that issues it can be captured in a CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "polar_gb300.h"
#include "polar_internal.h"

using namespace polar;

namespace {

// Log of the last polar_batch_create that failed on this thread.
thread_local std::string g_failed_log;

polar_status st_of(cudaError_t e) {
    if (e == cudaSuccess) return POLAR_OK;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? POLAR_ENOMEM : POLAR_ECUDA;
}

}  // namespace

polar_batch::~polar_batch() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (device >= 0) cudaSetDevice(device);
    cudaFree(d_codes);
    cudaFree(d_counter);
    cudaFree(scratch);
    if (ck.lib) cudaLibraryUnload(ck.lib);
    if (cur >= 0) cudaSetDevice(cur);
}

namespace polar {

cudaError_t batch_launch(polar_batch *b, const uint32_t *code_id, const uint64_t *llr_off,
                         const uint64_t *out_off, const void *llr, uint8_t *out, size_t n_frames,
                         unsigned int *counter, void *scratch, cudaStream_t stream) {
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned int), stream);
    if (e != cudaSuccess) return e;
    BatchArgs a{};
    a.codes = b->d_codes;
    a.code_id = code_id;
    a.llr_off = reinterpret_cast<const unsigned long long *>(llr_off);
    a.out_off = reinterpret_cast<const unsigned long long *>(out_off);
    a.llr = llr;
    a.out = out;
    a.counter = counter;
    a.gscratch = scratch;
    a.gstride = b->gstride;
    a.n_frames = n_frames;
    a.smem_alpha_elems = b->alpha_elems;
    a.smem_beta_words = b->beta_words;
    LaunchShape sh = b->shape;
    sh.grid = static_cast<uint32_t>(b->grid_for(n_frames));
    return launch_compiled(&b->ck, sh, &a, stream);
}

}  // namespace polar

extern "C" {

polar_status polar_batch_create(polar_code_t *const *codes, uint32_t n_codes, int is_i8,
                                uint32_t threads, const uint32_t *smem_stage_max,
                                const uint32_t *warp_stage_max, uint32_t ctas_per_sm,
                                polar_batch_t **out) {
    return polar_batch_create_ex(codes, n_codes, is_i8, threads, smem_stage_max, warp_stage_max,
                                 ctas_per_sm, 0, out);
}

polar_status polar_batch_create_ex(polar_code_t *const *codes, uint32_t n_codes, int is_i8,
                                   uint32_t threads, const uint32_t *smem_stage_max,
                                   const uint32_t *warp_stage_max, uint32_t ctas_per_sm,
                                   uint32_t flags, polar_batch_t **out) {
    if (!codes || !out || n_codes == 0 || n_codes > 64) return POLAR_EINVAL;
    if (flags & ~(POLAR_COMPILE_OUTLINE_SUBTREES | POLAR_BATCH_FRAME_PER_WARP)) return POLAR_EINVAL;
    if (threads == 0) threads = 32;
    if (threads % 32 || threads > 1024) return POLAR_EINVAL;
    const bool warp_frames = (flags & POLAR_BATCH_FRAME_PER_WARP) && threads > 32;
    if (warp_frames && threads > 32 * 8) return POLAR_EINVAL;  // at most 8 frames per CTA
    for (uint32_t c = 0; c < n_codes; ++c) {
        if (!codes[c]) return POLAR_EINVAL;
        if (smem_stage_max && smem_stage_max[c] && !is_pow2(smem_stage_max[c])) return POLAR_EINVAL;
        if (warp_stage_max && warp_stage_max[c] && !is_pow2(warp_stage_max[c])) return POLAR_EINVAL;
    }
    int device = -1;
    if (cudaGetDevice(&device) != cudaSuccess) {
        cudaGetLastError();
        return POLAR_ECUDA;
    }
    polar_batch *b = new (std::nothrow) polar_batch;
    if (!b) return POLAR_ENOMEM;
    b->is_i8 = is_i8 != 0;
    b->device = device;
    b->threads = threads;
    b->frames_per_cta = warp_frames ? threads / 32 : 1;
    const size_t es = b->elem_bytes();
    constexpr uint32_t kReg = 256;  // register-resident subtree size of every body
    std::vector<CodeDesc> desc(n_codes);
    std::vector<const polar_code *> cc;
    for (uint32_t c = 0; c < n_codes; ++c) {
        polar_code *code = codes[c];
        uint32_t s = smem_stage_max && smem_stage_max[c] ? smem_stage_max[c]
                                                         : (threads == 32 ? 512u : 2048u);
        s = std::min<uint32_t>(std::max<uint32_t>(s, 64), std::max<uint32_t>(code->N / 2, 1));
        const uint32_t w = warp_stage_max && warp_stage_max[c] ? warp_stage_max[c] : 2048u;
        b->codes.push_back(code);
        b->S.push_back(s);
        b->W.push_back(std::max(w, kReg));  // register subtrees run inside warp-0 runs
        b->R.push_back(kReg);
        cc.push_back(code);
        b->alpha_elems = std::max(b->alpha_elems, 2 * s);
        b->beta_words = std::max(b->beta_words, code->NW);
        const size_t g = (code->N / 2 > s) ? size_t(code->N) - 2 * size_t(s) : 0;
        b->gstride = std::max(b->gstride, g ? ((g * es + 127) / 128 * 128) / es : size_t(0));
    }
    // device tables of every code
    for (uint32_t c = 0; c < n_codes; ++c) {
        polar_code *code = b->codes[c];
        std::lock_guard<std::mutex> g(code->mu);
        if (!code->dev[device].ready) {
            delete b;
            return POLAR_EINVAL;  // create the codes with this device current
        }
        const DeviceState &ds = code->dev[device];
        const size_t nops = code->ops.size();
        desc[c].ext_mask = ds.tables + 2 * nops;
        desc[c].ext_pre = ds.tables + 2 * nops + code->NW;
        desc[c].ext_wstart = ds.tables + 2 * nops + 2 * code->NW;
        desc[c].N = code->N;
        desc[c].K = code->K;
        desc[c].NW = code->NW;
        desc[c].KW = code->KW;
        desc[c].out_row = (code->K + 7) / 8;
        desc[c].S = b->S[c];
    }
    const size_t smem =
        warp_frames ? b->frames_per_cta * batch_slot_bytes(b->alpha_elems, b->beta_words,
                                                           static_cast<uint32_t>(es))
                    : align_up(size_t(b->alpha_elems) * es, 128) +
                          align_up(size_t(b->beta_words) * 4, 16) + 32 * 8 + 32 * 4;
    int optin = 0, sms = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (smem > size_t(optin) || sms <= 0) {
        delete b;
        return POLAR_EINVAL;
    }
    // resident CTAs per SM the shared memory allows; the register budget of the
    // generated kernel is capped so that this many fit (or ctas_per_sm if lower)
    size_t min_blocks = std::min<size_t>({size_t(228 * 1024) / (smem + 1024), size_t(2048 / threads),
                                          size_t(32)});
    if (ctas_per_sm) min_blocks = std::min<size_t>(min_blocks, ctas_per_sm);
    min_blocks = std::max<size_t>(min_blocks, 1);
    const std::string src = generate_batch_source(
        cc, b->is_i8, b->S, b->W, b->R, threads, static_cast<uint32_t>(min_blocks),
        (flags & POLAR_COMPILE_OUTLINE_SUBTREES) ? kOutlineSubtrees : 0u, warp_frames);
    cudaError_t e = compile_source(src, &b->ck, &b->log, "polar_batch");
    if (e != cudaSuccess) {
        const polar_status st = st_of(e);
        g_failed_log = b->log + "\n(compile status " + std::to_string(static_cast<int>(e)) + ")";
        delete b;
        return st;
    }
    int occ = compiled_max_ctas(&b->ck, threads, smem);
    if (ctas_per_sm) occ = std::min<int>(occ, static_cast<int>(ctas_per_sm));
    if (occ <= 0) {
        g_failed_log = b->log + "\nno CTA of this shape can be resident (smem " +
                       std::to_string(smem) + " bytes, " + std::to_string(threads) + " threads)";
        delete b;
        return POLAR_ECUDA;
    }
    b->shape.threads = threads;
    b->shape.smem_bytes = smem;
    b->shape.grid = static_cast<uint32_t>(sms * occ);
    b->shape.ctas_per_sm = static_cast<uint32_t>(occ);
    b->shape.scratch_elems_per_cta = b->gstride;
    e = cudaMalloc(&b->d_codes, sizeof(CodeDesc) * n_codes);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_codes, desc.data(), sizeof(CodeDesc) * n_codes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_counter, sizeof(unsigned int));
    if (e == cudaSuccess && b->gstride)
        e = cudaMalloc(&b->scratch, b->scratch_bytes(size_t(b->shape.grid) * b->frames_per_cta));
    if (e != cudaSuccess) {
        const polar_status st = st_of(e);
        delete b;
        return st;
    }
    *out = b;
    return POLAR_OK;
}

void polar_batch_destroy(polar_batch_t *batch) { delete batch; }

polar_status polar_batch_decode(polar_batch_t *b, const uint32_t *code_id, const uint64_t *llr_off,
                                const uint64_t *out_off, const void *llr, uint8_t *bits_out,
                                size_t n_frames, polar_stream_t stream) {
    if (!b) return POLAR_EINVAL;
    if (n_frames == 0) return POLAR_OK;
    if (!code_id || !llr_off || !out_off || !llr || !bits_out) return POLAR_EINVAL;
    if (n_frames > 0xFFFFFFFFull) return POLAR_EINVAL;  // the work counter is 32-bit
    if (reinterpret_cast<uintptr_t>(llr) % 16 != 0) return POLAR_EALIGN;
    int device = -1;
    if (cudaGetDevice(&device) != cudaSuccess || device != b->device) {
        cudaGetLastError();
        return POLAR_ECUDA;
    }
    return st_of(batch_launch(b, code_id, llr_off, out_off, llr, bits_out, n_frames, b->d_counter,
                              b->scratch, reinterpret_cast<cudaStream_t>(stream)));
}

polar_status polar_batch_info(const polar_batch_t *b, uint32_t *threads, uint32_t *grid,
                              size_t *smem_bytes, size_t *scratch_bytes) {
    if (!b) return POLAR_EINVAL;
    if (threads) *threads = b->shape.threads;
    if (grid) *grid = b->shape.grid;
    if (smem_bytes) *smem_bytes = b->shape.smem_bytes;
    if (scratch_bytes) *scratch_bytes = b->scratch_bytes(size_t(b->shape.grid) * b->frames_per_cta);
    return POLAR_OK;
}

const char *polar_batch_log(const polar_batch_t *b) { return b ? b->log.c_str() : g_failed_log.c_str(); }

}  // extern "C"
