// Host side of libpolar_gb300: code handles, the Fast-SSC operation-list
// compiler, output-packing tables, the systematic encoder, launch-shape
// selection and the C ABI entry points declared in include/polar_gb300.h.
//
// Method: Giard et al., "Low-Latency Software Polar Decoders" (arXiv 1504.00353).
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdint>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include "polar_gb300.h"
#include "polar_internal.h"

using namespace polar;

polar_code::~polar_code() {
    int cur = -1;
    cudaGetDevice(&cur);
    for (auto &kv : compiled)
        if (kv.second.lib) cudaLibraryUnload(kv.second.lib);
    for (size_t d = 0; d < dev.size(); ++d) {
        DeviceState &s = dev[d];
        if (!s.ready) continue;
        if (cudaSetDevice(static_cast<int>(d)) != cudaSuccess) continue;
        cudaFree(s.status);
        cudaFree(s.tables);
    }
    if (cur >= 0) cudaSetDevice(cur);
}


namespace {

// Make sure `device` holds the code's tables (uploaded once, under the lock).
polar_status ensure_device(polar_code *c, int device, DeviceState **out) {
    std::lock_guard<std::mutex> g(c->mu);
    if (device < 0 || static_cast<size_t>(device) >= c->dev.size()) return POLAR_ECUDA;
    DeviceState &s = c->dev[device];
    if (!s.ready) {
        const size_t nops = c->ops.size();
        const size_t n = 2 * nops + size_t(c->NW) * 2 + c->KW;
        std::vector<uint32_t> h(std::max<size_t>(n, 1), 0);
        const std::vector<uint32_t> d = c->device_ops();
        std::copy(d.begin(), d.end(), h.begin());
        std::copy(c->trace_off.begin(), c->trace_off.end(), h.begin() + nops);
        std::copy(c->ext_mask.begin(), c->ext_mask.end(), h.begin() + 2 * nops);
        std::copy(c->ext_pre.begin(), c->ext_pre.end(), h.begin() + 2 * nops + c->NW);
        std::copy(c->ext_wstart.begin(), c->ext_wstart.end(), h.begin() + 2 * nops + 2 * c->NW);
        if (cudaMalloc(&s.status, sizeof(int)) != cudaSuccess) return POLAR_ENOMEM;
        if (cudaMalloc(&s.tables, h.size() * 4) != cudaSuccess) {
            cudaFree(s.status);
            s.status = nullptr;
            return POLAR_ENOMEM;
        }
        if (cudaMemset(s.status, 0, sizeof(int)) != cudaSuccess ||
            cudaMemcpy(s.tables, h.data(), h.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaFree(s.status);
            cudaFree(s.tables);
            s.status = nullptr;
            s.tables = nullptr;
            return POLAR_ECUDA;
        }
        s.ready = true;
    }
    *out = &s;
    return POLAR_OK;
}

struct DeviceProps {
    int sms = 0;
    int max_blocks_per_sm = 32;
    size_t smem_optin = 0;
};

DeviceProps device_props(int device) {
    static std::mutex mu;
    static std::map<int, DeviceProps> cache;
    std::lock_guard<std::mutex> g(mu);
    auto it = cache.find(device);
    if (it != cache.end()) return it->second;
    DeviceProps p;
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device) == cudaSuccess) p.sms = v;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) == cudaSuccess)
        p.smem_optin = static_cast<size_t>(v);
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxBlocksPerMultiprocessor, device) == cudaSuccess && v > 0)
        p.max_blocks_per_sm = v;
    cache[device] = p;
    return p;
}

// Resident CTAs per SM for a kernel variant and shape, cached per device.
int occupancy(int device, bool is_i8, bool stage, uint32_t T, size_t smem) {
    static std::mutex mu;
    static std::map<std::tuple<int, bool, bool, uint32_t, size_t>, int> cache;
    const auto key = std::make_tuple(device, is_i8, stage, T, smem);
    {
        std::lock_guard<std::mutex> g(mu);
        auto it = cache.find(key);
        if (it != cache.end()) return it->second;
    }
    const int n = kernel_max_ctas_per_sm(is_i8, stage, T, smem);
    std::lock_guard<std::mutex> g(mu);
    cache[key] = n;
    return n;
}

uint32_t pow2_floor(uint32_t v) {
    uint32_t p = 1;
    while (p * 2 <= v) p *= 2;
    return p;
}

// Launch shape for a decode of n_frames frames on `device`.
polar_status choose_shape(const polar_code *c, bool is_i8, size_t n_frames, int device,
                          LaunchShape *sh) {
    const DeviceProps dp = device_props(device);
    if (dp.sms <= 0 || dp.smem_optin == 0) return POLAR_ECUDA;
    const UserLaunch &u = c->user[is_i8 ? 1 : 0];
    const uint32_t es = is_i8 ? 1 : 4;
    const uint32_t N = c->N;
    const bool latency = n_frames * 2 <= static_cast<size_t>(dp.sms);

    // Throughput: many small CTAs per SM (the serial part of a frame runs on one
    // warp, so resident frames, not threads per frame, set the rate).
    // Latency: one CTA with every stage in shared memory.
    uint32_t T = u.threads;
    if (!T) {
        if (latency) T = N >= 8192 ? 1024 : std::max<uint32_t>(64, pow2_floor(std::max<uint32_t>(N / 8, 32)));
        else T = 128;
    }
    T = std::min<uint32_t>(std::max<uint32_t>(T, 32), 1024);

    const bool can_stage = (size_t(N) * es) % 16 == 0;
    const size_t budget = latency ? dp.smem_optin : std::min<size_t>(dp.smem_optin, 24 * 1024);
    uint32_t S = u.smem_stage_max ? std::max<uint32_t>(u.smem_stage_max, 64) : 0;
    if (!S) {
        S = std::max<uint32_t>(N / 2, 1);
        while (S > 64 && kernel_smem_bytes(N, S, T, is_i8, false) > budget) S /= 2;
    }
    S = std::min<uint32_t>(S, std::max<uint32_t>(N / 2, 1));
    uint32_t stage = 0;
    if (u.stage_channel == 1) stage = can_stage ? 1 : 0;
    else if (u.stage_channel == 2) stage = 0;
    else stage = (can_stage && kernel_smem_bytes(N, S, T, is_i8, true) <= budget) ? 1 : 0;
    // Too little SMEM for the chosen shape: fall back to smaller stages.
    while (kernel_smem_bytes(N, S, T, is_i8, stage) > dp.smem_optin && S > 64) S /= 2;
    if (kernel_smem_bytes(N, S, T, is_i8, stage) > dp.smem_optin) {
        if (stage) stage = 0;
        if (kernel_smem_bytes(N, S, T, is_i8, stage) > dp.smem_optin) return POLAR_EINVAL;
    }
    const uint32_t W = std::max<uint32_t>(u.warp_stage_max ? u.warp_stage_max : 512, kRegSubtree);
    const size_t smem = kernel_smem_bytes(N, S, T, is_i8, stage);
    sh->threads = T;
    sh->smem_stage_max = S;
    sh->warp_stage_max = W;
    sh->stage_channel = stage;
    sh->smem_bytes = smem;
    const size_t g = (N / 2 > S) ? size_t(N) - 2 * size_t(S) : 0;
    sh->scratch_elems_per_cta = g ? ((g * es + 127) / 128 * 128) / es : 0;
    sh->ctas_per_sm = 0;
    sh->grid = 0;
    return POLAR_OK;
}

// The decoder specialised to this code and shape, if one was compiled.
CompiledKernel *find_compiled(polar_code *c, bool is_i8, const LaunchShape &sh) {
    std::lock_guard<std::mutex> g(c->mu);
    auto it = c->compiled.find(CompiledKey{is_i8, sh.threads, sh.smem_stage_max,
                                           sh.warp_stage_max, sh.stage_channel,
                                           std::max<uint32_t>(sh.frames_per_cta, 1)});
    return it == c->compiled.end() ? nullptr : &it->second;
}

// The several-frames-per-CTA form of a throughput shape with one warp per
// frame, when the handle asks for it (polar_code_set_frames_per_cta): F warps,
// each with its own frame, shared-memory region and scratch; channel read in
// place. Returns false (sh untouched) when it does not apply.
bool multi_frame_shape(const polar_code *c, bool is_i8, size_t n_frames, int device,
                       LaunchShape *sh) {
    const uint32_t F = c->user[is_i8 ? 1 : 0].frames_per_cta;
    if (F <= 1 || sh->threads != 32) return false;
    if (n_frames * 2 <= static_cast<size_t>(device_props(device).sms)) return false;  // batch-1 shape
    const size_t per_frame =
        (kernel_smem_bytes(c->N, sh->smem_stage_max, 32, is_i8, false) + 127) / 128 * 128;
    if (per_frame * F > device_props(device).smem_optin) return false;
    sh->frames_per_cta = F;
    sh->threads = 32 * F;
    sh->stage_channel = 0;
    sh->smem_bytes = per_frame * F;
    return true;
}

// The specialised decoder for this decode, preferring the several-frames-per-CTA
// shape when one was compiled for it; *sh becomes the shape of what runs.
CompiledKernel *pick_compiled(polar_code *c, bool is_i8, size_t n_frames, int device,
                              LaunchShape *sh) {
    LaunchShape msh = *sh;
    if (multi_frame_shape(c, is_i8, n_frames, device, &msh)) {
        if (CompiledKernel *ck = find_compiled(c, is_i8, msh)) {
            *sh = msh;
            return ck;
        }
    }
    return find_compiled(c, is_i8, *sh);
}

int compiled_occupancy(polar_code *c, CompiledKernel *ck, int device, const LaunchShape &sh) {
    {
        std::lock_guard<std::mutex> g(c->mu);
        auto it = ck->occupancy.find(device);
        if (it != ck->occupancy.end()) return it->second;
    }
    const int n = compiled_max_ctas(ck, sh.threads, sh.smem_bytes);
    if (n <= 0) return 0;
    std::lock_guard<std::mutex> g(c->mu);
    ck->occupancy[device] = n;
    return n;
}

// Fill ctas_per_sm and grid from the resident-CTA count of the kernel used.
polar_status finish_grid(const polar_code *c, bool is_i8, size_t n_frames, int device, int occ,
                         LaunchShape *sh) {
    if (occ <= 0) return POLAR_EINVAL;
    const DeviceProps dp = device_props(device);
    const UserLaunch &u = c->user[is_i8 ? 1 : 0];
    const uint32_t cps = u.ctas_per_sm ? std::min<uint32_t>(u.ctas_per_sm, static_cast<uint32_t>(occ))
                                       : static_cast<uint32_t>(occ);
    const size_t F = std::max<uint32_t>(sh->frames_per_cta, 1);
    const size_t grid = std::min<size_t>((n_frames + F - 1) / F, size_t(dp.sms) * cps);
    sh->ctas_per_sm = cps;
    sh->grid = static_cast<uint32_t>(std::max<size_t>(grid, 1));
    return POLAR_OK;
}

polar_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return POLAR_OK;
    if (e == cudaErrorMemoryAllocation) return POLAR_ENOMEM;
    return POLAR_ECUDA;
}

polar_status decode_impl(const polar_code_t *code, const void *llr, bool is_i8,
                         uint8_t *bits_out, float *trace, size_t n_frames,
                         polar_stream_t stream) {
    if (!code) return POLAR_EINVAL;
    if (n_frames == 0) return POLAR_OK;
    if (!llr || (!bits_out && code->K > 0)) return POLAR_EINVAL;
    if (reinterpret_cast<uintptr_t>(llr) % 16 != 0) return POLAR_EALIGN;
    if (trace && code->trace_len == 0 && code->K == 0) return POLAR_OK;
    if (code->K == 0 && !trace) return POLAR_OK;  // nothing to write
    polar_code *c = const_cast<polar_code *>(code);
    int device = -1;
    if (cudaGetDevice(&device) != cudaSuccess) {
        cudaGetLastError();
        return POLAR_ECUDA;
    }
    LaunchShape sh{};
    polar_status st = choose_shape(c, is_i8, n_frames, device, &sh);
    if (st != POLAR_OK) return st;
    const LaunchShape sh1 = sh;  // one frame per CTA: what the interpreter runs
    CompiledKernel *ck = trace ? nullptr : pick_compiled(c, is_i8, n_frames, device, &sh);
    int occ = ck ? compiled_occupancy(c, ck, device, sh) : 0;
    if (occ <= 0) {  // no specialised decoder, or it cannot be resident: interpreter
        ck = nullptr;
        sh = sh1;
        occ = occupancy(device, is_i8, sh.stage_channel != 0, sh.threads, sh.smem_bytes);
    }
    st = finish_grid(c, is_i8, n_frames, device, occ, &sh);
    if (st != POLAR_OK) return st;
    DeviceState *ds = nullptr;
    st = ensure_device(c, device, &ds);
    if (st != POLAR_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);

    KernelArgs a{};
    const size_t nops = c->ops.size();
    a.ops = ds->tables;
    a.trace_offs = ds->tables + nops;
    a.ext_mask = ds->tables + 2 * nops;
    a.ext_pre = ds->tables + 2 * nops + c->NW;
    a.ext_wstart = ds->tables + 2 * nops + 2 * c->NW;
    a.status = ds->status;
    a.llr = llr;
    a.out = bits_out;
    a.trace = trace;
    a.n_frames = n_frames;
    a.trace_stride = c->trace_len;
    a.gstride = sh.scratch_elems_per_cta;
    a.n_ops = static_cast<uint32_t>(c->ops.size());
    a.N = c->N;
    a.log2N = c->log2N;
    a.K = c->K;
    a.S = sh.smem_stage_max;
    a.log2W = static_cast<uint32_t>(log2u(sh.warp_stage_max));
    a.NW = c->NW;
    a.KW = c->KW;
    a.out_row = (c->K + 7) / 8;

    void *scratch = nullptr;
    const size_t scratch_bytes = size_t(sh.grid) * std::max<uint32_t>(sh.frames_per_cta, 1) *
                                 sh.scratch_elems_per_cta * (is_i8 ? 1 : 4);
    if (scratch_bytes) {
        cudaError_t e = pool_alloc(&scratch, scratch_bytes, device, s);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return cuda_status(e);
        }
    }
    a.gscratch = scratch;
    cudaError_t e;
    if (ck) {
        e = launch_compiled(ck, sh, &a, s);
    } else {
        e = launch_decode(is_i8, trace != nullptr, sh.stage_channel != 0, sh, a, s);
    }
    if (scratch) cudaFreeAsync(scratch, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cuda_status(e);
    }
    return POLAR_OK;
}

}  // namespace

namespace polar {
polar_status code_device_state(polar_code *c, int device, DeviceState **out) {
    return ensure_device(c, device, out);
}

cudaMemPool_t device_pool(int device) {
    static std::mutex mu;
    static std::vector<cudaMemPool_t> pools(kMaxDevices, nullptr);
    static std::vector<bool> tried(kMaxDevices, false);
    if (device < 0 || static_cast<size_t>(device) >= kMaxDevices) return nullptr;
    std::lock_guard<std::mutex> g(mu);
    if (!tried[device]) {
        tried[device] = true;
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = device;
        cudaMemPool_t p = nullptr;
        if (cudaMemPoolCreate(&p, &props) == cudaSuccess) {
            uint64_t keep = ~0ull;  // never hand cached blocks back to the driver
            cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
            pools[device] = p;
        } else {
            cudaGetLastError();
        }
    }
    return pools[device];
}

cudaError_t pool_alloc(void **p, size_t bytes, int device, cudaStream_t s) {
    cudaMemPool_t pool = device_pool(device);
    return pool ? cudaMallocFromPoolAsync(p, bytes, pool, s) : cudaMallocAsync(p, bytes, s);
}
}  // namespace polar

extern "C" {

const char *polar_status_str(polar_status s) {
    switch (s) {
    case POLAR_OK: return "ok";
    case POLAR_EINVAL: return "invalid argument";
    case POLAR_ENOMEM: return "out of memory";
    case POLAR_ECUDA: return "CUDA error";
    case POLAR_EALIGN: return "LLR pointer not 16-byte aligned";
    case POLAR_ETIMEOUT: return "device wait timed out";
    }
    return "unknown status";
}

polar_status polar_code_create_ex(uint32_t N, uint32_t K, const uint8_t *frozen_mask,
                                  uint32_t max_rep, uint32_t max_spc, polar_code_t **out) {
    if (!out || !frozen_mask) return POLAR_EINVAL;
    if (N < 2 || N > kMaxN || !is_pow2(N) || K > N) return POLAR_EINVAL;
    uint32_t zeros = 0;
    for (uint32_t i = 0; i < N; ++i) {
        if (frozen_mask[i] > 1) return POLAR_EINVAL;
        zeros += frozen_mask[i] == 0;
    }
    if (zeros != K) return POLAR_EINVAL;
    polar_code *c = new (std::nothrow) polar_code;
    if (!c) return POLAR_ENOMEM;
    try {
        c->N = N;
        c->K = K;
        c->log2N = static_cast<uint32_t>(log2u(N));
        c->max_rep = max_rep;
        c->max_spc = max_spc;
        c->frozen.assign(frozen_mask, frozen_mask + N);
        c->build_tables();
    } catch (const std::bad_alloc &) {
        delete c;
        return POLAR_ENOMEM;
    }
    // Upload to the current device when one is present.
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) == cudaSuccess && ndev > 0) {
        int device = 0;
        DeviceState *ds = nullptr;
        if (cudaGetDevice(&device) != cudaSuccess) {
            delete c;
            return POLAR_ECUDA;
        }
        polar_status st = ensure_device(c, device, &ds);
        if (st != POLAR_OK) {
            delete c;
            return st;
        }
    } else {
        cudaGetLastError();
    }
    *out = c;
    return POLAR_OK;
}

polar_status polar_code_create(uint32_t N, uint32_t K, const uint8_t *frozen_mask,
                               polar_code_t **out) {
    return polar_code_create_ex(N, K, frozen_mask, UINT32_MAX, UINT32_MAX, out);
}

void polar_code_destroy(polar_code_t *code) { delete code; }

polar_status polar_code_info(const polar_code_t *code, uint32_t *N, uint32_t *K,
                             uint32_t *n_ops) {
    if (!code) return POLAR_EINVAL;
    if (N) *N = code->N;
    if (K) *K = code->K;
    if (n_ops) *n_ops = static_cast<uint32_t>(code->ops.size());
    return POLAR_OK;
}

polar_status polar_code_schedule(const polar_code_t *code, uint32_t *kind, uint32_t *nv,
                                 uint32_t *off, size_t capacity, size_t *n_ops) {
    if (!code) return POLAR_EINVAL;
    if (n_ops) *n_ops = code->ops.size();
    if (capacity < code->ops.size()) return POLAR_EINVAL;
    for (size_t i = 0; i < code->ops.size(); ++i) {
        if (kind) kind[i] = code->ops[i].kind;
        if (nv) nv[i] = 1u << code->ops[i].log2n;
        if (off) off[i] = code->ops[i].off;
    }
    return POLAR_OK;
}

size_t polar_code_trace_len(const polar_code_t *code) { return code ? code->trace_len : 0; }

// x = u F^{(x)n} on 64-bit words, bit i of the frame = bit (i % 64) of word i/64.
static void transform_words(uint64_t *w, uint32_t N) {
    static const uint64_t kMask[6] = {0x5555555555555555ull, 0x3333333333333333ull,
                                      0x0F0F0F0F0F0F0F0Full, 0x00FF00FF00FF00FFull,
                                      0x0000FFFF0000FFFFull, 0x00000000FFFFFFFFull};
    const uint32_t nw = N >= 64 ? N / 64 : 1;
    for (uint32_t h = 1, l = 0; h < 64 && h < N; h *= 2, ++l)
        for (uint32_t j = 0; j < nw; ++j) w[j] ^= (w[j] >> h) & kMask[l];
    for (uint32_t hw = 1; hw < nw; hw *= 2)
        for (uint32_t b = 0; b < nw; b += 2 * hw)
            for (uint32_t j = b; j < b + hw; ++j) w[j] ^= w[j + hw];
}

polar_status polar_encode_systematic(const polar_code_t *code, const uint8_t *info_packed,
                                     uint8_t *codeword_packed, size_t n_frames) {
    if (!code) return POLAR_EINVAL;
    if (n_frames == 0) return POLAR_OK;
    if ((!info_packed && code->K) || !codeword_packed) return POLAR_EINVAL;
    const uint32_t N = code->N, K = code->K;
    const uint32_t nw = N >= 64 ? N / 64 : 1;
    const size_t in_row = (K + 7) / 8, out_row = (N + 7) / 8;
    std::vector<uint64_t> info_words(nw, 0), w(nw);
    for (uint32_t i : code->info_idx) info_words[i >> 6] |= 1ull << (i & 63);
    for (size_t f = 0; f < n_frames; ++f) {
        const uint8_t *d = info_packed + f * in_row;
        std::fill(w.begin(), w.end(), 0ull);
        for (uint32_t k = 0; k < K; ++k)
            if ((d[k >> 3] >> (k & 7)) & 1u) {
                const uint32_t i = code->info_idx[k];
                w[i >> 6] |= 1ull << (i & 63);
            }
        transform_words(w.data(), N);
        for (uint32_t j = 0; j < nw; ++j) w[j] &= info_words[j];
        transform_words(w.data(), N);
        for (uint32_t k = 0; k < K; ++k) {
            const uint32_t i = code->info_idx[k];
            if (((w[i >> 6] >> (i & 63)) & 1ull) != ((d[k >> 3] >> (k & 7)) & 1u))
                return POLAR_EINVAL;
        }
        uint8_t *x = codeword_packed + f * out_row;
        for (size_t b = 0; b < out_row; ++b)
            x[b] = static_cast<uint8_t>((w[b >> 3] >> (8 * (b & 7))) & 0xFFu);
        if (N < 8) x[0] &= static_cast<uint8_t>((1u << N) - 1u);
    }
    return POLAR_OK;
}

polar_status polar_decode(const polar_code_t *code, const float *llr, uint8_t *bits_out,
                          size_t n_frames, polar_stream_t stream) {
    return decode_impl(code, llr, false, bits_out, nullptr, n_frames, stream);
}

polar_status polar_decode_noalloc(const polar_code_t *code, const float *llr, uint8_t *bits_out,
                                  size_t n_frames, polar_stream_t stream) {
    if (!code) return POLAR_EINVAL;
    if (n_frames == 0) return POLAR_OK;
    if (!llr || (!bits_out && code->K > 0)) return POLAR_EINVAL;
    if (reinterpret_cast<uintptr_t>(llr) % 16 != 0) return POLAR_EALIGN;
    if (code->K == 0) return POLAR_OK;
    polar_code *c = const_cast<polar_code *>(code);
    int device = -1;
    if (cudaGetDevice(&device) != cudaSuccess) {
        cudaGetLastError();
        return POLAR_ECUDA;
    }
    if (device < 0 || static_cast<size_t>(device) >= c->dev.size()) return POLAR_ECUDA;
    DeviceState *ds = nullptr;
    {
        // the per-device tables must already exist: uploading them would allocate
        std::lock_guard<std::mutex> g(c->mu);
        if (!c->dev[device].ready) return POLAR_EINVAL;
        ds = &c->dev[device];
    }
    LaunchShape sh{};
    polar_status st = choose_shape(c, false, n_frames, device, &sh);
    if (st != POLAR_OK) return st;
    st = finish_grid(c, false, n_frames, device,
                     occupancy(device, false, sh.stage_channel != 0, sh.threads, sh.smem_bytes), &sh);
    if (st != POLAR_OK) return st;
    void *scratch = nullptr;
    const size_t per_cta = sh.scratch_elems_per_cta * 4;
    if (per_cta) {
        if (per_cta > kNoAllocScratchBytes) return POLAR_EINVAL;  // one CTA needs more than the array
        sh.grid = static_cast<uint32_t>(std::min<size_t>(sh.grid, kNoAllocScratchBytes / per_cta));
        if (noalloc_scratch(&scratch) != cudaSuccess) {
            cudaGetLastError();
            return POLAR_ECUDA;
        }
    }
    const size_t nops = c->ops.size();
    KernelArgs a{};
    a.ops = ds->tables;
    a.trace_offs = ds->tables + nops;
    a.ext_mask = ds->tables + 2 * nops;
    a.ext_pre = ds->tables + 2 * nops + c->NW;
    a.ext_wstart = ds->tables + 2 * nops + 2 * c->NW;
    a.status = ds->status;
    a.llr = llr;
    a.out = bits_out;
    a.trace = nullptr;
    a.gscratch = scratch;
    a.n_frames = n_frames;
    a.trace_stride = c->trace_len;
    a.gstride = sh.scratch_elems_per_cta;
    a.n_ops = static_cast<uint32_t>(nops);
    a.N = c->N;
    a.log2N = c->log2N;
    a.K = c->K;
    a.S = sh.smem_stage_max;
    a.log2W = static_cast<uint32_t>(log2u(sh.warp_stage_max));
    a.NW = c->NW;
    a.KW = c->KW;
    a.out_row = (c->K + 7) / 8;
    const cudaError_t e = launch_decode(false, false, sh.stage_channel != 0, sh, a,
                                        reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cuda_status(e);
    }
    return POLAR_OK;
}

polar_status polar_decode_i8(const polar_code_t *code, const int8_t *llr, uint8_t *bits_out,
                             size_t n_frames, polar_stream_t stream) {
    return decode_impl(code, llr, true, bits_out, nullptr, n_frames, stream);
}

polar_status polar_decode_trace(const polar_code_t *code, const void *llr, int is_i8,
                                uint8_t *bits_out, float *alpha_trace, size_t n_frames,
                                polar_stream_t stream) {
    if (!code || (!alpha_trace && code->trace_len)) return POLAR_EINVAL;
    if (code->trace_len == 0 || !alpha_trace) {
        return decode_impl(code, llr, is_i8 != 0, bits_out, nullptr, n_frames, stream);
    }
    return decode_impl(code, llr, is_i8 != 0, bits_out, alpha_trace, n_frames, stream);
}

polar_status polar_code_set_launch(polar_code_t *code, int is_i8, uint32_t threads,
                                   uint32_t smem_stage_max, uint32_t warp_stage_max,
                                   uint32_t ctas_per_sm, uint32_t stage_channel) {
    if (!code) return POLAR_EINVAL;
    if (threads && (threads % 32 || threads > 1024)) return POLAR_EINVAL;
    if (smem_stage_max && (!is_pow2(smem_stage_max) || smem_stage_max < 64)) return POLAR_EINVAL;
    if (warp_stage_max && (!is_pow2(warp_stage_max) || warp_stage_max < 2)) return POLAR_EINVAL;
    if (stage_channel > 2) return POLAR_EINVAL;
    UserLaunch &u = code->user[is_i8 ? 1 : 0];
    u.threads = threads;
    u.smem_stage_max = smem_stage_max;
    u.warp_stage_max = warp_stage_max;
    u.ctas_per_sm = ctas_per_sm;
    u.stage_channel = stage_channel;
    return POLAR_OK;
}

polar_status polar_code_get_launch(const polar_code_t *code, int is_i8, size_t n_frames,
                                   uint32_t *threads, uint32_t *smem_stage_max,
                                   uint32_t *warp_stage_max, uint32_t *ctas_per_sm,
                                   uint32_t *stage_channel, uint32_t *grid, size_t *smem_bytes,
                                   size_t *scratch_bytes, uint32_t *unrolled) {
    if (!code) return POLAR_EINVAL;
    int device = -1;
    if (cudaGetDevice(&device) != cudaSuccess) {
        cudaGetLastError();
        return POLAR_ECUDA;
    }
    polar_code *c = const_cast<polar_code *>(code);
    const size_t n = std::max<size_t>(n_frames, 1);
    LaunchShape sh{};
    polar_status st = choose_shape(c, is_i8 != 0, n, device, &sh);
    if (st != POLAR_OK) return st;
    const LaunchShape sh1 = sh;
    CompiledKernel *ck = pick_compiled(c, is_i8 != 0, n, device, &sh);
    int occ = ck ? compiled_occupancy(c, ck, device, sh) : 0;
    if (occ <= 0) {
        ck = nullptr;
        sh = sh1;
        occ = occupancy(device, is_i8 != 0, sh.stage_channel != 0, sh.threads, sh.smem_bytes);
    }
    st = finish_grid(c, is_i8 != 0, n, device, occ, &sh);
    if (st != POLAR_OK) return st;
    if (threads) *threads = sh.threads;
    if (smem_stage_max) *smem_stage_max = sh.smem_stage_max;
    if (warp_stage_max) *warp_stage_max = sh.warp_stage_max;
    if (ctas_per_sm) *ctas_per_sm = sh.ctas_per_sm;
    if (stage_channel) *stage_channel = sh.stage_channel;
    if (grid) *grid = sh.grid;
    if (smem_bytes) *smem_bytes = sh.smem_bytes;
    if (scratch_bytes)
        *scratch_bytes = size_t(sh.grid) * std::max<uint32_t>(sh.frames_per_cta, 1) *
                         sh.scratch_elems_per_cta * (is_i8 ? 1 : 4);
    if (unrolled) *unrolled = ck ? ck->reg_subtree : 0u;
    return POLAR_OK;
}

polar_status polar_code_set_frames_per_cta(polar_code_t *code, int is_i8, uint32_t frames) {
    if (!code || frames > 8 || (frames > 1 && !is_pow2(frames))) return POLAR_EINVAL;
    std::lock_guard<std::mutex> g(code->mu);
    code->user[is_i8 ? 1 : 0].frames_per_cta = frames;
    return POLAR_OK;
}

polar_status polar_code_get_frames_per_cta(const polar_code_t *code, int is_i8, size_t n_frames,
                                           uint32_t *frames) {
    if (!code || !frames) return POLAR_EINVAL;
    int device = -1;
    if (cudaGetDevice(&device) != cudaSuccess) {
        cudaGetLastError();
        return POLAR_ECUDA;
    }
    polar_code *c = const_cast<polar_code *>(code);
    const size_t n = std::max<size_t>(n_frames, 1);
    LaunchShape sh{};
    const polar_status st = choose_shape(c, is_i8 != 0, n, device, &sh);
    if (st != POLAR_OK) return st;
    CompiledKernel *ck = pick_compiled(c, is_i8 != 0, n, device, &sh);
    *frames = ck ? std::max<uint32_t>(sh.frames_per_cta, 1) : 1u;
    return POLAR_OK;
}

polar_status polar_code_compile(polar_code_t *code, int is_i8, size_t n_frames,
                                uint32_t reg_subtree) {
    return polar_code_compile_ex(code, is_i8, n_frames, reg_subtree, 0);
}

polar_status polar_code_compile_ex(polar_code_t *code, int is_i8, size_t n_frames,
                                   uint32_t reg_subtree, uint32_t flags) {
    if (!code) return POLAR_EINVAL;
    if (flags & ~(POLAR_COMPILE_COMPACT | POLAR_COMPILE_FULL | POLAR_COMPILE_LOCAL_LEAVES) ||
        (flags & POLAR_COMPILE_COMPACT && flags & POLAR_COMPILE_FULL))
        return POLAR_EINVAL;
    const uint32_t form = flags & (POLAR_COMPILE_COMPACT | POLAR_COMPILE_FULL);
    uint32_t outline = flags & POLAR_COMPILE_COMPACT;  // subtrees (1) and/or memory ops (2)
    if (!form && code->ops.size() > kCompactOps) outline = kOutlineSubtrees | kOutlineMemory;
    if (flags & POLAR_COMPILE_LOCAL_LEAVES) outline |= kLocalLeaves;
    if (reg_subtree == 0) reg_subtree = 256;
    if (!is_pow2(reg_subtree) || reg_subtree < 32 || reg_subtree > 1024) return POLAR_EINVAL;
    int device = -1;
    if (cudaGetDevice(&device) != cudaSuccess) {
        cudaGetLastError();
        return POLAR_ECUDA;
    }
    if (n_frames == 0) {  // drop every specialised decoder of this LLR type
        std::lock_guard<std::mutex> g(code->mu);
        for (auto it = code->compiled.begin(); it != code->compiled.end();) {
            if (std::get<0>(it->first) == (is_i8 != 0)) {
                if (it->second.lib) cudaLibraryUnload(it->second.lib);
                it = code->compiled.erase(it);
            } else {
                ++it;
            }
        }
        return POLAR_OK;
    }
    LaunchShape sh{};
    polar_status st = choose_shape(code, is_i8 != 0, n_frames, device, &sh);
    if (st != POLAR_OK) return st;
    multi_frame_shape(code, is_i8 != 0, n_frames, device, &sh);
    const uint32_t F = std::max<uint32_t>(sh.frames_per_cta, 1);
    const CompiledKey key{is_i8 != 0, sh.threads, sh.smem_stage_max, sh.warp_stage_max,
                          sh.stage_channel, F};
    if (find_compiled(code, is_i8 != 0, sh)) return POLAR_OK;
    // register subtrees always run inside warp-0 runs
    LaunchShape gsh = sh;
    gsh.warp_stage_max = std::max(sh.warp_stage_max, reg_subtree);
    // resident CTAs the shared-memory footprint allows: the register budget of
    // the generated kernel is capped so that many fit
    const DeviceProps dp = device_props(device);
    const size_t per_cta = sh.smem_bytes + 1024;
    const size_t groups = (n_frames + F - 1) / F;
    gsh.ctas_per_sm = static_cast<uint32_t>(std::max<size_t>(
        1, std::min<size_t>({size_t(228 * 1024) / per_cta, size_t(2048 / sh.threads),
                             size_t(dp.max_blocks_per_sm),
                             size_t(groups + dp.sms - 1) / std::max(dp.sms, 1)})));
    if (code->user[is_i8 ? 1 : 0].ctas_per_sm)
        gsh.ctas_per_sm = std::min(gsh.ctas_per_sm, code->user[is_i8 ? 1 : 0].ctas_per_sm);
    CompiledKernel ck;
    ck.reg_subtree = reg_subtree;
    ck.outline = outline;
    std::string log;
    const std::string src = generate_source(*code, is_i8 != 0, gsh, reg_subtree, outline);
    const cudaError_t e = compile_source(src, &ck, &log);
    std::lock_guard<std::mutex> g(code->mu);
    code->compile_log = log;
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cuda_status(e);
    }
    code->compiled[key] = ck;
    return POLAR_OK;
}

const char *polar_code_compile_log(const polar_code_t *code) {
    return code ? code->compile_log.c_str() : "";
}

polar_status polar_selftest_bounded_wait(polar_code_t *code, uint32_t limit_us,
                                         polar_stream_t stream) {
    if (!code || limit_us == 0 || limit_us > 1000000) return POLAR_EINVAL;
    int device = -1;
    if (cudaGetDevice(&device) != cudaSuccess) {
        cudaGetLastError();
        return POLAR_ECUDA;
    }
    DeviceState *ds = nullptr;
    const polar_status st = ensure_device(code, device, &ds);
    if (st != POLAR_OK) return st;
    return cuda_status(launch_bounded_wait_selftest(
        ds->status, 1000ull * limit_us, reinterpret_cast<cudaStream_t>(stream)));
}

polar_status polar_code_check(polar_code_t *code, polar_stream_t stream) {
    if (!code) return POLAR_EINVAL;
    int device = -1;
    if (cudaGetDevice(&device) != cudaSuccess) {
        cudaGetLastError();
        return POLAR_ECUDA;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return POLAR_ECUDA;
    }
    std::lock_guard<std::mutex> g(code->mu);
    if (static_cast<size_t>(device) >= code->dev.size() || !code->dev[device].ready) return POLAR_OK;
    int v = 0;
    if (cudaMemcpy(&v, code->dev[device].status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return POLAR_ECUDA;
    if (v) {
        cudaMemset(code->dev[device].status, 0, sizeof(int));
        return POLAR_ETIMEOUT;
    }
    return POLAR_OK;
}

}  // extern "C"
