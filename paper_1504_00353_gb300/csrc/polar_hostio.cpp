// Decoding from host memory: channel LLRs in host buffers in, information bits
// in host buffers out, with the copies overlapped with decoding. The frames are
// cut into chunks; chunk c goes to one of kDepth internal streams (copy in,
// decode, copy out), so while one chunk decodes the next is copied in and the
// previous one copied out. Device buffers for the chunks in flight come from
// the library's stream-ordered pool (cached between calls).
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "polar_gb300.h"
#include "polar_internal.h"

namespace {

constexpr int kDepth = 6;  // chunks in flight: buffers are reused only beyond this

struct HostIoStreams {
    cudaStream_t s[kDepth] = {};
    bool ok = false;
};

// kDepth non-blocking streams per device, created on first use and kept.
const HostIoStreams &streams_for(int device) {
    static std::mutex mu;
    static std::vector<HostIoStreams> per(polar::kMaxDevices);
    std::lock_guard<std::mutex> g(mu);
    HostIoStreams &h = per[static_cast<size_t>(device)];
    if (!h.ok) {
        bool ok = true;
        for (int k = 0; k < kDepth && ok; ++k)
            ok = cudaStreamCreateWithFlags(&h.s[k], cudaStreamNonBlocking) == cudaSuccess;
        h.ok = ok;
    }
    return h;
}

polar_status status_of(cudaError_t e) {
    if (e == cudaSuccess) return POLAR_OK;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? POLAR_ENOMEM : POLAR_ECUDA;
}

}  // namespace

extern "C" {

polar_status polar_decode_host(const polar_code_t *code, int is_i8, const void *host_llr,
                               uint8_t *host_bits, size_t n_frames, size_t chunk_frames) {
    if (!code) return POLAR_EINVAL;
    if (n_frames == 0) return POLAR_OK;
    if (!host_llr || (!host_bits && code->K > 0)) return POLAR_EINVAL;
    int device = -1;
    if (cudaGetDevice(&device) != cudaSuccess || device < 0 ||
        static_cast<size_t>(device) >= polar::kMaxDevices) {
        cudaGetLastError();
        return POLAR_ECUDA;
    }
    const HostIoStreams &hs = streams_for(device);
    if (!hs.ok) return POLAR_ECUDA;
    const size_t es = is_i8 ? 1 : 4, in_row = size_t(code->N) * es, out_row = (code->K + 7) / 8;
    if (chunk_frames == 0) chunk_frames = std::max<size_t>(1, (n_frames + 7) / 8);
    chunk_frames = std::min(chunk_frames, n_frames);
    const size_t n_chunks = (n_frames + chunk_frames - 1) / chunk_frames;
    const int depth = static_cast<int>(std::min<size_t>(kDepth, n_chunks));

    // one device buffer pair per stream, reused by every chunk on that stream
    void *d_in[kDepth] = {};
    uint8_t *d_out[kDepth] = {};
    polar_status st = POLAR_OK;
    for (int k = 0; k < depth && st == POLAR_OK; ++k) {
        st = status_of(polar::pool_alloc(&d_in[k], chunk_frames * in_row, device, hs.s[k]));
        if (st == POLAR_OK && out_row)
            st = status_of(polar::pool_alloc(reinterpret_cast<void **>(&d_out[k]),
                                             chunk_frames * out_row, device, hs.s[k]));
    }
    const unsigned char *src = static_cast<const unsigned char *>(host_llr);
    for (size_t c = 0; c < n_chunks && st == POLAR_OK; ++c) {
        const int k = static_cast<int>(c % depth);
        cudaStream_t s = hs.s[k];
        const size_t f0 = c * chunk_frames, n = std::min(chunk_frames, n_frames - f0);
        st = status_of(cudaMemcpyAsync(d_in[k], src + f0 * in_row, n * in_row,
                                       cudaMemcpyHostToDevice, s));
        if (st != POLAR_OK) break;
        const polar_stream_t ps = reinterpret_cast<polar_stream_t>(s);
        st = is_i8 ? polar_decode_i8(code, static_cast<const int8_t *>(d_in[k]), d_out[k], n, ps)
                   : polar_decode(code, static_cast<const float *>(d_in[k]), d_out[k], n, ps);
        if (st == POLAR_OK && out_row)
            st = status_of(cudaMemcpyAsync(host_bits + f0 * out_row, d_out[k], n * out_row,
                                           cudaMemcpyDeviceToHost, s));
    }
    for (int k = 0; k < depth; ++k) {
        if (d_in[k]) cudaFreeAsync(d_in[k], hs.s[k]);
        if (d_out[k]) cudaFreeAsync(d_out[k], hs.s[k]);
    }
    for (int k = 0; k < depth; ++k) {
        const cudaError_t e = cudaStreamSynchronize(hs.s[k]);
        if (st == POLAR_OK) st = status_of(e);
    }
    if (st == POLAR_OK) st = polar_code_check(const_cast<polar_code_t *>(code), nullptr);
    return st;
}

}  // extern "C"
