// Decoding from host memory: channel LLRs in host buffers in, information bits
// in host buffers out, with the copies overlapped with decoding. The frames are
// cut into chunks; chunk c goes to one of kDepth internal streams (copy in,
// decode, copy out), so while one chunk decodes the next is copied in and the
// previous one copied out. The device buffers for the chunks in flight belong
// to the device and are kept between calls (they only grow), so a call does no
// allocation once the buffers are large enough; calls on one device take turns.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "polar_gb300.h"
#include "polar_internal.h"

namespace {

constexpr int kDepth = 6;  // chunks in flight: buffers are reused only beyond this

// Per device: kDepth non-blocking streams and one device buffer pair per
// stream, created on first use and kept; `mu` is held for a whole call.
struct HostIo {
    std::mutex mu;
    cudaStream_t s[kDepth] = {};
    bool ok = false;
    void *in[kDepth] = {};
    uint8_t *out[kDepth] = {};
    size_t in_cap = 0, out_cap = 0;  // bytes of each in[k] / out[k]
};

HostIo &hostio_for(int device) {
    static std::vector<HostIo> per(polar::kMaxDevices);
    return per[static_cast<size_t>(device)];
}

// Make every buffer hold at least in_bytes / out_bytes (caller holds h.mu).
cudaError_t ensure_buffers(HostIo &h, size_t in_bytes, size_t out_bytes) {
    if (!h.ok) {
        bool ok = true;
        for (int k = 0; k < kDepth && ok; ++k)
            ok = cudaStreamCreateWithFlags(&h.s[k], cudaStreamNonBlocking) == cudaSuccess;
        if (!ok) return cudaErrorUnknown;
        h.ok = true;
    }
    if (in_bytes > h.in_cap) {
        for (int k = 0; k < kDepth; ++k) {
            if (h.in[k]) cudaFree(h.in[k]);
            h.in[k] = nullptr;
        }
        h.in_cap = 0;
        for (int k = 0; k < kDepth; ++k) {
            const cudaError_t e = cudaMalloc(&h.in[k], in_bytes);
            if (e != cudaSuccess) return e;
        }
        h.in_cap = in_bytes;
    }
    if (out_bytes > h.out_cap) {
        for (int k = 0; k < kDepth; ++k) {
            if (h.out[k]) cudaFree(h.out[k]);
            h.out[k] = nullptr;
        }
        h.out_cap = 0;
        for (int k = 0; k < kDepth; ++k) {
            const cudaError_t e = cudaMalloc(reinterpret_cast<void **>(&h.out[k]), out_bytes);
            if (e != cudaSuccess) return e;
        }
        h.out_cap = out_bytes;
    }
    return cudaSuccess;
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
    const size_t es = is_i8 ? 1 : 4, in_row = size_t(code->N) * es, out_row = (code->K + 7) / 8;
    if (chunk_frames == 0) chunk_frames = std::max<size_t>(1, (n_frames + 7) / 8);
    chunk_frames = std::min(chunk_frames, n_frames);
    const size_t n_chunks = (n_frames + chunk_frames - 1) / chunk_frames;
    const int depth = static_cast<int>(std::min<size_t>(kDepth, n_chunks));

    HostIo &hs = hostio_for(device);
    std::lock_guard<std::mutex> g(hs.mu);
    polar_status st = status_of(ensure_buffers(hs, chunk_frames * in_row, chunk_frames * out_row));
    const unsigned char *src = static_cast<const unsigned char *>(host_llr);
    for (size_t c = 0; c < n_chunks && st == POLAR_OK; ++c) {
        const int k = static_cast<int>(c % depth);
        cudaStream_t s = hs.s[k];
        const size_t f0 = c * chunk_frames, n = std::min(chunk_frames, n_frames - f0);
        st = status_of(cudaMemcpyAsync(hs.in[k], src + f0 * in_row, n * in_row,
                                       cudaMemcpyHostToDevice, s));
        if (st != POLAR_OK) break;
        const polar_stream_t ps = reinterpret_cast<polar_stream_t>(s);
        st = is_i8 ? polar_decode_i8(code, static_cast<const int8_t *>(hs.in[k]), hs.out[k], n, ps)
                   : polar_decode(code, static_cast<const float *>(hs.in[k]), hs.out[k], n, ps);
        if (st == POLAR_OK && out_row)
            st = status_of(cudaMemcpyAsync(host_bits + f0 * out_row, hs.out[k], n * out_row,
                                           cudaMemcpyDeviceToHost, s));
    }
    if (hs.ok) {
        for (int k = 0; k < depth; ++k) {
            const cudaError_t e = cudaStreamSynchronize(hs.s[k]);
            if (st == POLAR_OK) st = status_of(e);
        }
    }
    if (st == POLAR_OK) st = polar_code_check(const_cast<polar_code_t *>(code), nullptr);
    return st;
}

}  // extern "C"
