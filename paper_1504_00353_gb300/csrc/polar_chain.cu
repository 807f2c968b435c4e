// Communication chain on the GPU around the decoder, for frame- and bit-error
// rates (the simulations behind the paper's error-rate figures, Sec. III):
// random information bits, the systematic encoder, BPSK over AWGN with
// float32 or int8 channel LLRs, and error counting.
//
// Random numbers come from Philox-4x32-10 (Salmon, Moraes, Dror, Shaw,
// "Parallel random numbers: as easy as 1, 2, 3", SC 2011), a counter-based
// generator: every output is a pure function of (key, counter), so any frame
// of any batch can be regenerated. Normals are Box-Muller pairs of its words.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <mutex>
#include <random>
#include <vector>

#include "polar_gb300.h"
#include "polar_internal.h"

using namespace polar;

namespace {

// ---------------------------------------------------------------- Philox-4x32-10

struct U4 {
    uint32_t x, y, z, w;
};

// One round: two 32x32 -> 64-bit products, their halves mixed with the key.
__host__ __device__ inline void philox_round(U4 &c, uint32_t k0, uint32_t k1) {
    const uint64_t p0 = uint64_t(0xD2511F53u) * c.x;
    const uint64_t p1 = uint64_t(0xCD9E8D57u) * c.z;
    const uint32_t hi0 = uint32_t(p0 >> 32), lo0 = uint32_t(p0);
    const uint32_t hi1 = uint32_t(p1 >> 32), lo1 = uint32_t(p1);
    c = U4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
}

// Ten rounds, the key bumped by the Weyl constants between rounds.
__host__ __device__ inline U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1) {
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        philox_round(c, k0, k1);
    }
    return c;
}

// Counter layout: (word index, frame low, frame high, stream).
constexpr uint32_t kStreamInfo = 1u, kStreamNoise = 2u;

__device__ inline U4 draw(uint64_t seed, uint32_t stream, uint64_t frame, uint32_t j) {
    return philox4x32_10(U4{j, uint32_t(frame), uint32_t(frame >> 32), stream}, uint32_t(seed),
                         uint32_t(seed >> 32));
}

// ---------------------------------------------------------------- kernels

// Information bits: row f of `info` (ceil(K/8) bytes) from Philox words; bits
// at and beyond K are zero.
__global__ void random_info_kernel(uint8_t *info, uint32_t K, size_t n_frames, uint64_t seed,
                                   uint64_t frame0) {
    const uint32_t row = (K + 7) / 8, words = (row + 15) / 16;
    const size_t total = n_frames * words;
    for (size_t t = blockIdx.x * size_t(blockDim.x) + threadIdx.x; t < total;
         t += size_t(gridDim.x) * blockDim.x) {
        const size_t f = t / words;
        const uint32_t j = static_cast<uint32_t>(t % words);
        const U4 r = draw(seed, kStreamInfo, frame0 + f, j);
        const uint32_t v[4] = {r.x, r.y, r.z, r.w};
        uint8_t *dst = info + f * row;
        for (uint32_t b = 0; b < 16; ++b) {
            const uint32_t byte = 16 * j + b;
            if (byte >= row) break;
            uint8_t x = static_cast<uint8_t>(v[b >> 2] >> (8 * (b & 3)));
            if (8 * byte + 8 > K) x &= static_cast<uint8_t>((1u << (K - 8 * byte)) - 1u);
            dst[byte] = x;
        }
    }
}

// Bit k of a packed LSB-first byte row.
__device__ inline uint32_t bits32(const uint8_t *row, uint32_t row_bytes, uint32_t k) {
    uint64_t v = 0;
    const uint32_t b0 = k >> 3;
    for (uint32_t b = 0; b < 5; ++b)
        if (b0 + b < row_bytes) v |= uint64_t(row[b0 + b]) << (8 * b);
    return static_cast<uint32_t>(v >> (k & 7));
}

// Scatter the low bits of v onto the set bits of m, lowest first.
__device__ inline uint32_t deposit(uint32_t v, uint32_t m) {
    uint32_t r = 0;
    while (m) {
        const uint32_t b = m & (0u - m);
        if (v & 1u) r |= b;
        v >>= 1;
        m &= m - 1u;
    }
    return r;
}

// x <- x F^{(x)n} on the frame's words in shared memory (bit i of the frame is
// bit i % 32 of word i / 32): x[i] ^= x[i + h] where bit h of i is clear, for
// every h < N (the stages commute).
__device__ void transform_smem(uint32_t *x, uint32_t N, uint32_t nw) {
    const uint32_t M[5] = {0x55555555u, 0x33333333u, 0x0F0F0F0Fu, 0x00FF00FFu, 0x0000FFFFu};
    for (uint32_t w = threadIdx.x; w < nw; w += blockDim.x) {
        uint32_t v = x[w];
        for (uint32_t l = 0, h = 1; l < 5 && h < N; ++l, h *= 2) v ^= (v >> h) & M[l];
        x[w] = v;
    }
    __syncthreads();
    for (uint32_t H = 1; H < nw; H *= 2) {
        for (uint32_t q = threadIdx.x; q < nw; q += blockDim.x)
            if (!(q & H)) x[q] ^= x[q + H];
        __syncthreads();
    }
}

// Systematic encoding (two transforms with the frozen positions cleared in
// between): info bits to the information set, transform, clear the frozen
// set, transform. One CTA per frame; the frame's N bits in shared memory.
__global__ void encode_kernel(const uint8_t *info, uint8_t *cw, const uint32_t *ext_mask,
                              const uint32_t *ext_pre, uint32_t N, uint32_t K, size_t n_frames) {
    extern __shared__ uint32_t xs[];
    const uint32_t nw = N >= 32 ? N / 32 : 1, in_row = (K + 7) / 8, out_row = (N + 7) / 8;
    for (size_t f = blockIdx.x; f < n_frames; f += gridDim.x) {
        const uint8_t *d = info + f * in_row;
        for (uint32_t w = threadIdx.x; w < nw; w += blockDim.x) {
            const uint32_t m = ext_mask[w];
            xs[w] = m ? deposit(bits32(d, in_row, ext_pre[w]), m) : 0u;
        }
        __syncthreads();
        transform_smem(xs, N, nw);
        for (uint32_t w = threadIdx.x; w < nw; w += blockDim.x) xs[w] &= ext_mask[w];
        __syncthreads();
        transform_smem(xs, N, nw);
        uint8_t *o = cw + f * out_row;
        for (uint32_t b = threadIdx.x; b < out_row; b += blockDim.x) {
            uint8_t v = static_cast<uint8_t>(xs[b >> 2] >> (8 * (b & 3)));
            if (N < 8) v &= static_cast<uint8_t>((1u << N) - 1u);
            o[b] = v;
        }
        __syncthreads();
    }
}

// BPSK (bit 0 -> +1) over AWGN: y = s + sigma n, LLR = 2 y / sigma^2 in
// float32, or q = clamp(rint(8 LLR), -127, 127) for int8. Four elements per
// Philox draw (two Box-Muller pairs).
template <typename T>
__global__ void awgn_kernel(const uint8_t *cw, T *llr, uint32_t N, size_t n_frames, float sigma,
                            float scale, uint64_t seed, uint64_t frame0) {
    const uint32_t quads = (N + 3) / 4, row = (N + 7) / 8;
    const size_t total = n_frames * quads;
    for (size_t t = blockIdx.x * size_t(blockDim.x) + threadIdx.x; t < total;
         t += size_t(gridDim.x) * blockDim.x) {
        const size_t f = t / quads;
        const uint32_t j = static_cast<uint32_t>(t % quads);
        const U4 r = draw(seed, kStreamNoise, frame0 + f, j);
        const float u1a = (float(r.x) + 1.0f) * 2.3283064365386963e-10f;  // (0, 1]
        const float u1b = (float(r.z) + 1.0f) * 2.3283064365386963e-10f;
        const float ra = sqrtf(-2.0f * logf(u1a)), rb = sqrtf(-2.0f * logf(u1b));
        float sa, ca, sb, cb;
        sincospif(2.0f * (float(r.y) * 2.3283064365386963e-10f), &sa, &ca);
        sincospif(2.0f * (float(r.w) * 2.3283064365386963e-10f), &sb, &cb);
        const float nz[4] = {ra * ca, ra * sa, rb * cb, rb * sb};
        const uint8_t *x = cw + f * row;
        T *out = llr + f * size_t(N);
        for (uint32_t e = 0; e < 4; ++e) {
            const uint32_t i = 4 * j + e;
            if (i >= N) break;
            const float s = ((x[i >> 3] >> (i & 7)) & 1u) ? -1.0f : 1.0f;
            const float l = scale * (s + sigma * nz[e]);
            if constexpr (sizeof(T) == 1) {
                out[i] = static_cast<T>(fminf(fmaxf(rintf(8.0f * l), -127.0f), 127.0f));
            } else {
                out[i] = l;
            }
        }
    }
}

// Frame and bit errors between two packed rows per frame: counters[0] +=
// frames that differ, counters[1] += differing bits.
__global__ void count_errors_kernel(const uint8_t *a, const uint8_t *b, uint32_t row,
                                    size_t n_frames, unsigned long long *counters) {
    unsigned long long fe = 0, be = 0;
    for (size_t f = blockIdx.x * size_t(blockDim.x) + threadIdx.x; f < n_frames;
         f += size_t(gridDim.x) * blockDim.x) {
        uint32_t bits = 0;
        for (uint32_t k = 0; k < row; ++k) bits += __popc(uint32_t(a[f * row + k] ^ b[f * row + k]));
        fe += bits ? 1u : 0u;
        be += bits;
    }
    if (fe) atomicAdd(&counters[0], fe);
    if (be) atomicAdd(&counters[1], be);
}

// ---------------------------------------------------------------- host helpers

polar_status status_of(cudaError_t e) {
    if (e == cudaSuccess) return POLAR_OK;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? POLAR_ENOMEM : POLAR_ECUDA;
}

int grid_for(size_t work, uint32_t threads) {
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t g = (work + threads - 1) / threads;
    return static_cast<int>(std::max<size_t>(1, std::min<size_t>(g, size_t(std::max(sms, 1)) * 16)));
}

// Whether the two-step encoder reproduces the information bits for this frozen
// set (checked once per handle on random words, on the host): true for the
// domination-contiguous sets polar constructions give.
bool systematic_ok(polar_code *c) {
    std::lock_guard<std::mutex> g(c->mu);
    if (c->systematic_checked) return c->systematic_valid;
    const uint32_t K = c->K;
    const size_t row = (K + 7) / 8;
    std::mt19937_64 rng(0x5eedu);
    bool ok = true;
    std::vector<uint8_t> d(row), x((c->N + 7) / 8);
    for (int t = 0; t < 16 && ok && K; ++t) {
        for (auto &b : d) b = static_cast<uint8_t>(rng());
        if (K % 8) d[row - 1] &= static_cast<uint8_t>((1u << (K % 8)) - 1u);
        ok = polar_encode_systematic(c, d.data(), x.data(), 1) == POLAR_OK;
    }
    c->systematic_checked = true;
    c->systematic_valid = ok;
    return ok;
}

}  // namespace

extern "C" {

polar_status polar_random_info(const polar_code_t *code, uint8_t *info_packed, size_t n_frames,
                               uint64_t seed, uint64_t frame0, polar_stream_t stream) {
    if (!code) return POLAR_EINVAL;
    if (n_frames == 0 || code->K == 0) return POLAR_OK;
    if (!info_packed) return POLAR_EINVAL;
    const uint32_t words = ((code->K + 7) / 8 + 15) / 16;
    random_info_kernel<<<grid_for(n_frames * words, 256), 256, 0,
                         reinterpret_cast<cudaStream_t>(stream)>>>(info_packed, code->K, n_frames,
                                                                   seed, frame0);
    return status_of(cudaGetLastError());
}

polar_status polar_encode_systematic_device(const polar_code_t *code, const uint8_t *info_packed,
                                            uint8_t *codeword_packed, size_t n_frames,
                                            polar_stream_t stream) {
    if (!code) return POLAR_EINVAL;
    if (n_frames == 0) return POLAR_OK;
    if ((!info_packed && code->K) || !codeword_packed) return POLAR_EINVAL;
    polar_code *c = const_cast<polar_code *>(code);
    if (!systematic_ok(c)) return POLAR_EINVAL;
    int device = -1;
    if (cudaGetDevice(&device) != cudaSuccess) return status_of(cudaErrorNoDevice);
    DeviceState *ds = nullptr;
    const polar_status st = code_device_state(c, device, &ds);
    if (st != POLAR_OK) return st;
    const size_t nops = c->ops.size();
    const uint32_t nw = c->N >= 32 ? c->N / 32 : 1;
    const size_t smem = nw * sizeof(uint32_t);  // the frame's N bits: 128 KB at N = 2^20
    if (smem > 48 * 1024) {
        static std::mutex mu;
        static size_t raised[64] = {};
        std::lock_guard<std::mutex> g(mu);
        if (device < 64 && raised[device] < smem) {
            const cudaError_t e = cudaFuncSetAttribute(
                encode_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
            if (e != cudaSuccess) return status_of(e);
            raised[device] = smem;
        }
    }
    const int grid = static_cast<int>(std::min<size_t>(n_frames, 152 * 8));
    encode_kernel<<<grid, 256, smem, reinterpret_cast<cudaStream_t>(stream)>>>(
        info_packed, codeword_packed, ds->tables + 2 * nops, ds->tables + 2 * nops + c->NW, c->N,
        c->K, n_frames);
    return status_of(cudaGetLastError());
}

polar_status polar_channel_awgn(const polar_code_t *code, const uint8_t *codeword_packed,
                                void *llr, int is_i8, size_t n_frames, float ebn0_db,
                                uint64_t seed, uint64_t frame0, polar_stream_t stream) {
    if (!code) return POLAR_EINVAL;
    if (n_frames == 0) return POLAR_OK;
    if (!codeword_packed || !llr || code->K == 0) return POLAR_EINVAL;
    const double rate = double(code->K) / code->N;
    const double s2 = 1.0 / (2.0 * rate * std::pow(10.0, ebn0_db / 10.0));
    const float sigma = static_cast<float>(std::sqrt(s2)), scale = static_cast<float>(2.0 / s2);
    const uint32_t quads = (code->N + 3) / 4;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int grid = grid_for(n_frames * quads, 256);
    if (is_i8)
        awgn_kernel<int8_t><<<grid, 256, 0, s>>>(codeword_packed, static_cast<int8_t *>(llr),
                                                 code->N, n_frames, sigma, scale, seed, frame0);
    else
        awgn_kernel<float><<<grid, 256, 0, s>>>(codeword_packed, static_cast<float *>(llr),
                                                code->N, n_frames, sigma, scale, seed, frame0);
    return status_of(cudaGetLastError());
}

polar_status polar_count_errors(const polar_code_t *code, const uint8_t *decoded,
                                const uint8_t *sent, size_t n_frames,
                                unsigned long long *counters, polar_stream_t stream) {
    if (!code || !counters) return POLAR_EINVAL;
    if (n_frames == 0 || code->K == 0) return POLAR_OK;
    if (!decoded || !sent) return POLAR_EINVAL;
    count_errors_kernel<<<grid_for(n_frames, 128), 128, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        decoded, sent, (code->K + 7) / 8, n_frames, counters);
    return status_of(cudaGetLastError());
}

polar_status polar_fer_run(const polar_code_t *code, int is_i8, float ebn0_db, uint64_t seed,
                           size_t n_frames, size_t batch, uint64_t *frame_errors,
                           uint64_t *bit_errors) {
    if (!code || !frame_errors || !bit_errors || code->K == 0) return POLAR_EINVAL;
    *frame_errors = *bit_errors = 0;
    if (n_frames == 0) return POLAR_OK;
    if (batch == 0) batch = 16384;
    batch = std::min(batch, n_frames);
    const size_t in_row = (code->K + 7) / 8, cw_row = (code->N + 7) / 8;
    const size_t es = is_i8 ? 1 : 4;
    uint8_t *d = nullptr, *x = nullptr, *out = nullptr;
    void *llr = nullptr;
    unsigned long long *cnt = nullptr;
    cudaStream_t s = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&d, batch * in_row);
    if (e == cudaSuccess) e = cudaMalloc(&x, batch * cw_row);
    if (e == cudaSuccess) e = cudaMalloc(&out, batch * in_row);
    if (e == cudaSuccess) e = cudaMalloc(&llr, batch * code->N * es);
    if (e == cudaSuccess) e = cudaMalloc(&cnt, 2 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, 2 * sizeof(unsigned long long), s);
    polar_status st = status_of(e);
    const polar_stream_t ps = reinterpret_cast<polar_stream_t>(s);
    for (size_t f0 = 0; f0 < n_frames && st == POLAR_OK; f0 += batch) {
        const size_t n = std::min(batch, n_frames - f0);
        st = polar_random_info(code, d, n, seed, f0, ps);
        if (st == POLAR_OK) st = polar_encode_systematic_device(code, d, x, n, ps);
        if (st == POLAR_OK) st = polar_channel_awgn(code, x, llr, is_i8, n, ebn0_db, seed, f0, ps);
        if (st == POLAR_OK)
            st = is_i8 ? polar_decode_i8(code, static_cast<const int8_t *>(llr), out, n, ps)
                       : polar_decode(code, static_cast<const float *>(llr), out, n, ps);
        if (st == POLAR_OK) st = polar_count_errors(code, out, d, n, cnt, ps);
    }
    unsigned long long h[2] = {0, 0};
    if (st == POLAR_OK) st = status_of(cudaMemcpyAsync(h, cnt, sizeof h, cudaMemcpyDeviceToHost, s));
    if (s) {
        const cudaError_t e2 = cudaStreamSynchronize(s);
        if (st == POLAR_OK) st = status_of(e2);
    }
    if (st == POLAR_OK) st = polar_code_check(const_cast<polar_code_t *>(code), ps);
    *frame_errors = h[0];
    *bit_errors = h[1];
    cudaFree(d);
    cudaFree(x);
    cudaFree(out);
    cudaFree(llr);
    cudaFree(cnt);
    if (s) cudaStreamDestroy(s);
    return st;
}

}  // extern "C"
