// Serving loop: continuous batching of decode requests onto the mixed-batch
// decoder (polar_batch.cpp).
//
// Requests are descriptors in a caller-owned circular array; each names a
// code and the place of its channel LLRs and of its output bytes in two
// caller-owned buffers: pinned host memory (asynchronous copies over the
// host link) or device memory (the copies stay in HBM). The
// caller publishes requests by advancing a count. One host thread runs the
// loop: whenever a launch slot is free and published requests wait, it admits
// as many as fit in the device LLR and output rings (the memory budget) and in
// one launch, copies their LLRs to the device (consecutive requests whose
// host data is contiguous in one copy), decodes them with one launch of the
// batch decoder (longest codes first), copies the bits back and records an
// event. Slots have their own stream, work counter and alpha scratch, so
// launches admitted while others run overlap on the GPU (copies of one with
// the decode of another, and the tail of one kernel with the next). A launch's
// requests get their completion time stamp as soon as it is seen finished;
// launches are retired (ring space and slot released, requests counted
// complete) in admission order.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <deque>
#include <new>
#include <numeric>
#include <thread>
#include <vector>

#include "polar_gb300.h"
#include "polar_internal.h"
#include "polar_ring.h"

using namespace polar;

namespace {

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    unsigned int *counter = nullptr;
    void *scratch = nullptr;
    unsigned char *d_desc = nullptr;  // llr_off[n] | out_off[n] | code_id[n]
    unsigned char *h_desc = nullptr;  // pinned staging of the same
    uint64_t first = 0, count = 0;    // requests [first, first + count)
    bool finished = false;            // its event completed; not yet retired
};

inline uint64_t now_ns() {
    return static_cast<uint64_t>(std::chrono::duration_cast<std::chrono::nanoseconds>(
                                     std::chrono::steady_clock::now().time_since_epoch())
                                     .count());
}

inline size_t round16(size_t v) { return (v + 15) / 16 * 16; }

}  // namespace

struct polar_server {
    polar_batch *batch = nullptr;
    const polar_request *reqs = nullptr;
    size_t capacity = 0;
    const unsigned char *h_llr = nullptr;
    size_t h_llr_bytes = 0;
    uint8_t *h_out = nullptr;
    size_t h_out_bytes = 0;
    uint64_t *done_ns = nullptr;
    uint32_t max_frames = 0;
    size_t es = 4;
    std::vector<uint32_t> code_N, code_K;

    unsigned char *d_llr = nullptr;
    uint8_t *d_out = nullptr;
    polar::Ring llr_ring, out_ring;
    std::vector<Slot> slots;
    std::vector<int> free_slots;
    std::deque<int> inflight;
    std::vector<uint32_t> order;  // scratch of the dispatcher

    uint64_t admitted = 0;  // dispatcher thread only
    uint32_t flags = 0;
    std::atomic<uint64_t> published{0}, completed{0}, launches{0}, admissions{0};
    std::atomic<int> error{POLAR_OK};
    std::atomic<bool> stop{false};
    std::thread thread;

    size_t llr_bytes(uint32_t c) const { return round16(size_t(code_N[c]) * es); }
    size_t out_bytes(uint32_t c) const { return (code_K[c] + 7) / 8; }

    void fail(polar_status s) {
        int ok = POLAR_OK;
        error.compare_exchange_strong(ok, s);
    }

    // Stamp every in-flight launch that has finished (its requests' completion
    // time is when it is seen finished, whatever launches are older), then
    // retire finished launches from the oldest on: release their ring space and
    // slot, and count their requests complete.
    bool retire() {
        bool any = false;
        for (const int k : inflight) {
            Slot &s = slots[k];
            if (s.finished) continue;
            const cudaError_t q = cudaEventQuery(s.done);
            if (q == cudaErrorNotReady) continue;
            if (q != cudaSuccess) {
                cudaGetLastError();
                fail(POLAR_ECUDA);
            }
            const uint64_t t = now_ns();
            for (uint64_t i = s.first; i < s.first + s.count; ++i) done_ns[i % capacity] = t;
            s.finished = true;
            any = true;
        }
        while (!inflight.empty() && slots[inflight.front()].finished) {
            const int k = inflight.front();
            Slot &s = slots[k];
            completed.store(s.first + s.count, std::memory_order_release);
            llr_ring.release_oldest();
            out_ring.release_oldest();
            inflight.pop_front();
            s.finished = false;
            free_slots.push_back(k);
            any = true;
        }
        return any;
    }

    // Admit waiting requests into one launch if a slot and ring space are free.
    bool admit() {
        if (free_slots.empty() || error.load() != POLAR_OK) return false;
        const uint64_t pub = published.load(std::memory_order_acquire);
        if (admitted == pub) return false;
        const size_t a_llr = llr_ring.avail(), a_out = out_ring.avail();
        size_t n = 0, bl = 0, bo = 0;
        for (uint64_t i = admitted; i < pub && n < max_frames; ++i, ++n) {
            const uint32_t c = reqs[i % capacity].code_id;
            if (bl + llr_bytes(c) > a_llr || bo + out_bytes(c) > a_out) break;
            bl += llr_bytes(c);
            bo += out_bytes(c);
        }
        if (n == 0) return false;  // waits for ring space
        const int k = free_slots.back();
        free_slots.pop_back();
        Slot &s = slots[k];
        s.first = admitted;
        s.count = n;
        const polar::Ring::Range rl = llr_ring.alloc(bl), ro = out_ring.alloc(bo);

        // descriptors, longest codes first (stable: arrival order among equals)
        order.resize(n);
        std::iota(order.begin(), order.end(), 0u);
        std::stable_sort(order.begin(), order.end(), [&](uint32_t x, uint32_t y) {
            const uint32_t cx = reqs[(s.first + x) % capacity].code_id;
            const uint32_t cy = reqs[(s.first + y) % capacity].code_id;
            return code_N[cx] != code_N[cy] ? code_N[cx] > code_N[cy] : cx < cy;
        });
        std::vector<uint64_t> dl(n), dout(n);
        size_t pl = rl.lo, po = ro.lo;
        for (size_t j = 0; j < n; ++j) {
            const uint32_t c = reqs[(s.first + j) % capacity].code_id;
            dl[j] = pl / es;
            dout[j] = po;
            pl += llr_bytes(c);
            po += out_bytes(c);
        }
        uint64_t *h_lo = reinterpret_cast<uint64_t *>(s.h_desc);
        uint64_t *h_oo = h_lo + n;
        uint32_t *h_id = reinterpret_cast<uint32_t *>(h_oo + n);
        for (size_t j = 0; j < n; ++j) {
            const uint32_t r = order[j];
            h_lo[j] = dl[r];
            h_oo[j] = dout[r];
            h_id[j] = reqs[(s.first + r) % capacity].code_id;
        }
        cudaError_t e = cudaMemcpyAsync(s.d_desc, s.h_desc, n * 20, cudaMemcpyHostToDevice, s.stream);
        // LLRs in: one copy per run of requests contiguous in host memory
        for (size_t j = 0; j < n && e == cudaSuccess;) {
            const polar_request &r0 = reqs[(s.first + j) % capacity];
            size_t len = llr_bytes(r0.code_id), m = j + 1;
            while (m < n) {
                const polar_request &r = reqs[(s.first + m) % capacity];
                if (r.llr_off != r0.llr_off + len) break;
                len += llr_bytes(r.code_id);
                ++m;
            }
            // the last request of a run may end short of its 16-byte rounding
            const polar_request &rl_last = reqs[(s.first + m - 1) % capacity];
            const size_t tail_pad = llr_bytes(rl_last.code_id) - size_t(code_N[rl_last.code_id]) * es;
            e = cudaMemcpyAsync(d_llr + dl[j] * es, h_llr + r0.llr_off, len - tail_pad,
                                cudaMemcpyDefault, s.stream);
            j = m;
        }
        // one launch over the admitted frames, or (per-code policy) one launch
        // per run of equal codes in the sorted list, one after another
        const uint64_t *d_lo = reinterpret_cast<const uint64_t *>(s.d_desc);
        const uint32_t *d_id = reinterpret_cast<const uint32_t *>(d_lo + 2 * n);
        for (size_t j = 0; j < n && e == cudaSuccess;) {
            size_t m = n;
            if (flags & POLAR_SERVE_LAUNCH_PER_CODE) {
                m = j + 1;
                while (m < n && h_id[m] == h_id[j]) ++m;
            }
            e = batch_launch(batch, d_id + j, d_lo + j, d_lo + n + j, d_llr, d_out, m - j,
                             s.counter, s.scratch, s.stream);
            launches.fetch_add(1, std::memory_order_relaxed);
            j = m;
        }
        // bits out: one copy per run contiguous in host memory
        for (size_t j = 0; j < n && e == cudaSuccess;) {
            const polar_request &r0 = reqs[(s.first + j) % capacity];
            size_t len = out_bytes(r0.code_id), m = j + 1;
            while (m < n) {
                const polar_request &r = reqs[(s.first + m) % capacity];
                if (r.out_off != r0.out_off + len) break;
                len += out_bytes(r.code_id);
                ++m;
            }
            e = cudaMemcpyAsync(h_out + r0.out_off, d_out + dout[j], len, cudaMemcpyDefault,
                                s.stream);
            j = m;
        }
        if (e == cudaSuccess) e = cudaEventRecord(s.done, s.stream);
        if (e != cudaSuccess) {
            cudaGetLastError();
            fail(POLAR_ECUDA);
        }
        admitted += n;
        admissions.fetch_add(1, std::memory_order_relaxed);
        inflight.push_back(k);
        return true;
    }

    void run() {
        cudaSetDevice(batch->device);
        for (;;) {
            bool worked = retire();
            worked = admit() || worked;
            if (inflight.empty() &&
                (error.load() != POLAR_OK ||
                 (stop.load() && admitted == published.load(std::memory_order_acquire))))
                break;
            if (!worked) std::this_thread::yield();
        }
    }

    void release() {
        for (Slot &s : slots) {
            if (s.done) cudaEventDestroy(s.done);
            if (s.stream) cudaStreamDestroy(s.stream);
            cudaFree(s.counter);
            cudaFree(s.scratch);
            cudaFree(s.d_desc);
            cudaFreeHost(s.h_desc);
        }
        slots.clear();
        cudaFree(d_llr);
        cudaFree(d_out);
        d_llr = nullptr;
        d_out = nullptr;
    }
};

extern "C" {

polar_status polar_server_create(polar_batch_t *batch, const polar_request *reqs, size_t capacity,
                                 const void *host_llr, size_t host_llr_bytes, uint8_t *host_out,
                                 size_t host_out_bytes, uint64_t *done_ns,
                                 size_t device_budget_bytes, uint32_t max_frames, uint32_t slots,
                                 uint32_t flags, polar_server_t **out) {
    if (!batch || !reqs || capacity == 0 || !host_llr || !host_out || !done_ns || !out ||
        max_frames == 0 || slots == 0 || slots > 64 || (flags & ~POLAR_SERVE_LAUNCH_PER_CODE))
        return POLAR_EINVAL;
    int device = -1;
    if (cudaGetDevice(&device) != cudaSuccess || device != batch->device) {
        cudaGetLastError();
        return POLAR_ECUDA;
    }
    polar_server *s = new (std::nothrow) polar_server;
    if (!s) return POLAR_ENOMEM;
    s->batch = batch;
    s->reqs = reqs;
    s->capacity = capacity;
    s->h_llr = static_cast<const unsigned char *>(host_llr);
    s->h_llr_bytes = host_llr_bytes;
    s->h_out = host_out;
    s->h_out_bytes = host_out_bytes;
    s->done_ns = done_ns;
    s->max_frames = max_frames;
    s->flags = flags;
    s->es = batch->elem_bytes();
    size_t max_llr = 0, max_out = 0;
    for (polar_code *c : batch->codes) {
        s->code_N.push_back(c->N);
        s->code_K.push_back(c->K);
        max_llr = std::max(max_llr, round16(size_t(c->N) * s->es));
        max_out = std::max<size_t>(max_out, (c->K + 7) / 8);
    }
    // the budget holds both rings; output bytes per frame are at most 1/(8 es)
    // of its LLR bytes
    s->out_ring.cap = round16(device_budget_bytes / (8 * s->es + 1) + max_out);
    s->llr_ring.cap = device_budget_bytes > s->out_ring.cap
                          ? (device_budget_bytes - s->out_ring.cap) / 16 * 16 : 0;
    if (s->llr_ring.cap < max_llr) {  // a frame of the longest code must fit
        delete s;
        return POLAR_EINVAL;
    }
    cudaError_t e = cudaMalloc(&s->d_llr, s->llr_ring.cap);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_out, s->out_ring.cap);
    s->slots.resize(slots);
    const size_t desc_bytes = size_t(max_frames) * 20;
    const size_t scratch = batch->scratch_bytes(max_frames);
    for (uint32_t k = 0; k < slots && e == cudaSuccess; ++k) {
        Slot &sl = s->slots[k];
        e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMalloc(&sl.counter, sizeof(unsigned int));
        if (e == cudaSuccess && scratch) e = cudaMalloc(&sl.scratch, scratch);
        if (e == cudaSuccess) e = cudaMalloc(&sl.d_desc, desc_bytes);
        if (e == cudaSuccess) e = cudaMallocHost(&sl.h_desc, desc_bytes);
        s->free_slots.push_back(static_cast<int>(slots - 1 - k));
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        s->release();
        delete s;
        return e == cudaErrorMemoryAllocation ? POLAR_ENOMEM : POLAR_ECUDA;
    }
    try {
        s->thread = std::thread([s] { s->run(); });
    } catch (...) {
        s->release();
        delete s;
        return POLAR_ENOMEM;
    }
    *out = s;
    return POLAR_OK;
}

polar_status polar_server_publish(polar_server_t *s, uint64_t n_published) {
    if (!s) return POLAR_EINVAL;
    const uint64_t old = s->published.load(std::memory_order_relaxed);
    if (n_published < old) return POLAR_EINVAL;
    if (n_published - s->completed.load(std::memory_order_acquire) > s->capacity) return POLAR_EINVAL;
    for (uint64_t i = old; i < n_published; ++i) {
        const polar_request &r = s->reqs[i % s->capacity];
        if (r.code_id >= s->code_N.size()) return POLAR_EINVAL;
        const size_t lb = size_t(s->code_N[r.code_id]) * s->es, ob = s->out_bytes(r.code_id);
        if (r.llr_off > s->h_llr_bytes || s->h_llr_bytes - r.llr_off < lb ||
            r.out_off > s->h_out_bytes || s->h_out_bytes - r.out_off < ob)
            return POLAR_EINVAL;
    }
    s->published.store(n_published, std::memory_order_release);
    return POLAR_OK;
}

polar_status polar_server_progress(const polar_server_t *s, uint64_t *n_completed,
                                   uint64_t *n_admissions, uint64_t *n_launches) {
    if (!s) return POLAR_EINVAL;
    if (n_completed) *n_completed = s->completed.load(std::memory_order_acquire);
    if (n_admissions) *n_admissions = s->admissions.load(std::memory_order_relaxed);
    if (n_launches) *n_launches = s->launches.load(std::memory_order_relaxed);
    return static_cast<polar_status>(s->error.load());
}

polar_status polar_server_destroy(polar_server_t *s) {
    if (!s) return POLAR_EINVAL;
    s->stop.store(true);
    if (s->thread.joinable()) s->thread.join();
    const polar_status st = static_cast<polar_status>(s->error.load());
    int cur = -1;
    cudaGetDevice(&cur);
    cudaSetDevice(s->batch->device);
    s->release();
    if (cur >= 0) cudaSetDevice(cur);
    delete s;
    return st;
}

}  // extern "C"
