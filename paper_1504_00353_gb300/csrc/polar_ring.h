// First-in first-out allocator of contiguous byte ranges in a ring buffer,
// used by the serving loop for its device LLR and output rings. Host-only C++
// with no CUDA dependency, so that it can be unit-tested on its own.
#pragma once

#include <algorithm>
#include <cstddef>
#include <deque>

namespace polar {

// First-in first-out allocator of contiguous byte ranges in a ring of `cap`
// bytes: ranges are released in the order they were taken.
struct Ring {
    struct Range {
        size_t lo, hi;
    };
    size_t cap = 0, head = 0;
    std::deque<Range> live;

    // Largest range alloc() can return now.
    size_t avail() const {
        if (live.empty()) return cap;
        const size_t tail = live.front().lo;
        if (head > tail) return std::max(cap - head, tail);  // [head, cap) or wrap to [0, tail)
        return tail - head;                                   // wrapped: [head, tail)
    }
    // Take b bytes (0 < b <= avail()).
    Range alloc(size_t b) {
        size_t lo = 0;
        if (!live.empty()) {
            const size_t tail = live.front().lo;
            lo = (head > tail && cap - head < b) ? 0 : head;
        }
        head = lo + b;
        live.push_back({lo, lo + b});
        return live.back();
    }
    void release_oldest() {
        live.pop_front();
        if (live.empty()) head = 0;
    }
};

}  // namespace polar
