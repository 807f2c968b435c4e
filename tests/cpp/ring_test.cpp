// Randomised check of the serving loop's ring allocator (polar_ring.h): live
// ranges never overlap, stay inside the ring, are released oldest first, and
// every size up to avail() can be taken.
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>

#include "polar_ring.h"

static int fail(const char *what, int step) {
    std::printf("FAIL %s at step %d\n", what, step);
    return 1;
}

int main() {
    std::mt19937_64 rng(12345);
    for (int trial = 0; trial < 200; ++trial) {
        polar::Ring r;
        r.cap = 64 + rng() % 4096;
        std::deque<polar::Ring::Range> mirror;
        for (int step = 0; step < 2000; ++step) {
            const size_t a = r.avail();
            if (r.live.empty() && a != r.cap) return fail("empty ring not fully available", step);
            if (a > 0 && rng() % 3 != 0) {
                const size_t b = 1 + rng() % a;
                const polar::Ring::Range g = r.alloc(b);
                if (g.hi - g.lo != b || g.hi > r.cap) return fail("range outside ring", step);
                for (const auto &m : mirror)
                    if (g.lo < m.hi && m.lo < g.hi) return fail("overlap", step);
                mirror.push_back(g);
            } else if (!mirror.empty()) {
                if (r.live.front().lo != mirror.front().lo) return fail("not oldest first", step);
                r.release_oldest();
                mirror.pop_front();
            }
            // total live bytes never exceed the ring
            size_t used = 0;
            for (const auto &m : mirror) used += m.hi - m.lo;
            if (used > r.cap) return fail("over capacity", step);
        }
    }
    // a full drain returns the whole ring
    polar::Ring r;
    r.cap = 100;
    r.alloc(60);
    r.alloc(40);
    if (r.avail() != 0) return fail("full ring has space", 0);
    r.release_oldest();
    if (r.avail() != 60) return fail("wrap space after release", 0);
    r.alloc(50);  // wraps to [0, 50)
    if (r.avail() != 10) return fail("space between wrapped head and tail", 0);
    r.release_oldest();
    r.release_oldest();
    if (r.avail() != 100) return fail("drained ring", 0);
    std::printf("OK\n");
    return 0;
}
