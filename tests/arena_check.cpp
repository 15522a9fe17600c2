// Randomised check of the serving loop's arena allocator (rk::Arena) against
// a granule map: first fit, no overlap, the used-bytes count, merging of
// released neighbours, and the admission rule (an empty arena of
// round_up(cap) bytes takes any request of up to cap bytes).  Prints "ok"
// and exits 0, or prints the first violation and exits 1.
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>

#include "rk_arena.h"

using rk::Arena;

namespace {

int fail(const char *what, unsigned long long a, unsigned long long b) {
    std::printf("FAIL %s (%llu, %llu)\n", what, a, b);
    return 1;
}

// Lowest granule index starting a free run of at least g granules, or -1.
long long first_fit(const std::vector<char> &busy, uint64_t g) {
    uint64_t run = 0;
    for (uint64_t i = 0; i < busy.size(); ++i) {
        run = busy[i] ? 0 : run + 1;
        if (run == g) return (long long)(i + 1 - g);
    }
    return -1;
}

int run(uint64_t cap, uint32_t seed, int ops) {
    const uint64_t G = Arena::kGranule;
    const uint64_t bytes = Arena::round_up(cap);
    Arena a;
    a.reset(bytes);
    std::vector<char> busy(bytes / G, 0);
    std::vector<std::pair<uint64_t, uint64_t>> live;  // offset, bytes
    std::mt19937_64 rng(seed);
    uint64_t used = 0;
    for (int op = 0; op < ops; ++op) {
        if (live.empty() || rng() % 100 < 55) {
            // sizes: empty, tiny, around a granule, up to the whole cap
            const uint64_t kind = rng() % 4;
            const uint64_t n = kind == 0 ? 0
                               : kind == 1 ? rng() % 300
                               : kind == 2 ? rng() % (cap / 8 + 1)
                                           : rng() % (cap + 1);
            const uint64_t need = Arena::round_up(n);
            const long long want = first_fit(busy, need / G);
            uint64_t off = ~0ull;
            const bool ok = a.alloc(n, &off);
            if (ok != (want >= 0)) return fail("fits iff a free run is long enough", n, ok);
            if (!ok) continue;
            if (off != (uint64_t)want * G) return fail("first fit", off, (uint64_t)want * G);
            if (off % G || off + need > bytes) return fail("inside the arena", off, need);
            for (uint64_t i = off / G; i < (off + need) / G; ++i) {
                if (busy[i]) return fail("overlap", off, i);
                busy[i] = 1;
            }
            live.emplace_back(off, need);
            used += need;
        } else {
            const size_t k = rng() % live.size();
            const auto [off, need] = live[k];
            live[k] = live.back();
            live.pop_back();
            a.release(off);
            for (uint64_t i = off / G; i < (off + need) / G; ++i) busy[i] = 0;
            used -= need;
            a.release(off);  // a second release of the same offset is ignored
        }
        if (a.used() != used) return fail("used bytes", a.used(), used);
        a.release(bytes + 12345);  // never allocated: ignored
    }
    // everything released: the free ranges merge back into one
    for (const auto &[off, need] : live) a.release(off);
    if (a.used() != 0) return fail("used after releasing all", a.used(), 0);
    if (a.free_ranges() != 1) return fail("free ranges after releasing all", a.free_ranges(), 1);
    uint64_t off = 1;
    if (!a.alloc(cap, &off) || off != 0) return fail("whole cap after releasing all", cap, off);
    return 0;
}

}  // namespace

int main() {
    // caps that are and are not granule multiples, down to below one granule
    const uint64_t caps[] = {1, 100, 256, 1000, 4096, 65536 + 17, 1 << 20, (4u << 20) + 255};
    uint32_t seed = 1;
    for (uint64_t cap : caps) {
        // the admission rule on an empty arena
        for (uint64_t n : {uint64_t(0), cap / 2, cap}) {
            Arena a;
            a.reset(Arena::round_up(cap));
            uint64_t off = 1;
            if (!a.alloc(n, &off) || off != 0) return fail("empty arena admits n <= cap", cap, n);
        }
        for (int r = 0; r < 20; ++r)
            if (run(cap, seed++, 400)) return 1;
    }
    std::printf("ok\n");
    return 0;
}
