// A6: ascending order of the match keys key = (id << 40) | x, which is the
// ascending (pattern id, offset) order the match list is defined in.
//
// Least-significant-digit radix sort over 8-bit digits.  Only the digits
// that can be non-zero are sorted: those of the offset field (bits below
// ceil(log2(n))) and of the id field (bits 40.. up to ceil(log2(k))).
//
//   1. one histogram kernel reads the keys once and counts every pass's
//      digits (the totals do not depend on the order), and clears the
//      per-tile status words of the passes;
//   2. one kernel per pass: each CTA takes the next tile of 4096 keys from a
//      counter, ranks its keys stably (ballot multisplit + per-warp digit counters),
//      publishes its digit counts, adds up the counts of the tiles before it
//      by looking back through their published words (decoupled look-back),
//      and scatters.  Look-back waits are bounded: a wait that runs out
//      records RK_ETIMEOUT in d_info[1].
//
// Every kernel reads the key count from d_info on the device, so nothing
// returns to the host between the scan and the sorted list.
#include <algorithm>
#include <mutex>

#include "rk_internal.cuh"
#include "rk_sortws.cuh"

namespace rk {
namespace {

constexpr uint32_t kThreads = 256;
constexpr uint32_t kWarps = kThreads / 32;
constexpr uint32_t kPerWarp = kSortTile / kWarps;  // 512 consecutive keys per warp
constexpr uint64_t kFlagAgg = 1ull << 62;          // tile's own counts published
constexpr uint64_t kFlagInc = 2ull << 62;          // inclusive prefix published
constexpr uint64_t kCountMask = (1ull << 62) - 1;
constexpr uint64_t kLookbackTimeoutNs = 2000000000ull;

__device__ __forceinline__ bool sort_count(const unsigned long long *info, uint64_t cap,
                                           uint64_t *m, uint32_t *tiles) {
    const uint64_t M = info[0];
    if (M > cap || M < 2 || info[1] != RK_OK) return false;
    *m = M;
    *tiles = (uint32_t)((M + kSortTile - 1) / kSortTile);
    return true;
}

// Lanes holding a valid key whose 8-bit digit equals this lane's: one ballot
// per digit bit, a fixed cost whatever the number of distinct digits (a
// warp match instruction takes longer the more distinct values there are).
__device__ __forceinline__ uint32_t digit_peers(uint32_t d, bool valid) {
    uint32_t peers = __ballot_sync(0xffffffffu, valid);
#pragma unroll
    for (uint32_t b = 0; b < 8; ++b) {
        const bool bit = (d >> b) & 1u;
        const uint32_t bal = __ballot_sync(0xffffffffu, bit);
        peers &= bit ? bal : ~bal;
    }
    return peers;
}

struct Shifts {
    uint32_t s[kMaxSortPasses];
    uint32_t n;
};

__global__ void __launch_bounds__(kThreads) rk_sort_hist_kernel(const uint64_t *keys,
                                                                const unsigned long long *info,
                                                                uint64_t cap, Shifts sh,
                                                                uint32_t *ghist,
                                                                uint64_t *status,
                                                                uint64_t tiles_max) {
    uint64_t M;
    uint32_t T;
    if (!sort_count(info, cap, &M, &T)) return;
    __shared__ uint32_t h[kMaxSortPasses][256];
    for (uint32_t p = 0; p < sh.n; ++p) h[p][threadIdx.x] = 0;
    __syncthreads();
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < M; i += stride) {
        const uint64_t k = keys[i];
        for (uint32_t p = 0; p < sh.n; ++p) atomicAdd(&h[p][(uint32_t)(k >> sh.s[p]) & 255u], 1u);
    }
    // clear the look-back words of every pass (tiles actually used)
    const uint64_t per_pass = (uint64_t)T * 256u;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < sh.n * per_pass;
         i += stride)
        status[(i / per_pass) * tiles_max * 256u + i % per_pass] = 0;
    __syncthreads();
    for (uint32_t p = 0; p < sh.n; ++p)
        if (h[p][threadIdx.x]) atomicAdd(&ghist[p * 256 + threadIdx.x], h[p][threadIdx.x]);
}

__global__ void __launch_bounds__(kThreads) rk_sort_pass_kernel(
    const uint64_t *in, uint64_t *out, unsigned long long *info, uint64_t cap, uint32_t shift,
    const uint32_t *ghist, uint64_t *status, uint32_t *counter) {
    uint64_t M;
    uint32_t T;
    if (!sort_count(info, cap, &M, &T)) return;
    __shared__ uint32_t wcnt[kWarps][256];  // per-warp digit counts, then exclusive offsets
    __shared__ uint32_t dbase[256];         // global start of each digit in this tile
    __shared__ uint32_t s_tile;
    __shared__ int s_abort;
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t lt = (1u << lane) - 1u;

    // exclusive prefix of this pass's digit totals (thread d owns digit d):
    // shuffle scan within each warp, then over the 8 warp totals
    uint32_t gbase;
    {
        __shared__ uint32_t wsum[kWarps];
        const uint32_t v = ghist[tid];
        uint32_t incl = v;
#pragma unroll
        for (uint32_t d = 1; d < 32; d <<= 1) {
            const uint32_t o = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += o;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        uint32_t before = 0;
        for (uint32_t w = 0; w < warp; ++w) before += wsum[w];
        gbase = before + incl - v;
    }
    for (;;) {
        __syncthreads();
        if (tid == 0) {
            s_tile = atomicAdd(counter, 1u);
            s_abort = 0;
        }
        for (uint32_t w = 0; w < kWarps; ++w) wcnt[w][tid] = 0;
        __syncthreads();
        const uint32_t tile = s_tile;
        if (tile >= T) return;

        // stable local ranks: warp w takes keys [w*512, (w+1)*512) of the tile
        const uint64_t base = (uint64_t)tile * kSortTile + (uint64_t)warp * kPerWarp;
        uint64_t key[kPerWarp / 32];
        uint32_t rank[kPerWarp / 32];
        // all of this warp's keys first (independent loads in flight together)
#pragma unroll
        for (uint32_t r = 0; r < kPerWarp / 32; ++r) {
            const uint64_t idx = base + r * 32 + lane;
            key[r] = idx < M ? __ldcg(in + idx) : 0;
        }
#pragma unroll
        for (uint32_t r = 0; r < kPerWarp / 32; ++r) {
            const uint64_t idx = base + r * 32 + lane;
            const bool valid = idx < M;
            const uint32_t d = (uint32_t)(key[r] >> shift) & 255u;
            const uint32_t peers = digit_peers(d, valid);
            const uint32_t before = valid ? wcnt[warp][d] : 0;
            rank[r] = before + __popc(peers & lt);
            __syncwarp();
            if (valid && (peers & lt) == 0) wcnt[warp][d] = before + __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        // thread d: per-warp exclusive offsets and the tile's count of digit d
        uint32_t cnt = 0;
        for (uint32_t w = 0; w < kWarps; ++w) {
            const uint32_t c = wcnt[w][tid];
            wcnt[w][tid] = cnt;
            cnt += c;
        }
        // decoupled look-back over the tiles before this one
        uint64_t *st = status + (uint64_t)tile * 256u + tid;
        uint64_t excl = 0;
        if (tile == 0) {
            *reinterpret_cast<volatile uint64_t *>(st) = kFlagInc | cnt;
        } else {
            *reinterpret_cast<volatile uint64_t *>(st) = kFlagAgg | cnt;
            // read kWindow predecessors per step (loads in flight together),
            // add their counts back to the first inclusive prefix
            constexpr int kWindow = 16;
            int64_t j = (int64_t)tile - 1;
            uint64_t t0 = 0;
            bool done = false;
            while (!done && j >= 0) {
                uint64_t v[kWindow];
#pragma unroll
                for (int u = 0; u < kWindow; ++u)
                    v[u] = j - u >= 0 ? *reinterpret_cast<volatile const uint64_t *>(
                                            status + (uint64_t)(j - u) * 256u + tid)
                                      : kFlagInc;
                int consumed = 0;
                bool stalled = false;
#pragma unroll
                for (int u = 0; u < kWindow; ++u) {
                    if (done || stalled) continue;
                    if (v[u] & kFlagInc) {
                        excl += v[u] & kCountMask;
                        done = true;
                    } else if (v[u] & kFlagAgg) {
                        excl += v[u] & kCountMask;
                        ++consumed;
                    } else {
                        stalled = true;  // not published yet (claimed earlier, so it runs)
                    }
                }
                j -= consumed;
                if (stalled) {
                    if (t0 == 0) t0 = globaltimer_ns();
                    else if (globaltimer_ns() - t0 > kLookbackTimeoutNs) {
                        info[1] = RK_ETIMEOUT;
                        s_abort = 1;
                        break;
                    }
                }
            }
            __threadfence();
            *reinterpret_cast<volatile uint64_t *>(st) = kFlagInc | (excl + cnt);
        }
        dbase[tid] = gbase + (uint32_t)excl;
        __syncthreads();
        if (s_abort) return;
#pragma unroll
        for (uint32_t r = 0; r < kPerWarp / 32; ++r) {
            const uint64_t idx = base + r * 32 + lane;
            if (idx < M) {
                const uint32_t d = (uint32_t)(key[r] >> shift) & 255u;
                out[dbase[d] + wcnt[warp][d] + rank[r]] = key[r];
            }
        }
    }
}

// Arrival with release semantics (gpu scope): the CTA's writes ordered
// before it by the preceding __syncthreads are visible to any thread that
// acquires the counter value.
__device__ __forceinline__ void arrive_release(unsigned int *ctr) {
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(ctr) : "memory");
}

__device__ __forceinline__ unsigned int load_acquire(const unsigned int *ctr) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(ctr) : "memory");
    return v;
}

// Grid-wide barrier of a cooperative launch (every CTA resident): one
// arrival counter in global memory, target = barriers passed x CTAs; a
// release arrival and acquire loads order the phases' memory.  The wait is
// bounded; on a timeout RK_ETIMEOUT is recorded and false returned.
__device__ __forceinline__ bool grid_sync(unsigned int *ctr, unsigned int target,
                                          unsigned long long *info, int *s_ok) {
    __syncthreads();
    if (threadIdx.x == 0) {
        arrive_release(ctr);
        int ok = 1;
        uint64_t t0 = 0;
        while (load_acquire(ctr) < target) {
            const uint64_t now = globaltimer_ns();
            if (t0 == 0) {
                t0 = now;
            } else if (now - t0 > kLookbackTimeoutNs) {
                info[1] = RK_ETIMEOUT;
                ok = 0;
                break;
            }
        }
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

// Inclusive sum of v over the lanes up to this one.
__device__ __forceinline__ uint32_t warp_incl(uint32_t v, uint32_t lane) {
#pragma unroll
    for (uint32_t d = 1; d < 32; d <<= 1) {
        const uint32_t o = __shfl_up_sync(0xffffffffu, v, d);
        if (lane >= d) v += o;
    }
    return v;
}

// Stable ranks of one tile's keys (warp w: keys [w*256, (w+1)*256) of the
// tile): key[r] and rank[r] per lane, the warp's digit counts in wc.
__device__ __forceinline__ void rank_tile(const uint64_t *src, uint64_t M, uint64_t base,
                                          uint32_t shift, uint64_t (&key)[kPerWarp / 32],
                                          uint32_t (&rank)[kPerWarp / 32], uint32_t *wc,
                                          uint32_t lane, uint32_t lt) {
#pragma unroll
    for (uint32_t r = 0; r < kPerWarp / 32; ++r) {
        const uint64_t idx = base + r * 32 + lane;
        key[r] = idx < M ? __ldcg(src + idx) : 0;
    }
#pragma unroll
    for (uint32_t r = 0; r < kPerWarp / 32; ++r) {
        const bool valid = base + r * 32 + lane < M;
        const uint32_t d = (uint32_t)(key[r] >> shift) & 255u;
        const uint32_t peers = digit_peers(d, valid);
        const uint32_t bef = valid ? wc[d] : 0;
        rank[r] = bef + __popc(peers & lt);
        __syncwarp();
        if (valid && (peers & lt) == 0) wc[d] = bef + __popc(peers);
        __syncwarp();
    }
}

// Every pass over a single tile (at most kSortTile keys) in one CTA: the keys
// stay in registers (warp w: keys [w*256, (w+1)*256)), each pass ranks them,
// scatters them to their place in the pass's order in shared memory and
// reads them back.  No grid barrier, no global round trip between passes.
__device__ __forceinline__ void sort_one_tile(uint64_t *keys, uint64_t M, const Shifts &sh,
                                              uint64_t *sbuf, uint32_t (&wcnt)[kWarps][256],
                                              uint32_t *dbase, uint32_t *wsum) {
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    const uint32_t base = warp * kPerWarp;
    uint64_t key[kPerWarp / 32];
    uint32_t rank[kPerWarp / 32];
#pragma unroll
    for (uint32_t r = 0; r < kPerWarp / 32; ++r) {
        const uint32_t idx = base + r * 32 + lane;
        key[r] = idx < M ? __ldcg(keys + idx) : 0;
    }
    for (uint32_t p = 0; p < sh.n; ++p) {
        const uint32_t shift = sh.s[p];
        for (uint32_t w = 0; w < kWarps; ++w) wcnt[w][tid] = 0;
        __syncthreads();
#pragma unroll
        for (uint32_t r = 0; r < kPerWarp / 32; ++r) {
            const bool valid = base + r * 32 + lane < M;
            const uint32_t d = (uint32_t)(key[r] >> shift) & 255u;
            const uint32_t peers = digit_peers(d, valid);
            const uint32_t bef = valid ? wcnt[warp][d] : 0;
            rank[r] = bef + __popc(peers & lt);
            __syncwarp();
            if (valid && (peers & lt) == 0) wcnt[warp][d] = bef + __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        uint32_t c = 0;  // digit tid: per-warp exclusive offsets, tile count
        for (uint32_t w = 0; w < kWarps; ++w) {
            const uint32_t x = wcnt[w][tid];
            wcnt[w][tid] = c;
            c += x;
        }
        const uint32_t incl = warp_incl(c, lane);
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        uint32_t before = 0;
        for (uint32_t w = 0; w < warp; ++w) before += wsum[w];
        dbase[tid] = before + incl - c;
        __syncthreads();
#pragma unroll
        for (uint32_t r = 0; r < kPerWarp / 32; ++r)
            if (base + r * 32 + lane < M) {
                const uint32_t d = (uint32_t)(key[r] >> shift) & 255u;
                sbuf[dbase[d] + wcnt[warp][d] + rank[r]] = key[r];
            }
        __syncthreads();
#pragma unroll
        for (uint32_t r = 0; r < kPerWarp / 32; ++r)
            if (base + r * 32 + lane < M) key[r] = sbuf[base + r * 32 + lane];
        __syncthreads();
    }
#pragma unroll
    for (uint32_t r = 0; r < kPerWarp / 32; ++r) {
        const uint32_t idx = base + r * 32 + lane;
        if (idx < M) keys[idx] = key[r];
    }
}

// Every pass in one cooperative launch, for outputs of a few thousand tiles.
// cnt holds, digit-major, the count of digit d among the keys of tile t at
// [d * pitch + t].  Per pass:
//   A  each CTA ranks its tile's keys stably (per-warp digit counters) and
//      publishes the tile's digit counts;
//   B  one warp per digit turns its row into exclusive prefixes over the
//      tiles (in place) and a total;
//   C  each CTA scatters its keys to (start of the digit) + (prefix of the
//      tile) + (rank within the tile);
// with a grid barrier after each phase.  With one tile per CTA the keys,
// ranks and counters stay on chip from A to C; with more, C ranks again.
// A single tile is sorted by one CTA alone, without barriers.
// A fixed number of barriers replaces the chain of look-back waits, whose
// length grows with the tile count.  An odd pass count ends with a copy
// back from the second buffer.  CTAs beyond the tile count leave at once.
__global__ void __launch_bounds__(kThreads) rk_sort_fused_kernel(
    uint64_t *keys, uint64_t *tmp, unsigned long long *info, uint64_t cap, Shifts sh,
    uint32_t *cnt, uint32_t pitch, uint32_t *totals, unsigned int *bar) {
    uint64_t M;
    uint32_t T;
    if (!sort_count(info, cap, &M, &T)) return;
    const uint32_t G = min(gridDim.x, T);  // CTAs taking part
    if (blockIdx.x >= G) return;
    __shared__ uint32_t wcnt[kWarps][256];
    __shared__ uint32_t dbase[256];
    __shared__ uint32_t wsum[kWarps];
    __shared__ int s_ok;
    if (T == 1) {
        __shared__ uint64_t sbuf[kSortTile];
        sort_one_tile(keys, M, sh, sbuf, wcnt, dbase, wsum);
        return;
    }
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    const bool one = T <= G;  // one tile per CTA: state kept from A to C
    unsigned int passed = 0;
    uint64_t key[kPerWarp / 32];
    uint32_t rank[kPerWarp / 32];
    for (uint32_t p = 0; p < sh.n; ++p) {
        const uint64_t *src = (p & 1) ? tmp : keys;
        uint64_t *dst = (p & 1) ? keys : tmp;
        const uint32_t shift = sh.s[p];

        // A: rank each tile, publish its digit counts
        for (uint32_t t = blockIdx.x; t < T; t += G) {
            for (uint32_t w = 0; w < kWarps; ++w) wcnt[w][tid] = 0;
            __syncthreads();
            rank_tile(src, M, (uint64_t)t * kSortTile + (uint64_t)warp * kPerWarp, shift, key,
                      rank, wcnt[warp], lane, lt);
            __syncthreads();
            uint32_t c = 0;
            for (uint32_t w = 0; w < kWarps; ++w) c += wcnt[w][tid];
            cnt[(uint64_t)tid * pitch + t] = c;
            __syncthreads();
        }
        if (!grid_sync(bar, ++passed * G, info, &s_ok)) return;

        // B: per digit, exclusive prefix over the tiles (in place) and total:
        // under 32 tiles one thread per digit (its loads issued together),
        // else one warp per digit (256 warps or more take part)
        if (T < 32) {
            if (blockIdx.x == 0) {
                uint32_t *row = cnt + (uint64_t)tid * pitch;
                uint32_t v[32];
#pragma unroll
                for (uint32_t t = 0; t < 32; ++t) v[t] = t < T ? __ldcg(row + t) : 0u;
                uint32_t sum = 0;
#pragma unroll
                for (uint32_t t = 0; t < 32; ++t)
                    if (t < T) {
                        row[t] = sum;
                        sum += v[t];
                    }
                totals[tid] = sum;
            }
        } else
        for (uint32_t d = blockIdx.x * kWarps + warp; d < 256; d += G * kWarps) {
            uint32_t *row = cnt + (uint64_t)d * pitch;
            uint32_t carry = 0;
            for (uint32_t t0 = 0; t0 < T; t0 += 8 * 32) {
                uint32_t v[8];
#pragma unroll
                for (uint32_t j = 0; j < 8; ++j) {
                    const uint32_t t = t0 + 32 * j + lane;
                    v[j] = t < T ? __ldcg(row + t) : 0u;
                }
#pragma unroll
                for (uint32_t j = 0; j < 8; ++j) {
                    const uint32_t t = t0 + 32 * j + lane;
                    const uint32_t incl = warp_incl(v[j], lane);
                    if (t < T) row[t] = carry + incl - v[j];
                    carry += __shfl_sync(0xffffffffu, incl, 31);
                }
            }
            if (lane == 0) totals[d] = carry;
        }
        if (!grid_sync(bar, ++passed * G, info, &s_ok)) return;

        // C: scatter
        for (uint32_t t = blockIdx.x; t < T; t += G) {
            const uint32_t tot = __ldcg(totals + tid);
            const uint32_t tpre = __ldcg(cnt + (uint64_t)tid * pitch + t);
            const uint64_t base = (uint64_t)t * kSortTile + (uint64_t)warp * kPerWarp;
            if (!one) {
                for (uint32_t w = 0; w < kWarps; ++w) wcnt[w][tid] = 0;
                __syncthreads();
                rank_tile(src, M, base, shift, key, rank, wcnt[warp], lane, lt);
                __syncthreads();
            }
            // per-warp exclusive offsets of digit tid within the tile
            uint32_t c = 0;
            for (uint32_t w = 0; w < kWarps; ++w) {
                const uint32_t x = wcnt[w][tid];
                wcnt[w][tid] = c;
                c += x;
            }
            const uint32_t incl = warp_incl(tot, lane);
            if (lane == 31) wsum[warp] = incl;
            __syncthreads();
            uint32_t before = 0;
            for (uint32_t w = 0; w < warp; ++w) before += wsum[w];
            dbase[tid] = before + incl - tot + tpre;
            __syncthreads();
#pragma unroll
            for (uint32_t r = 0; r < kPerWarp / 32; ++r) {
                if (base + r * 32 + lane < M) {
                    const uint32_t d = (uint32_t)(key[r] >> shift) & 255u;
                    dst[dbase[d] + wcnt[warp][d] + rank[r]] = key[r];
                }
            }
            __syncthreads();
        }
        if (p + 1 < sh.n || (sh.n & 1))
            if (!grid_sync(bar, ++passed * G, info, &s_ok)) return;
    }
    if (sh.n & 1)
        for (uint64_t i = blockIdx.x * (uint64_t)kThreads + tid; i < M; i += (uint64_t)G * kThreads)
            keys[i] = __ldcg(tmp + i);
}

__global__ void rk_sort_copy_kernel(const uint64_t *in, uint64_t *out,
                                    const unsigned long long *info, uint64_t cap) {
    uint64_t M;
    uint32_t T;
    if (!sort_count(info, cap, &M, &T)) return;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < M;
         i += (uint64_t)gridDim.x * blockDim.x)
        out[i] = in[i];
}

uint32_t bits_for(uint64_t max_value) {
    uint32_t b = 0;
    while (b < 64 && (max_value >> b)) ++b;
    return b;
}

// CTAs of the fused sort: at most two per SM, all resident (0: the kernel
// does not fit on this device).
uint32_t fused_grid(int sm_count) {
    constexpr int kMaxDevices = 64;
    static std::mutex mu;
    static bool dev_seen[kMaxDevices] = {};
    static uint32_t per_sm[kMaxDevices];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return 0;
    std::lock_guard<std::mutex> lk(mu);
    if (!dev_seen[dev]) {
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, rk_sort_fused_kernel, kThreads, 0) !=
            cudaSuccess)
            nb = 0;
        per_sm[dev] = (uint32_t)std::max(0, std::min(nb, 2));
        dev_seen[dev] = true;
    }
    return per_sm[dev] * (uint32_t)sm_count;
}

// Most tiles of 2048 keys per resident CTA that the fused sort takes: with
// more than one per CTA, phases A and C loop over them (C ranks again).
constexpr uint64_t kFusedTilesPerCta = 32;

// CTAs of the fused sort for an output of `capacity` keys (0: the look-back
// kernels are used instead).
uint32_t fused_ctas(int sm_count, uint64_t capacity, bool allow_fused) {
    const uint32_t gmax = allow_fused ? fused_grid(sm_count) : 0;
    const uint64_t tiles = sort_ws_layout(capacity).tiles;
    if (!gmax || tiles > kFusedTilesPerCta * gmax) return 0;
    return (uint32_t)std::min<uint64_t>(tiles, gmax);
}

// The digit shifts of a plain search's keys: the offset field's bits below
// ceil(log2(n)), then the id field's bits up to ceil(log2(k)).
uint32_t plain_shifts(uint64_t n, uint32_t k, uint32_t *shifts) {
    uint32_t ns = 0;
    const uint32_t ob = bits_for(n - 1), pb = bits_for(k - 1);
    for (uint32_t s = 0; s < ob; s += 8) shifts[ns++] = s;
    for (uint32_t s = 0; s < pb; s += 8) shifts[ns++] = RK_KEY_OFFSET_BITS + s;
    return ns;
}

}  // namespace

uint64_t sort_workspace_bytes(uint64_t capacity) { return sort_ws_bytes(capacity); }

int launch_sort_shifts(int sm_count, const uint32_t *shifts, uint32_t nshift, uint64_t *d_keys,
                       uint64_t capacity, const uint64_t *d_info, void *d_ws, uint64_t ws_bytes,
                       cudaStream_t stream, bool allow_fused) {
    if (capacity < 2 || nshift == 0) return RK_OK;
    if (nshift > kMaxSortPasses || ws_bytes < sort_ws_bytes(capacity)) return RK_EINVAL;
    const SortWsLayout L = sort_ws_layout(capacity);
    uint8_t *ws = reinterpret_cast<uint8_t *>(d_ws);
    uint64_t *tmp = reinterpret_cast<uint64_t *>(ws + L.tmp_off);
    uint32_t *counters = reinterpret_cast<uint32_t *>(ws + L.ctrl_off);
    uint32_t *ghist = reinterpret_cast<uint32_t *>(ws + L.ghist_off);
    uint64_t *status = reinterpret_cast<uint64_t *>(ws + L.status_off);
    unsigned long long *info =
        reinterpret_cast<unsigned long long *>(const_cast<uint64_t *>(d_info));
    Shifts sh{};
    for (uint32_t i = 0; i < nshift; ++i) sh.s[sh.n++] = shifts[i];

    if (cudaMemsetAsync(ws + L.ctrl_off, 0, L.status_off - L.ctrl_off, stream) != cudaSuccess)
        return RK_ECUDA;
    // up to kFusedTilesPerCta tiles per CTA: every pass in one cooperative launch
    if (const uint32_t g = fused_ctas(sm_count, capacity, allow_fused)) {
        // digit-major counts, 256 x tiles (in the look-back words' space)
        uint32_t *cnt = reinterpret_cast<uint32_t *>(status);
        uint32_t pitch = (uint32_t)L.tiles;
        uint32_t *totals = ghist;
        unsigned int *bar = counters + 32;
        void *args[] = {&d_keys, &tmp, &info, &capacity, &sh, &cnt, &pitch, &totals, &bar};
        if (cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(rk_sort_fused_kernel), g,
                                        kThreads, args, 0, stream) != cudaSuccess) {
            cudaGetLastError();
            return RK_ECUDA;
        }
        return RK_OK;
    }
    // histogram grid: about one CTA per 4096 keys of the capacity, at most 4 per SM
    const uint32_t grid =
        (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)sm_count * 4,
                                                           (capacity + 4095) / 4096));
    const uint64_t tiles = L.tiles;
    rk_sort_hist_kernel<<<grid, kThreads, 0, stream>>>(d_keys, info, capacity, sh, ghist, status,
                                                       tiles);
    for (uint32_t p = 0; p < sh.n; ++p) {
        const uint64_t *src = (p & 1) ? tmp : d_keys;
        uint64_t *dst = (p & 1) ? d_keys : tmp;
        const uint32_t pgrid = (uint32_t)std::min<uint64_t>(tiles, (uint64_t)sm_count * 8);
        rk_sort_pass_kernel<<<pgrid, kThreads, 0, stream>>>(
            src, dst, info, capacity, sh.s[p], ghist + p * 256, status + (uint64_t)p * tiles * 256,
            counters + p);
    }
    if (sh.n & 1)
        rk_sort_copy_kernel<<<(uint32_t)sm_count * 4, 256, 0, stream>>>(tmp, d_keys, info, capacity);
    return cudaGetLastError() == cudaSuccess ? RK_OK : RK_ECUDA;
}

int launch_sort(const rk_table *t, uint64_t n, uint64_t *d_keys, uint64_t capacity,
                const uint64_t *d_info, void *d_ws, uint64_t ws_bytes, cudaStream_t stream) {
    if (n == 0 || t->dev.n_patterns == 0) return RK_OK;
    uint32_t shifts[kMaxSortPasses];
    const uint32_t ns = plain_shifts(n, t->dev.n_patterns, shifts);
    return launch_sort_shifts(t->sm_count, shifts, ns, d_keys, capacity, d_info, d_ws, ws_bytes,
                              stream, true);
}

uint32_t sort_launches(const rk_table *t, uint64_t n, uint64_t capacity) {
    if (n == 0 || t->dev.n_patterns == 0 || capacity < 2) return 0;
    uint32_t shifts[kMaxSortPasses];
    const uint32_t ns = plain_shifts(n, t->dev.n_patterns, shifts);
    if (ns == 0) return 0;
    if (fused_ctas(t->sm_count, capacity, true)) return 1;
    return 1 + ns + (ns & 1);  // histogram, one kernel per pass, copy back
}

}  // namespace rk
