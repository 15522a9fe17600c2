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
//      counter, ranks its keys stably (warp match + per-warp digit counters),
//      publishes its digit counts, adds up the counts of the tiles before it
//      by looking back through their published words (decoupled look-back),
//      and scatters.  Look-back waits are bounded: a wait that runs out
//      records RK_ETIMEOUT in d_info[1].
//
// Every kernel reads the key count from d_info on the device, so nothing
// returns to the host between the scan and the sorted list.
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
            const uint32_t d = valid ? ((uint32_t)(key[r] >> shift) & 255u) : 256u + lane;
            const uint32_t peers = __match_any_sync(0xffffffffu, d);
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

}  // namespace

uint64_t sort_workspace_bytes(uint64_t capacity) { return sort_ws_bytes(capacity); }

int launch_sort_shifts(int sm_count, const uint32_t *shifts, uint32_t nshift, uint64_t *d_keys,
                       uint64_t capacity, const uint64_t *d_info, void *d_ws, uint64_t ws_bytes,
                       cudaStream_t stream) {
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
    uint32_t shifts[kMaxSortPasses], ns = 0;
    const uint32_t ob = bits_for(n - 1), pb = bits_for(t->dev.n_patterns - 1);
    for (uint32_t s = 0; s < ob; s += 8) shifts[ns++] = s;
    for (uint32_t s = 0; s < pb; s += 8) shifts[ns++] = RK_KEY_OFFSET_BITS + s;
    return launch_sort_shifts(t->sm_count, shifts, ns, d_keys, capacity, d_info, d_ws, ws_bytes,
                              stream);
}

}  // namespace rk
