// A6: ascending order of the match keys key = (id << 40) | x, which is the
// ascending (pattern id, offset) order the match list is defined in.
//
// Least-significant-digit radix sort over 8-bit digits.  Only the digits
// that can be non-zero are sorted: those of the offset field (bits below
// ceil(log2(n))) and of the id field (bits 40.. up to ceil(log2(k))).  Each
// pass is histogram -> exclusive scan -> stable scatter, every kernel reading
// the key count from d_info on the device, so nothing returns to the host
// between the scan and the sorted list.
#include "rk_internal.cuh"

namespace rk {
namespace {

constexpr uint32_t kSortThreads = 256;
constexpr uint32_t kSortRounds = 16;
constexpr uint32_t kSortTile = kSortThreads * kSortRounds;  // keys per tile
constexpr uint32_t kScanThreads = 1024;

__device__ __forceinline__ bool sort_count(const unsigned long long *info, uint64_t cap,
                                           uint64_t *m, uint32_t *tiles) {
    uint64_t M = info[0];
    if (M > cap || M < 2) return false;
    *m = M;
    *tiles = (uint32_t)((M + kSortTile - 1) / kSortTile);
    return true;
}

__global__ void __launch_bounds__(kSortThreads) rk_sort_hist_kernel(const uint64_t *keys,
                                                            const unsigned long long *info,
                                                            uint64_t cap, uint32_t shift,
                                                            uint32_t *hist) {
    uint64_t M;
    uint32_t T;
    if (!sort_count(info, cap, &M, &T)) return;
    __shared__ uint32_t h[256];
    const uint32_t tid = threadIdx.x;
    for (uint32_t tile = blockIdx.x; tile < T; tile += gridDim.x) {
        h[tid] = 0;
        __syncthreads();
        const uint64_t base = (uint64_t)tile * kSortTile;
#pragma unroll 4
        for (uint32_t r = 0; r < kSortRounds; ++r) {
            uint64_t idx = base + r * kSortThreads + tid;
            if (idx < M) atomicAdd(&h[(uint32_t)(keys[idx] >> shift) & 255u], 1u);
        }
        __syncthreads();
        hist[(uint64_t)tid * T + tile] = h[tid];
        __syncthreads();
    }
}

// Exclusive prefix sum, in place, of hist[0 .. 256*T) (digit-major order).
__global__ void __launch_bounds__(kScanThreads) rk_sort_prefix_kernel(const unsigned long long *info,
                                                            uint64_t cap, uint32_t *hist) {
    uint64_t M;
    uint32_t T;
    if (!sort_count(info, cap, &M, &T)) return;
    __shared__ uint32_t wsum[kScanThreads / 32];
    __shared__ uint32_t s_carry;
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint64_t total = 256ull * T;
    if (tid == 0) s_carry = 0;
    __syncthreads();
    for (uint64_t base = 0; base < total; base += kScanThreads * 4ull) {
        uint32_t v[4], s = 0;
        for (int j = 0; j < 4; ++j) {
            uint64_t idx = base + tid * 4ull + j;
            v[j] = idx < total ? hist[idx] : 0;
            s += v[j];
        }
        uint32_t incl = s;
        for (int d = 1; d < 32; d <<= 1) {
            uint32_t o = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= (uint32_t)d) incl += o;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            uint32_t ws = wsum[lane], wi = ws;
            for (int d = 1; d < 32; d <<= 1) {
                uint32_t o = __shfl_up_sync(0xffffffffu, wi, d);
                if (lane >= (uint32_t)d) wi += o;
            }
            wsum[lane] = wi - ws;  // exclusive warp offsets
        }
        __syncthreads();
        uint32_t run = s_carry + wsum[warp] + incl - s;
        for (int j = 0; j < 4; ++j) {
            uint64_t idx = base + tid * 4ull + j;
            if (idx < total) hist[idx] = run;
            run += v[j];
        }
        __syncthreads();
        if (tid == kScanThreads - 1) s_carry = run;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kSortThreads) rk_sort_scatter_kernel(const uint64_t *in, uint64_t *out,
                                                               const unsigned long long *info,
                                                               uint64_t cap, uint32_t shift,
                                                               const uint32_t *hist) {
    uint64_t M;
    uint32_t T;
    if (!sort_count(info, cap, &M, &T)) return;
    constexpr uint32_t NW = kSortThreads / 32;
    __shared__ uint32_t cnt[NW][256];
    __shared__ uint32_t off[NW][256];
    __shared__ uint32_t gbase[256];
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    for (uint32_t w = 0; w < NW; ++w) cnt[w][tid] = 0;
    for (uint32_t tile = blockIdx.x; tile < T; tile += gridDim.x) {
        __syncthreads();
        gbase[tid] = hist[(uint64_t)tid * T + tile];
        uint32_t run = 0;  // keys of digit `tid` already placed in this tile
        const uint64_t base = (uint64_t)tile * kSortTile;
        for (uint32_t r = 0; r < kSortRounds; ++r) {
            const uint64_t idx = base + r * kSortThreads + tid;
            const bool valid = idx < M;
            const uint64_t key = valid ? in[idx] : 0;
            const uint32_t d = valid ? ((uint32_t)(key >> shift) & 255u) : 256u;
            const uint32_t peers = __match_any_sync(0xffffffffu, d);
            const uint32_t rank = __popc(peers & lt);
            if (valid && rank == 0) cnt[warp][d] = __popc(peers);
            __syncthreads();
            {  // thread `tid` owns digit `tid`: offsets of each warp's run
                uint32_t acc = run;
                for (uint32_t w = 0; w < NW; ++w) {
                    uint32_t c = cnt[w][tid];
                    cnt[w][tid] = 0;
                    off[w][tid] = acc;
                    acc += c;
                }
                run = acc;
            }
            __syncthreads();
            if (valid) out[gbase[d] + off[warp][d] + rank] = key;
        }
    }
}

__global__ void rk_sort_copy_kernel(const uint64_t *in, uint64_t *out, const unsigned long long *info,
                            uint64_t cap) {
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

uint64_t max_sort_tiles(uint64_t capacity) { return (capacity + kSortTile - 1) / kSortTile; }

}  // namespace

uint64_t sort_workspace_bytes(uint64_t capacity) {
    uint64_t keys = (capacity * 8 + 255) / 256 * 256;
    uint64_t hist = (256ull * max_sort_tiles(capacity) * 4 + 255) / 256 * 256;
    return keys + hist + 256;
}

int launch_sort(const rk_table *t, uint64_t n, uint64_t *d_keys, uint64_t capacity,
                const uint64_t *d_info, void *d_ws, uint64_t ws_bytes, cudaStream_t stream) {
    if (capacity < 2 || n == 0 || t->dev.n_patterns == 0) return RK_OK;
    if (ws_bytes < sort_workspace_bytes(capacity)) return RK_EINVAL;
    uint64_t *tmp = reinterpret_cast<uint64_t *>(d_ws);
    uint32_t *hist = reinterpret_cast<uint32_t *>(reinterpret_cast<uint8_t *>(d_ws) +
                                                  (capacity * 8 + 255) / 256 * 256);
    const unsigned long long *info = reinterpret_cast<const unsigned long long *>(d_info);

    std::vector<uint32_t> shifts;
    const uint32_t ob = bits_for(n - 1), pb = bits_for(t->dev.n_patterns - 1);
    for (uint32_t s = 0; s < ob; s += 8) shifts.push_back(s);
    for (uint32_t s = 0; s < pb; s += 8) shifts.push_back(RK_KEY_OFFSET_BITS + s);

    uint64_t tiles = max_sort_tiles(capacity);
    uint64_t grid64 = std::min<uint64_t>(tiles, (uint64_t)t->sm_count * 4);
    uint32_t grid = (uint32_t)std::max<uint64_t>(1, grid64);
    uint64_t *src = d_keys, *dst = tmp;
    for (uint32_t sh : shifts) {
        rk_sort_hist_kernel<<<grid, kSortThreads, 0, stream>>>(src, info, capacity, sh, hist);
        rk_sort_prefix_kernel<<<1, kScanThreads, 0, stream>>>(info, capacity, hist);
        rk_sort_scatter_kernel<<<grid, kSortThreads, 0, stream>>>(src, dst, info, capacity, sh, hist);
        std::swap(src, dst);
    }
    if (src != d_keys)
        rk_sort_copy_kernel<<<(uint32_t)t->sm_count * 4, 256, 0, stream>>>(src, d_keys, info, capacity);
    return cudaGetLastError() == cudaSuccess ? RK_OK : RK_ECUDA;
}

}  // namespace rk
