// Second pass of a deferred scan: A2 hash, A3 probe, A4 verify and A5 emit
// for every candidate the tiled scan listed (a window whose exact q-byte
// prefix starts some pattern and whose next four bytes pass that prefix's
// fingerprint set).  The scan kernel handles one tile at a time, so its
// survivor rounds hold only the few candidates of one warp's share of a
// tile and a warp pays for the longest hash among them; here every warp
// takes 32 listed candidates at a time; a window's first 8 bytes come with
// the candidate, longer windows read the rest from the text in global memory.
#include "rk_scan_body.cuh"
#include "rk_sortws.cuh"

namespace rk {
namespace {

constexpr uint32_t kVerifyThreads = 256;
constexpr uint32_t kVerifyWarps = kVerifyThreads / 32;
constexpr uint32_t kVerifySmemMax = 32u << 10;  // survivor tables staged in shared memory

struct VerifyParams {
    DevTable tab;
    GText text;         // 16-byte aligned base at or before the text start
    uint64_t mis;       // text start - base
    uint64_t n;         // text length
    const ulonglong2 *list;
    uint64_t cap;
    const unsigned long long *count;
    uint64_t *keys;
    uint64_t capacity;
    unsigned long long *info;
};

// S2S: the survivor tables (P.tab.s2_bytes) are first copied to the block's
// dynamic shared memory, so each candidate's chain of table loads stays on
// chip; otherwise they are read through L1/L2.  Eight blocks per SM (32
// registers a thread): the kernel waits on global loads, and more resident
// warps hide more of that latency.
template <bool S2S>
__global__ void __launch_bounds__(kVerifyThreads, 8)
    rk_verify_kernel(const __grid_constant__ VerifyParams P) {
    extern __shared__ __align__(128) uint8_t ss2[];
    __shared__ uint32_t mcount[kVerifyWarps];
    __shared__ uint64_t mbuf[kVerifyWarps][kMatchCap];
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) mcount[warp] = 0;
    if (S2S) {
        const uint4 *src = reinterpret_cast<const uint4 *>(P.tab.s2_base);
        uint4 *dst = reinterpret_cast<uint4 *>(ss2);
        for (uint32_t i = threadIdx.x; i < (P.tab.s2_bytes + 15u) / 16u; i += kVerifyThreads)
            dst[i] = src[i];
    }
    __syncthreads();
    WarpCtx w{mcount + warp, mbuf[warp], P.keys, P.capacity, P.info};
    WinCtx C{};
    C.s2 = make_s2(P.tab, S2S ? ss2 : P.tab.s2_base);
    C.mis = P.mis;
    C.n = P.n;
    C.key_prefix = 0;
    C.pid_shift = RK_KEY_OFFSET_BITS;
    C.q = P.tab.q;
    C.gram_bits = P.tab.gram_bits;
    C.base_log2 = P.tab.base_log2;
    C.n_lengths = P.tab.n_lengths;

    const uint64_t nc = min((uint64_t)*P.count, P.cap);
    const uint64_t stride = (uint64_t)gridDim.x * kVerifyThreads;
    // warp-uniform loop: every lane reaches the flushes
    for (uint64_t i0 = (uint64_t)blockIdx.x * kVerifyThreads + warp * 32; i0 < nc; i0 += stride) {
        const uint64_t i = i0 + lane;
        if (i < nc) {
            const ulonglong2 c = P.list[i];
            const uint64_t x = cand_x(c.x);
            const WText win{P.text, x + P.mis, c.y};
            probe_slot(C, w, win, x + P.mis, x, cand_slot(c.x), cand_class(c.x));
        }
        __syncwarp();
        if (*reinterpret_cast<volatile uint32_t *>(w.mcount) >= kMatchCap - 32) flush(w, lane);
    }
    flush(w, lane);
}

}  // namespace

int launch_verify(const rk_table *t, const uint8_t *d_text, uint64_t n, const CandList &cand,
                  uint64_t *d_keys, uint64_t capacity, uint64_t *d_info, cudaStream_t stream) {
    if (n == 0 || t->dev.n_patterns == 0) return RK_OK;
    VerifyParams p{};
    p.tab = t->dev;
    const uintptr_t addr = reinterpret_cast<uintptr_t>(d_text);
    p.mis = addr & 15u;
    p.text = GText{reinterpret_cast<const uint8_t *>(addr & ~uintptr_t(15)),
                   (p.mis + n + 15) & ~uint64_t(15)};
    p.n = n;
    p.list = cand.list;
    p.cap = cand.cap;
    p.count = cand.count;
    p.keys = d_keys;
    p.capacity = capacity;
    p.info = reinterpret_cast<unsigned long long *>(d_info);
    const uint32_t grid = (uint32_t)t->sm_count * 8;
    // tables up to 32 KiB go to shared memory (with the static 8 KiB, at
    // least five blocks of 256 threads per SM); larger ones stay in L2
    const uint32_t s2 = t->dev.s2_bytes;
    if (s2 <= kVerifySmemMax) {
        rk_verify_kernel<true><<<grid, kVerifyThreads, (s2 + 15u) / 16u * 16u, stream>>>(p);
    } else {
        rk_verify_kernel<false><<<grid, kVerifyThreads, 0, stream>>>(p);
    }
    return cudaGetLastError() == cudaSuccess ? RK_OK : RK_ECUDA;
}

}  // namespace rk
