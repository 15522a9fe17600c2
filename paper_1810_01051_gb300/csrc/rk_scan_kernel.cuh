// The scan kernel (the stages are described in rk_scan.cu) and its launch
// helpers.  The translation units rk_scan_k_*.cu each instantiate one group
// of its variants, so that they compile in parallel.
#pragma once

#include "rk_scan_body.cuh"

namespace rk {
namespace scan {

struct ScanParams {
    DevTable tab;
    const uint8_t *base;     // 16-byte aligned address at or before the text start
    uint64_t mis;            // text start - base (0..15)
    uint64_t n;              // text length
    uint64_t x_begin, x_end; // window starts scanned: [x_begin, x_end)
    uint64_t u_first;        // position (from base) of tile 0, 16-byte aligned
    uint64_t n16;            // readable bytes from base (text end rounded up to 16)
    uint64_t n_tiles;
    uint64_t *keys;
    uint64_t capacity;
    unsigned long long *info;
    uint64_t timeout_ns;     // limit of every pipeline wait
    uint32_t tile, stages, halo, warps, s2_smem;
    uint32_t sv_warps;       // role-filter kernel: survivor warps
    uint32_t withhold;       // diagnostics: the producer issues no copy at all
    CandList cand;           // deferred verification: candidate list (DEFER kernels)
};

// MAXW: most consumer warps this instance is launched with; the register
// budget per thread follows from (MAXW + 1) warps per SM.  S2S: the
// survivor-stage tables are staged in shared memory (their loads then
// compile to shared-memory loads).  DEFER: survivors stop after the
// prefix-map stage and go to the candidate list (verified by
// rk_verify_kernel).
// SAMP: 0, every position against the prefix bit set; 1 (DEFER, q = 4),
// every 4th position against the bit set of the patterns' grams at offsets
// 0..3 (P.tab.filter is the bit set staged in each case).  Tables with a
// role filter have a kernel of their own (rk_scan_rf.cuh).
template <int MODE, bool Q4, int MAXW, bool S2S, bool DEFER, int SAMP>
__global__ void __launch_bounds__((MAXW + 1) * 32, 1)
    rk_scan_tiles_kernel(const __grid_constant__ ScanParams P) {
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ volatile uint32_t s_abort;
    const SmemLayout lay =
        smem_layout(P.tab.filter_bytes, P.s2_smem, P.warps, P.stages, P.tile, P.halo);
    uint8_t *sfilt = smem;  // the bit set is first (offset 0): its base folds into addresses
    uint8_t *ss2 = smem + lay.s2_off;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + lay.bar_off);
    uint64_t *empty = full + P.stages;
    uint16_t *queues = reinterpret_cast<uint16_t *>(smem + lay.queue_off);
    uint32_t *mcount = reinterpret_cast<uint32_t *>(smem + lay.mcount_off);
    uint64_t *mbuf = reinterpret_cast<uint64_t *>(smem + lay.match_off);
    uint8_t *stage0 = smem + lay.stage_off;

    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t nw = P.warps;

    if (MODE != kFilterNone) {
        const uint4 *src = reinterpret_cast<const uint4 *>(P.tab.filter);
        uint4 *dst = reinterpret_cast<uint4 *>(sfilt);
        for (uint32_t i = tid; i < P.tab.filter_bytes / 16u; i += blockDim.x) dst[i] = src[i];
    }
    if (S2S) {
        const uint4 *src = reinterpret_cast<const uint4 *>(P.tab.s2_base);
        uint4 *dst = reinterpret_cast<uint4 *>(ss2);
        for (uint32_t i = tid; i < (P.s2_smem + 15u) / 16u; i += blockDim.x) dst[i] = src[i];
    }
    if (tid == 0) {
        for (uint32_t s = 0; s < P.stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], nw);
        }
        s_abort = 0;
        fence_mbar_init();
    }
    if (tid < nw) mcount[tid] = 0;
    __syncthreads();

    const uint64_t my_tiles =
        P.n_tiles > blockIdx.x ? (P.n_tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;

    if (warp == nw) {  // ---------------- producer warp
        if (lane != 0 || P.withhold) return;
        uint64_t issued = 0;
        for (uint64_t i = 0; i < my_tiles; ++i) {
            const uint32_t s = (uint32_t)(i % P.stages);
            if (i >= P.stages &&
                !mbar_wait_bounded(&empty[s], (uint32_t)((i / P.stages) + 1) & 1u, P.timeout_ns)) {
                s_abort = 1;
                P.info[1] = RK_ETIMEOUT;
                break;
            }
            if (s_abort) break;
            const uint64_t t = blockIdx.x + i * gridDim.x;
            const uint64_t u0 = P.u_first + t * P.tile;
            const uint64_t u1 = min(P.n16, u0 + P.tile + P.halo);
            const uint32_t bytes = (uint32_t)(u1 - u0);
            uint8_t *dst = stage0 + (size_t)s * lay.stage_stride;
            mbar_arrive_expect_tx(&full[s], bytes);
            bulk_g2s(dst, P.base + u0, bytes, &full[s]);
            issued = i + 1;
        }
        // every copy issued must have landed before the CTA may exit
        for (uint64_t i = issued > P.stages ? issued - P.stages : 0; i < issued; ++i)
            mbar_wait_bounded(&full[i % P.stages], (uint32_t)(i / P.stages) & 1u, P.timeout_ns);
        return;
    }

    // -------------------------------------- consumer warps
    WinCtx C;
    C.s2 = make_s2(P.tab, S2S ? ss2 : P.tab.s2_base);
    C.lo = P.mis + P.x_begin;
    C.hi = P.mis + P.x_end;
    C.mis = P.mis;
    C.n = P.n;
    C.key_prefix = 0;
    C.pid_shift = RK_KEY_OFFSET_BITS;
    C.q = P.tab.q;
    C.gram_bits = P.tab.gram_bits;
    C.base_log2 = P.tab.base_log2;
    C.n_lengths = P.tab.n_lengths;
    C.smap_bits = P.tab.smap_bits;
    uint16_t *q = queues + warp * kQueueCap;
    WarpCtx w{mcount + warp, mbuf + (size_t)warp * kMatchCap, P.keys, P.capacity, P.info};
    const uint32_t lane4 = lane << 2;
    const uint32_t fmask = P.tab.filter_mask;
    const uint32_t qmask = P.tab.q == 4 ? 0xFFFFFFFFu : (1u << (8u * P.tab.q)) - 1u;
    const uint32_t last = P.tile / 16u - 1u;

    for (uint64_t i = 0; i < my_tiles; ++i) {
        const uint32_t s = (uint32_t)(i % P.stages);
        if (!mbar_wait_bounded(&full[s], (uint32_t)(i / P.stages) & 1u, P.timeout_ns)) {
            s_abort = 1;
            P.info[1] = RK_ETIMEOUT;
            break;
        }
        const uint8_t *buf = stage0 + (size_t)s * lay.stage_stride;
        const uint64_t t = blockIdx.x + i * gridDim.x;
        const uint64_t u0 = P.u_first + t * P.tile;
        const uint64_t wend = min(u0 + P.tile, C.hi);
        const uint32_t nchunks = (uint32_t)((wend - u0 + 15) / 16);
        if constexpr (SAMP == 1)
            consume_tile_s4<MODE>(C, w, q, buf, u0, nchunks, P.tile, sfilt, fmask, lane4, warp, nw,
                                  lane, P.cand);
        else
            consume_tile<MODE, Q4, DEFER>(C, w, q, buf, u0, nchunks, last, sfilt, fmask, lane4,
                                          qmask, warp, nw, lane, &P.cand);
        if (lane == 0) mbar_arrive(&empty[s]);
    }
    if (!DEFER) flush(w, lane);  // (a deferred scan flushes its candidates per tile)
}

template <int MODE, bool Q4, int MAXW, bool DEFER, int SAMP>
cudaError_t launch_w(const ScanParams &p, uint32_t grid, uint32_t threads, uint32_t smem,
                     cudaStream_t st) {
    auto fn = p.s2_smem ? rk_scan_tiles_kernel<MODE, Q4, MAXW, true, DEFER, SAMP>
                        : rk_scan_tiles_kernel<MODE, Q4, MAXW, false, DEFER, SAMP>;
    // raise the dynamic shared-memory limit once per device and size
    static thread_local int seen_dev[4] = {-1, -1, -1, -1};
    static thread_local uint32_t seen_smem[4] = {0, 0, 0, 0};
    const int slot = p.s2_smem ? 1 : 0;
    int dev = 0;
    cudaGetDevice(&dev);
    if (seen_dev[slot] != dev || seen_smem[slot] < smem) {
        cudaError_t e =
            cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        seen_dev[slot] = dev;
        seen_smem[slot] = smem;
    }
    fn<<<grid, threads, smem, st>>>(p);
    return cudaGetLastError();
}

template <int MODE, bool Q4, bool DEFER, int SAMP>
cudaError_t launch_d(const ScanParams &p, uint32_t grid, uint32_t threads, uint32_t smem,
                     cudaStream_t st) {
    if (p.warps <= 8) return launch_w<MODE, Q4, 8, DEFER, SAMP>(p, grid, threads, smem, st);
    if (p.warps <= 16) return launch_w<MODE, Q4, 16, DEFER, SAMP>(p, grid, threads, smem, st);
    if (p.warps <= 24) return launch_w<MODE, Q4, 24, DEFER, SAMP>(p, grid, threads, smem, st);
    return launch_w<MODE, Q4, 31, DEFER, SAMP>(p, grid, threads, smem, st);
}


template <int MODE, bool Q4>
inline cudaError_t launch_one(const ScanParams &p, uint32_t grid, uint32_t threads, uint32_t smem,
                       cudaStream_t st, bool samp) {
    constexpr bool kCanDefer = MODE != kFilterNone;
    constexpr bool kCanSample = kCanDefer && Q4;
    if (kCanSample && p.cand.list && samp)
        return launch_d<MODE, Q4, kCanDefer, kCanSample ? 1 : 0>(p, grid, threads, smem, st);
    if (kCanDefer && p.cand.list)
        return launch_d<MODE, Q4, kCanDefer, 0>(p, grid, threads, smem, st);
    return launch_d<MODE, Q4, false, 0>(p, grid, threads, smem, st);
}

// Launchers of the variants, one translation unit each: the prefix bit set
// without a filter, replicated or flat (SAMP 0, or SAMP 1 for deferred scans
// of flat or replicated sets), and the role-filter kernel (rk_scan_rf.cuh).
cudaError_t launch_none(const ScanParams &p, uint32_t grid, uint32_t threads, uint32_t smem,
                        cudaStream_t st, bool q4);
cudaError_t launch_replicated(const ScanParams &p, uint32_t grid, uint32_t threads,
                              uint32_t smem, cudaStream_t st, bool q4, bool samp);
cudaError_t launch_flat(const ScanParams &p, uint32_t grid, uint32_t threads, uint32_t smem,
                        cudaStream_t st, bool q4, bool samp);
cudaError_t launch_role(const ScanParams &p, uint32_t grid, uint32_t threads, uint32_t smem,
                        cudaStream_t st, uint32_t step, bool side);

}  // namespace scan
}  // namespace rk
