// Scan kernel: the GPU matcher of Section 3.1, rebuilt for sm_103a.
//
// The paper's kernel gives each thread one text offset x, recomputes the
// O(m) shift-add hash of T[x..x+m) from global memory, compares it with the
// pattern hash and then the bytes, and sets result[x].  Here, per CTA of a
// persistent grid:
//
//  A1 stage   one producer thread streams tiles of `tile` bytes plus a halo
//             of (longest pattern - 1) bytes (rounded up to 16) into a ring
//             of shared-memory buffers with 1-D bulk copies (TMA engine),
//             signalled on mbarriers; consumer warps release buffers on a
//             second set of mbarriers.
//  stage 1    every window's q-byte prefix (q = min(4, shortest pattern)),
//             read from registers as a little-endian word, is tested against
//             a shared-memory bit set of the patterns' prefixes (an exact
//             prefilter: it can only drop windows that start no pattern).
//             Survivors are queued per warp and processed one per lane: the
//             prefix map gives the lengths of the patterns with that prefix
//             and a fingerprint of their next four bytes.
//  A2 hash    each surviving window gets the Rabin hash mod 2^61 - 1 of its
//             first L bytes for each such length L.
//  A3 probe   that hash is looked up in the table of its length group.
//  A4 verify  each pattern of the matching slot is compared byte for byte
//             (Section 3.1's compare(P, T + x, m) after hx == hy).
//  A5 emit    matches collect in a per-warp shared buffer and are appended
//             to the output with one atomic per warp flush.
//
// The survivor-stage tables (prefix map, length groups, pattern bytes) are
// copied to shared memory when they fit, else read through L1/L2.
//
// All waits are bounded; on a timeout the kernel records RK_ETIMEOUT in
// d_info[1], stops issuing copies, waits (bounded) for its copies in flight
// and returns.
#include <algorithm>

#include "rk_scan_body.cuh"

namespace rk {
namespace {

constexpr uint64_t kWaitTimeoutNs = 4000000000ull;  // 4 s per wait (default)

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
    uint32_t withhold;       // diagnostics: the producer issues no copy at all
    CandList cand;           // deferred verification: candidate list (DEFER kernels)
};

// MAXW: most consumer warps this instance is launched with; the register
// budget per thread follows from (MAXW + 1) warps per SM.  S2S: the
// survivor-stage tables are staged in shared memory (their loads then
// compile to shared-memory loads).  DEFER: survivors stop after the
// prefix-map stage and go to the candidate list (verified by
// rk_verify_kernel).
// SAMP (DEFER, q = 4): stage 1 tests every 4th position against the bit set
// of the patterns' grams at offsets 0..3 (P.tab.filter is that bit set).
template <int MODE, bool Q4, int MAXW, bool S2S, bool DEFER, bool SAMP>
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
        if (SAMP)
            consume_tile_s4<MODE>(C, w, q, buf, u0, nchunks, P.tile, sfilt, fmask, lane4, warp, nw,
                                  lane, P.cand);
        else
            consume_tile<MODE, Q4, DEFER>(C, w, q, buf, u0, nchunks, last, sfilt, fmask, lane4,
                                          qmask, warp, nw, lane, &P.cand);
        if (lane == 0) mbar_arrive(&empty[s]);
    }
    if (!DEFER) flush(w, lane);  // (a deferred scan flushes its candidates per tile)
}

template <int MODE, bool Q4, int MAXW, bool DEFER, bool SAMP>
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

template <int MODE, bool Q4, bool DEFER, bool SAMP>
cudaError_t launch_d(const ScanParams &p, uint32_t grid, uint32_t threads, uint32_t smem,
                     cudaStream_t st) {
    if (p.warps <= 8) return launch_w<MODE, Q4, 8, DEFER, SAMP>(p, grid, threads, smem, st);
    if (p.warps <= 16) return launch_w<MODE, Q4, 16, DEFER, SAMP>(p, grid, threads, smem, st);
    if (p.warps <= 24) return launch_w<MODE, Q4, 24, DEFER, SAMP>(p, grid, threads, smem, st);
    return launch_w<MODE, Q4, 31, DEFER, SAMP>(p, grid, threads, smem, st);
}

template <int MODE, bool Q4>
cudaError_t launch_one(const ScanParams &p, uint32_t grid, uint32_t threads, uint32_t smem,
                       cudaStream_t st, bool samp) {
    constexpr bool kCanDefer = MODE != kFilterNone;
    constexpr bool kCanSample = kCanDefer && Q4;
    if (kCanSample && p.cand.list && samp)
        return launch_d<MODE, Q4, kCanDefer, kCanSample>(p, grid, threads, smem, st);
    if (kCanDefer && p.cand.list)
        return launch_d<MODE, Q4, kCanDefer, false>(p, grid, threads, smem, st);
    return launch_d<MODE, Q4, false, false>(p, grid, threads, smem, st);
}

}  // namespace

int launch_scan(const rk_table *t, const uint8_t *d_text, uint64_t n, uint64_t x_begin,
                uint64_t x_end, uint64_t *d_keys, uint64_t capacity, uint64_t *d_info,
                cudaStream_t stream, const CandList *cand) {
    return launch_scan_opts(t, d_text, n, x_begin, x_end, d_keys, capacity, d_info, stream,
                            kWaitTimeoutNs, false, cand);
}

bool can_defer(const rk_table *t) {
    return t->dev.filter_mode != kFilterNone && t->dev.gram_bits <= 64 - kCandSlotShift;
}

int launch_scan_opts(const rk_table *t, const uint8_t *d_text, uint64_t n, uint64_t x_begin,
                     uint64_t x_end, uint64_t *d_keys, uint64_t capacity, uint64_t *d_info,
                     cudaStream_t stream, uint64_t timeout_ns, bool withhold,
                     const CandList *cand) {
    if (x_end > n) x_end = n;
    if (x_begin >= x_end || t->dev.n_patterns == 0) return RK_OK;
    const Tuning &tu = t->tune;
    ScanParams p{};
    p.tab = t->dev;
    uintptr_t addr = reinterpret_cast<uintptr_t>(d_text);
    p.base = reinterpret_cast<const uint8_t *>(addr & ~uintptr_t(15));
    p.mis = addr & 15u;
    p.n = n;
    p.x_begin = x_begin;
    p.x_end = x_end;
    p.u_first = (p.mis + x_begin) & ~uint64_t(15);
    p.n16 = (p.mis + n + 15) & ~uint64_t(15);
    // A text shorter than one tile per CTA takes smaller tiles (whole
    // stage-1 rounds of every warp, warps x 1 KiB) so that every SM works;
    // they fit the shared memory sized for the table's tile.
    const uint64_t span = p.mis + x_end - p.u_first;
    const uint64_t max_ctas = (uint64_t)t->sm_count * tu.ctas_per_sm;
    const uint64_t round_bytes = (uint64_t)tu.warps * 1024u;
    const uint64_t per_cta = (span + max_ctas - 1) / max_ctas;
    const uint32_t tile = (uint32_t)std::min<uint64_t>(
        tu.tile_bytes, std::max<uint64_t>(round_bytes, (per_cta + round_bytes - 1) / round_bytes *
                                                           round_bytes));
    p.n_tiles = (span + tile - 1) / tile;
    p.keys = d_keys;
    p.capacity = capacity;
    p.info = reinterpret_cast<unsigned long long *>(d_info);
    p.tile = tile;
    p.stages = tu.stages;
    p.halo = tu.halo;
    p.warps = tu.warps;
    p.s2_smem = tu.s2_smem;
    p.timeout_ns = timeout_ns;
    p.withhold = withhold ? 1u : 0u;
    if (cand && can_defer(t)) p.cand = *cand;
    // a deferred scan of a sampled table stages the grams' bit set instead
    const bool samp = p.cand.list && t->dev.sample == 4;
    if (samp) {
        p.tab.filter = t->dev.sfilter;
        p.tab.filter_bytes = t->dev.sfilter_bytes;
        p.tab.filter_mode = t->dev.sfilter_mode;
        p.tab.filter_mask = t->dev.sfilter_mask;
    }
    uint32_t grid = (uint32_t)(p.n_tiles < max_ctas ? p.n_tiles : max_ctas);
    uint32_t threads = (tu.warps + 1) * 32;
    bool q4 = t->dev.q == 4;
    const uint32_t sm = tu.smem_bytes;
    cudaError_t e;
    switch (p.tab.filter_mode) {
        case kFilterNone:
            e = q4 ? launch_one<kFilterNone, true>(p, grid, threads, sm, stream, samp)
                   : launch_one<kFilterNone, false>(p, grid, threads, sm, stream, samp);
            break;
        case kFilterReplicated:
            e = q4 ? launch_one<kFilterReplicated, true>(p, grid, threads, sm, stream, samp)
                   : launch_one<kFilterReplicated, false>(p, grid, threads, sm, stream, samp);
            break;
        default:
            e = q4 ? launch_one<kFilterFlat, true>(p, grid, threads, sm, stream, samp)
                   : launch_one<kFilterFlat, false>(p, grid, threads, sm, stream, samp);
            break;
    }
    return e == cudaSuccess ? RK_OK : RK_ECUDA;
}

}  // namespace rk
