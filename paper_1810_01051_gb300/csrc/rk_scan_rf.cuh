// The scan kernel for tables with a role filter (DevTable::rf_step), warp-
// specialised.  Per CTA of a persistent grid:
//   - a producer warp streams tiles plus halo into a ring of shared-memory
//     stages with 1-D bulk copies (as the other scan kernel does);
//   - stage-1 warps test every 2nd or 4th position of each staged tile against
//     the role filter and push the sampled positions that survive (absolute
//     text positions) into rings in shared memory, one per survivor warp;
//   - each survivor warp takes its ring's entries 32 at a time and handles the windows
//     each stands for (prefix map, then the candidate list or the hash,
//     probe and byte comparison), reading those windows from the text in
//     global memory, where the tiles passed through L2 moments before.
// Stage-1 warps never wait on memory beyond shared memory, and staged tiles
// are released as soon as stage 1 is done with them.  Every wait is bounded.
#pragma once

#include "rk_scan_kernel.cuh"

namespace rk {
namespace scan {

// A ring entry is one 64-bit word: a lane's survivors of one stage-1 round,
//   bits 57..63  the ticket's lap (ticket / ring size, mod 128),
//   bits 16..56  the buffer position of the lane's first chunk, / 16,
//   bits  0..15  its candidate mask (rf_mask16).
// A consumer waits for its ticket's lap in the slot, so a slot still holding
// the previous lap (at the start: lap -1) is never taken for its entry;
// producers write a slot only once the ring's freed count shows its previous
// lap consumed (rf_room).
constexpr uint32_t kRfLapShift = 57;

__host__ __device__ __forceinline__ uint64_t rf_lap_bits(uint32_t ticket, uint32_t rsize_log2) {
    return (uint64_t)((ticket >> rsize_log2) & 0x7Fu) << kRfLapShift;
}

// A round's candidates (bits 4n + k: position 7 - n of the lane's chunk k,
// n < 8) in 16 bits.  Step 2 (chunks k < 2): bit 2n + k.  Step 4 (4 chunks,
// positions n >= 4 only): bit 4(n - 4) + k.
template <int STEP>
__device__ __forceinline__ uint32_t rf_mask16(uint32_t m) {
    if constexpr (STEP == 2) {
        m = (m | (m >> 2)) & 0x0F0F0F0Fu;
        m = (m | (m >> 4)) & 0x00FF00FFu;
        return (m | (m >> 8)) & 0xFFFFu;
    } else {
        return m >> 16;
    }
}

// Buffer position of bit c of an entry's mask, for its first chunk at base.
template <int STEP>
__device__ __forceinline__ uint64_t rf_mask_pos(uint64_t base, uint32_t c) {
    if constexpr (STEP == 2)
        return base + 16u * 32u * (c & 1u) + 2u * (7u - (c >> 1));
    else
        return base + 16u * 32u * (c & 3u) + 4u * (3u - (c >> 2));
}

struct RfCtl {
    unsigned int s1_done;  // stage-1 warps that have finished
    unsigned int tiles;    // tiles stage-1 warp 0 has finished (progress)
    unsigned int pad[2];
};

// One ring per survivor warp, fed by the stage-1 warps w with w mod nsv
// equal to its index; its consumer finishes batches in ticket order.
struct RfRingCtl {
    unsigned int tail;     // tickets issued to the ring's producers
    unsigned int freed;    // tickets below it have been consumed
    unsigned int pad[2];
};

// Entries of each of nsv rings, log2: the largest power of two that lets
// them share the kRfRing slots.
__host__ __device__ __forceinline__ uint32_t rf_ring_log2(uint32_t nsv) {
    uint32_t r = 0;
    while ((2u << r) * nsv <= kRfRing) ++r;
    return r;
}

// Whether tickets up to ticket_end - 1 may be written into a ring of rsize
// slots: the slot of ticket t last held ticket t - rsize, consumed once freed
// is above it.
__device__ __forceinline__ bool rf_room(uint32_t ticket_end, uint32_t freed, uint32_t rsize) {
    return (int32_t)(freed + rsize - ticket_end) >= 0;
}

// Wait until ring slot `idx` holds an entry of the given lap; false if the
// wait ran out.
__device__ __forceinline__ bool rf_slot_wait(volatile uint64_t *ring, uint32_t idx, uint64_t lap,
                                             uint64_t timeout_ns, uint64_t *val) {
    uint64_t v = ring[idx];
    if ((v >> kRfLapShift) << kRfLapShift == lap) {
        *val = v;
        return true;
    }
    const uint64_t t0 = globaltimer_ns();
    for (;;) {
        __nanosleep(32);
        v = ring[idx];
        if ((v >> kRfLapShift) << kRfLapShift == lap) {
            *val = v;
            return true;
        }
        if (globaltimer_ns() - t0 > timeout_ns) return false;
    }
}

// Stage 1 of one staged tile by one stage-1 warp.  Per round a lane takes
// NCH chunks, c0 + lane + 32k (k < NCH; 16 sampled positions); successive
// rounds of the CTA's stage-1 warps step through the tile.  A chunk's last
// positions need the next chunk's roles: from the next lane (for the tile's
// last chunk, the next tile's first, read from the halo), from lane 0's next
// chunk for lane 31, and for lane 31's last chunk (which belongs to another
// warp) every second gram counts as present.  The sampled positions of
// chunks [0, nchunks) are tested; each stands for the windows up to 3
// bytes before it.  A lane with survivors in a round writes one ring entry
// (its first chunk and candidate mask); the warp reserves its entries with
// one atomic.  Returns false if a wait for a free ring slot ran out.
template <int KIND>
__device__ __forceinline__ bool rf_stage1_tile(const uint8_t *buf, uint64_t u0, uint32_t nchunks,
                                               uint32_t tile, const uint8_t *rfilt,
                                               uint32_t rshift, uint32_t side_off, uint32_t warp,
                                               uint32_t nw,
                                               uint32_t lane, volatile uint64_t *ring,
                                               RfRingCtl *rc, uint32_t rsize_log2,
                                               uint64_t timeout_ns) {
    const uint32_t rsize = 1u << rsize_log2;
    volatile RfRingCtl *vc = rc;
    constexpr int STEP = rf_step_of(KIND);
    constexpr uint32_t NCH = STEP == 2 ? 2 : 4;
    const uint8_t *side = rfilt + side_off;
    const uint32_t lane4 = lane << 2;
    constexpr uint32_t kFull = 0xffffffffu;
    const uint32_t lastc = tile / 16u;
    const uint32_t step = nw * 32u * NCH;
    const uint32_t src = (lane + 1u) & 31u;
    bool ok = true;
    uint32_t c0 = warp * 32u * NCH;
    uint4 v[NCH];
#pragma unroll
    for (uint32_t k = 0; k < NCH; ++k)
        v[k] = *reinterpret_cast<const uint4 *>(buf + 16u * min(c0 + lane + 32u * k, lastc));
    while (c0 < nchunks) {
        const uint32_t freed = vc->freed;  // read early: only a lower bound is needed
        uint4 nv[NCH];
#pragma unroll
        for (uint32_t k = 0; k < NCH; ++k)
            nv[k] = *reinterpret_cast<const uint4 *>(
                buf + 16u * min(c0 + step + lane + 32u * k, lastc));
        uint32_t v4[NCH];
        if constexpr (STEP == 2) {
#pragma unroll
            for (uint32_t k = 0; k + 1 < NCH; ++k)
                v4[k] = __shfl_sync(kFull, lane == 0 ? v[k + 1].x : v[k].x, src);
            uint32_t t = __shfl_sync(kFull, v[NCH - 1].x, src);
            if (lane == 31)
                t = *reinterpret_cast<const uint32_t *>(buf + 16u * min(c0 + 32u * NCH, lastc));
            v4[NCH - 1] = t;
        } else {
#pragma unroll
            for (uint32_t k = 0; k < NCH; ++k) v4[k] = 0;
        }
        uint32_t acc[NCH];
#pragma unroll
        for (uint32_t k = 0; k < NCH; ++k)
            acc[k] = rf_chunk<KIND>(v[k], v4[k], rfilt, rshift, side, lane4);
        uint32_t m = 0;
#pragma unroll
        for (uint32_t k = 0; k < NCH; ++k) {
            uint32_t an = __shfl_sync(kFull, (k + 1 < NCH && lane == 0) ? acc[k + 1] : acc[k], src);
            if (k + 1 == NCH && lane == 31) an = 0xFFFFFFFFu;
            const uint32_t c = c0 + lane + 32u * k;
            m |= (c < nchunks ? rf_cands<STEP>(acc[k], an) : 0u) << k;
        }
#pragma unroll
        for (uint32_t k = 0; k < NCH; ++k) v[k] = nv[k];
        const uint32_t cbase = c0 + lane;
        c0 += step;
        // one ring entry per lane with survivors in this round, the warp's
        // entries reserved with one atomic
        const uint32_t who = __ballot_sync(kFull, m != 0);
        if (who) {
            uint32_t at = 0;
            if (lane == 0) at = atomicAdd(&rc->tail, (unsigned int)__popc(who));
            at = __shfl_sync(kFull, at, 0) + __popc(who & ((1u << lane) - 1u));
            if (m) {
                if (!rf_room(at + 1u, freed, rsize)) {
                    // the ring is full: wait for its survivor warp
                    const uint64_t t0 = globaltimer_ns();
                    while (!rf_room(at + 1u, vc->freed, rsize)) {
                        __nanosleep(64);
                        if (globaltimer_ns() - t0 > timeout_ns) {
                            ok = false;  // the slot stays unwritten: its consumer gives up
                            m = 0;
                            break;
                        }
                    }
                }
                if (m)
                    ring[at & (rsize - 1u)] = rf_lap_bits(at, rsize_log2) |
                                              (((u0 >> 4) + cbase) << 16) | rf_mask16<STEP>(m);
            }
        }
    }
    return __all_sync(kFull, ok);
}

// The windows a surviving sampled position up (buffer position) stands
// for, each handled by rf_window_g: up - j for j < the step; kind 6: at a
// main position (0 mod 4) j = 0, 1 for every pattern length and j = 2, 3
// for lengths from kRfSplit on, at a side position (2 mod 4) j = 0, 1 for
// the shorter lengths.  The 16 bytes from the word at or before the first of
// them hold every window's bytes 0..7 and are read with four independent
// loads.
template <int KIND, bool DEFER>
__device__ __forceinline__ void rf_position(const WinCtx &C, const WarpCtx &w, const CandList *cc,
                                            const GText &g, uint64_t up) {
    const bool side = KIND == 6 && (up & 3u) != 0;
    const uint32_t nwin = KIND == 2 || side ? 2u : 4u;
    const uint64_t first = up >= nwin - 1 ? up - (nwin - 1) : 0;
    const uint64_t a = first & ~uint64_t(3), last = g.end - 4;
    const uint32_t *tw = reinterpret_cast<const uint32_t *>(g.base);
    uint32_t wd[4];
#pragma unroll
    for (uint32_t i = 0; i < 4; ++i) wd[i] = __ldg(tw + (min(a + 4u * i, last) >> 2));
#pragma unroll
    for (uint32_t j = 0; j < 4; ++j) {
        if (j >= nwin || up < j) continue;
        const uint64_t ua = up - j;
        const uint32_t d = (uint32_t)(ua - a);  // 0..6
        const uint32_t s8 = (d & 3u) * 8u;
        const uint32_t w0 = d >= 4 ? wd[1] : wd[0], w1 = d >= 4 ? wd[2] : wd[1],
                       w2 = d >= 4 ? wd[3] : wd[2];
        const uint64_t v8 =
            ((uint64_t)__funnelshift_r(w1, w2, s8) << 32) | __funnelshift_r(w0, w1, s8);
        const uint32_t cls = KIND != 6 ? kLenAll : side ? kLenShort : j < 2 ? kLenAll : kLenLong;
        rf_window_g<DEFER>(C, w, cc, g, ua, v8, cls);
    }
}

// A survivor warp's positions set aside: an entry's second and later
// positions wait here, so that a batch of entries costs one round trip to
// L2; they are handled 32 at a time.
struct RfXBuf {
    uint64_t *pos;   // kRfXCap buffer positions
    uint32_t *count;
};

// A survivor warp: takes its ring's entries 32 at a time (fewer only once
// every stage-1 warp has finished) until the ring is drained.  Each lane
// handles its entry's first sampled position and sets the others aside
// (handled where the set-aside buffer is full); full rounds of set-aside
// positions follow as 32 gather.  Flushes its buffered candidates (DEFER)
// or matches as they fill and at the end.  Returns false if a wait ran out.
template <int KIND, bool DEFER>
__device__ __forceinline__ bool rf_survivor_warp(const WinCtx &C, const WarpCtx &w,
                                                 const CandList *cc, const GText &g,
                                                 volatile uint64_t *ring, RfRingCtl *rc,
                                                 uint32_t rsize_log2, const RfCtl *ctl,
                                                 const RfXBuf &xb, uint32_t nw1, uint32_t lane,
                                                 uint64_t timeout_ns) {
    const uint32_t rsize = 1u << rsize_log2;
    constexpr uint32_t kFull = 0xffffffffu;
    volatile RfRingCtl *vr = rc;
    const volatile RfCtl *vc = ctl;
    bool ok = true;
    uint32_t head = 0;
    if (lane == 0) *xb.count = 0;
    __syncwarp();
    // an idle wait runs out only when the stage-1 warps make no progress
    // (no ring entry, no finished tile) for timeout_ns
    uint64_t idle_since = globaltimer_ns();
    uint32_t seen = 0xFFFFFFFFu;
    for (;;) {
        uint32_t tail = 0, done = 0, prog = 0;
        if (lane == 0) {
            done = vc->s1_done == nw1;
            __threadfence_block();
            tail = vr->tail;
            prog = vc->tiles + tail;
        }
        tail = __shfl_sync(kFull, tail, 0);
        done = __shfl_sync(kFull, done, 0);
        prog = __shfl_sync(kFull, prog, 0);
        if (prog != seen) {
            seen = prog;
            idle_since = globaltimer_ns();
        }
        const uint32_t avail = tail - head;
        // full batches of 32 while stage 1 runs (a batch costs one round trip
        // to L2 however many lanes it fills), the rest at the end
        if (avail < 32u && !(done && avail)) {
            if (done) break;  // drained
            if (globaltimer_ns() - idle_since > timeout_ns) {
                ok = false;
                break;
            }
            __nanosleep(256);
            continue;
        }
        const uint32_t got = min(avail, 32u);
        if (lane < got) {
            const uint32_t ticket = head + lane;
            uint64_t word;
            if (rf_slot_wait(ring, ticket & (rsize - 1u), rf_lap_bits(ticket, rsize_log2),
                             timeout_ns, &word)) {
                const uint64_t base = ((word >> 16) & ((1ull << (kRfLapShift - 16)) - 1ull)) << 4;
                uint32_t mask = (uint32_t)word & 0xFFFFu;
                const uint32_t c0 = __ffs(mask) - 1u;  // every entry has a candidate
                mask &= mask - 1u;
                while (mask) {  // the rest set aside (handled at once when that is full)
                    const uint32_t c = __ffs(mask) - 1u;
                    mask &= mask - 1u;
                    const uint32_t at = atomicAdd(xb.count, 1u);
                    if (at < kRfXCap) xb.pos[at] = rf_mask_pos<rf_step_of(KIND)>(base, c);
                    else rf_position<KIND, DEFER>(C, w, cc, g, rf_mask_pos<rf_step_of(KIND)>(base, c));
                }
                rf_position<KIND, DEFER>(C, w, cc, g, rf_mask_pos<rf_step_of(KIND)>(base, c0));
            } else {
                ok = false;
            }
        }
        __syncwarp();
        head += got;
        if (lane == 0) {
            __threadfence_block();  // the slots were read before they are handed back
            vr->freed = head;
            if (*xb.count > kRfXCap) *xb.count = kRfXCap;
        }
        __syncwarp();
        // set-aside positions, a full round of 32 at a time
        for (uint32_t xn = *reinterpret_cast<volatile uint32_t *>(xb.count); xn >= 32u; xn -= 32u) {
            rf_position<KIND, DEFER>(C, w, cc, g, xb.pos[xn - 32u + lane]);
            __syncwarp();
            if (lane == 0) *reinterpret_cast<volatile uint32_t *>(xb.count) = xn - 32u;
        }
        __syncwarp();
        // (a buffer that fills up mid-round sends the rest straight out)
        if (*reinterpret_cast<volatile uint32_t *>(w.mcount) >= (DEFER ? kCandBuf : kMatchCap) / 2) {
            if (DEFER) rf_cand_flush(C, w, *cc, g, lane);
            else flush(w, lane);
        }
        if (!__all_sync(kFull, ok)) break;
    }
    // the set-aside positions left
    const uint32_t xn = *reinterpret_cast<volatile uint32_t *>(xb.count);
    if (lane < xn) rf_position<KIND, DEFER>(C, w, cc, g, xb.pos[lane]);
    __syncwarp();
    if (DEFER) rf_cand_flush(C, w, *cc, g, lane);
    else flush(w, lane);
    return __all_sync(kFull, ok);
}

// MAXW: most stage-1 plus survivor warps this instance is launched with (the
// register budget follows); P.warps stage-1 warps, P.sv_warps survivor
// warps, then the producer warp.  S2S: survivor tables staged in shared
// memory.  DEFER: survivors stop after the prefix-map lookup and go to the
// candidate list (verified by rk_verify_kernel).
template <int KIND, int MAXW, bool S2S, bool DEFER>
__global__ void __launch_bounds__((MAXW + 1) * 32, 1)
    rk_scan_rf_kernel(const __grid_constant__ ScanParams P) {
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ volatile uint32_t s_abort;
    const uint32_t nw1 = P.warps, nsv = P.sv_warps;
    const RfSmemLayout lay =
        rf_smem_layout(P.tab.filter_bytes, P.s2_smem, nsv, P.stages, P.tile, P.halo);
    const uint8_t *rfilt = smem;  // offset 0: its base folds into the addresses
    uint8_t *ss2 = smem + lay.s2_off;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + lay.bar_off);
    uint64_t *empty = full + P.stages;
    volatile uint64_t *ring = reinterpret_cast<volatile uint64_t *>(smem + lay.ring_off);
    RfCtl *ctl = reinterpret_cast<RfCtl *>(smem + lay.ctl_off);
    RfRingCtl *rctl = reinterpret_cast<RfRingCtl *>(ctl + 1);
    const uint32_t rlog = rf_ring_log2(nsv), rsize = 1u << rlog;
    uint32_t *mcount = reinterpret_cast<uint32_t *>(smem + lay.mcount_off);
    uint64_t *mbuf = reinterpret_cast<uint64_t *>(smem + lay.match_off);
    uint8_t *stage0 = smem + lay.stage_off;
    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    {
        const uint4 *src = reinterpret_cast<const uint4 *>(P.tab.filter);
        uint4 *dst = reinterpret_cast<uint4 *>(smem);
        for (uint32_t i = tid; i < P.tab.filter_bytes / 16u; i += blockDim.x) dst[i] = src[i];
    }
    if (S2S) {
        const uint4 *src = reinterpret_cast<const uint4 *>(P.tab.s2_base);
        uint4 *dst = reinterpret_cast<uint4 *>(ss2);
        for (uint32_t i = tid; i < (P.s2_smem + 15u) / 16u; i += blockDim.x) dst[i] = src[i];
    }
    // every slot starts in lap -1: no consumer takes it for an entry
    for (uint32_t i = tid; i < kRfRing; i += blockDim.x) ring[i] = 0x7Full << kRfLapShift;
    if (tid < nsv) rctl[tid].tail = rctl[tid].freed = 0;
    if (tid == 0) {
        for (uint32_t s = 0; s < P.stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], nw1);
        }
        s_abort = 0;
        ctl->s1_done = ctl->tiles = 0;
        fence_mbar_init();
    }
    if (tid < nsv) mcount[tid] = 0;
    __syncthreads();

    const uint64_t my_tiles =
        P.n_tiles > blockIdx.x ? (P.n_tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;

    if (warp == nw1 + nsv) {  // ---------------- producer warp
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

    const uint64_t lo = P.mis + P.x_begin, hi = P.mis + P.x_end;
    if (warp < nw1) {  // ---------------- stage-1 warps
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
            // the chunks holding the sampled positions of this tile's windows
            // (a window belongs to the tile of its sampled position); in the
            // last tile they reach up to 1 (kind 2) or 3 bytes past its last
            // window
            const uint64_t wend = hi <= u0 + P.tile ? hi + (KIND == 2 ? 1 : 3) : u0 + P.tile;
            const uint32_t nchunks = (uint32_t)((wend - u0 + 15) / 16);
            if (!rf_stage1_tile<KIND>(buf, u0, nchunks, P.tile, rfilt, P.tab.rf_shift,
                                      P.tab.rf_side_off, warp, nw1,
                                      lane, ring + (warp % nsv) * rsize, rctl + warp % nsv, rlog,
                                      P.timeout_ns) &&
                lane == 0)
                P.info[1] = RK_ETIMEOUT;
            if (lane == 0) {
                mbar_arrive(&empty[s]);
                if (warp == 0) atomicAdd(&ctl->tiles, 1u);
            }
        }
        __syncwarp();
        if (lane == 0) {
            __threadfence_block();
            atomicAdd(&ctl->s1_done, 1u);
        }
        return;
    }

    // -------------------------------------- survivor warps
    WinCtx C;
    C.s2 = make_s2(P.tab, S2S ? ss2 : P.tab.s2_base);
    C.lo = lo;
    C.hi = hi;
    C.mis = P.mis;
    C.n = P.n;
    C.key_prefix = 0;
    C.pid_shift = RK_KEY_OFFSET_BITS;
    C.q = P.tab.q;
    C.gram_bits = P.tab.gram_bits;
    C.base_log2 = P.tab.base_log2;
    C.n_lengths = P.tab.n_lengths;
    C.smap_bits = 0;
    const uint32_t sw = warp - nw1;
    WarpCtx w{mcount + sw, mbuf + (size_t)sw * kMatchCap, P.keys, P.capacity, P.info};
    const GText g{P.base, P.n16};
    uint8_t *xraw = smem + lay.xbuf_off + sw * (kRfXCap * 8 + 16);
    const RfXBuf xb{reinterpret_cast<uint64_t *>(xraw), reinterpret_cast<uint32_t *>(xraw + kRfXCap * 8)};
    if (!rf_survivor_warp<KIND, DEFER>(C, w, &P.cand, g, ring + sw * rsize, rctl + sw, rlog, ctl,
                                       xb, nw1, lane, P.timeout_ns) &&
        lane == 0)
        P.info[1] = RK_ETIMEOUT;
}

template <int KIND, bool DEFER, int MAXW>
cudaError_t launch_rf_w(const ScanParams &p, uint32_t grid, uint32_t threads, uint32_t smem,
                        cudaStream_t st) {
    auto fn = p.s2_smem ? rk_scan_rf_kernel<KIND, MAXW, true, DEFER>
                        : rk_scan_rf_kernel<KIND, MAXW, false, DEFER>;
    // raise the dynamic shared-memory limit once per device and size
    static thread_local int seen_dev[2] = {-1, -1};
    static thread_local uint32_t seen_smem[2] = {0, 0};
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

template <int KIND, bool DEFER>
cudaError_t launch_rf_d(const ScanParams &p, uint32_t grid, uint32_t threads, uint32_t smem,
                        cudaStream_t st) {
    const uint32_t nw = p.warps + p.sv_warps;
    if (nw <= 16) return launch_rf_w<KIND, DEFER, 16>(p, grid, threads, smem, st);
    if (nw <= 24) return launch_rf_w<KIND, DEFER, 24>(p, grid, threads, smem, st);
    return launch_rf_w<KIND, DEFER, 31>(p, grid, threads, smem, st);
}

}  // namespace scan
}  // namespace rk
