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
#include "rk_internal.cuh"
#include "rk_layout.cuh"

namespace rk {
namespace {

constexpr uint64_t kWaitTimeoutNs = 4000000000ull;  // 4 s per wait

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
    uint32_t tile, stages, halo, warps, s2_smem;
};

// 8 bytes starting at any position of a 16-byte aligned shared buffer,
// little-endian (byte i of the window in bits 8i..8i+7).
__device__ __forceinline__ uint64_t ld8(const uint8_t *buf, uint32_t pos) {
    uint32_t a = pos & ~7u, s = (pos & 7u) * 8u;
    uint64_t lo = *reinterpret_cast<const uint64_t *>(buf + a);
    uint64_t hi = *reinterpret_cast<const uint64_t *>(buf + a + 8);
    return s ? (lo >> s) | (hi << (64u - s)) : lo;
}

// Rabin hash of buf[pos .. pos+L) mod 2^61-1 with B = 2^k.
__device__ __forceinline__ uint64_t window_hash(const uint8_t *buf, uint32_t pos, uint32_t L,
                                               uint32_t k) {
    if (k == 8) {
        // 8-byte blocks: the block's big-endian value, and 256^8 = 2^64 = 2^3 (mod p).
        uint32_t r = ((L - 1u) & 7u) + 1u;  // leading partial block, 1..8 bytes
        uint64_t h = fold61(bswap64(ld8(buf, pos)) >> (64u - 8u * r));
        for (uint32_t i = r; i < L; i += 8)
            h = addmod61(rotl61(h, 3), fold61(bswap64(ld8(buf, pos + i))));
        return h;
    }
    uint64_t h = 0;
    for (uint32_t i = 0; i < L; ++i) {
        h = rotl61(h, k) + buf[pos + i];
        if (h >= kP61) h -= kP61;
    }
    return h;
}

// pat: 8-byte aligned, zero padded to a multiple of 8 (shared or global).
__device__ __forceinline__ bool verify(const uint8_t *buf, uint32_t pos, const uint8_t *pat,
                                       uint32_t L) {
    for (uint32_t i = 0; i < L; i += 8) {
        uint64_t d = ld8(buf, pos + i) ^ *reinterpret_cast<const uint64_t *>(pat + i);
        uint32_t rem = L - i;
        if (rem < 8) d &= (1ull << (8u * rem)) - 1ull;
        if (d) return false;
    }
    return true;
}

// Survivor-stage tables, as generic pointers into shared or global memory.
struct S2 {
    const GramSlot *grams;
    const uint32_t *gram_lens;
    const uint2 *group_hdr;
    const GroupSlot *slots;
    const uint32_t *group_pids;
    const uint8_t *pbytes;
    const uint64_t *poff;
    const uint32_t *lengths;
};

template <class T>
__device__ __forceinline__ const T *rebase(const T *p, const uint8_t *from, const uint8_t *to) {
    return reinterpret_cast<const T *>(to + (reinterpret_cast<const uint8_t *>(p) - from));
}

struct WarpCtx {
    uint32_t *mcount;  // this warp's buffered-match counter
    uint64_t *mbuf;    // this warp's match buffer
    uint64_t *keys;
    uint64_t capacity;
    unsigned long long *info;
};

__device__ __forceinline__ void emit(const WarpCtx &w, uint64_t key) {
    uint32_t s = atomicAdd(w.mcount, 1u);
    if (s < kMatchCap) {
        w.mbuf[s] = key;
    } else {  // buffer full: append directly
        unsigned long long g = atomicAdd(&w.info[0], 1ull);
        if (g < w.capacity) w.keys[g] = key;
    }
}

// Warp-converged: move the buffered matches to the output with one atomic.
__device__ __forceinline__ void flush(const WarpCtx &w, uint32_t lane) {
    __syncwarp();
    uint32_t cnt = min(*reinterpret_cast<volatile uint32_t *>(w.mcount), kMatchCap);
    if (cnt) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(&w.info[0], (unsigned long long)cnt);
        base = __shfl_sync(0xffffffffu, base, 0);
        for (uint32_t i = lane; i < cnt; i += 32)
            if (base + i < w.capacity) w.keys[base + i] = w.mbuf[i];
    }
    __syncwarp();
    if (lane == 0) *reinterpret_cast<volatile uint32_t *>(w.mcount) = 0;
    __syncwarp();
}

// Probe the length-L group with the window's hash; verify and emit.
__device__ __forceinline__ void probe_length(const S2 &s2, uint32_t base_log2, const WarpCtx &w,
                                             const uint8_t *buf, uint32_t pos, uint64_t x,
                                             uint32_t L) {
    const uint2 hdr = s2.group_hdr[L];
    if (hdr.y == 0) return;
    const uint64_t h = window_hash(buf, pos, L, base_log2);
    const uint64_t mask = (1ull << hdr.y) - 1ull;
    uint64_t idx = (h * kGroupMult) >> (64u - hdr.y);
    for (;;) {
        const GroupSlot s = s2.slots[hdr.x + idx];
        if (s.count == 0) return;
        if (s.h == h) {
            for (uint32_t j = 0; j < s.count; ++j) {
                const uint32_t pid = s2.group_pids[s.first + j];
                if (verify(buf, pos, s2.pbytes + s2.poff[pid], L))
                    emit(w, ((uint64_t)pid << RK_KEY_OFFSET_BITS) | x);
            }
            return;
        }
        idx = (idx + 1) & mask;
    }
}

// Stage 2 for one window at buffer position pos.
template <int MODE>
__device__ __forceinline__ void process_window(const ScanParams &P, const S2 &s2,
                                               const WarpCtx &w, const uint8_t *buf,
                                               uint32_t pos, uint64_t u0) {
    const uint64_t ua = u0 + pos;
    if (ua < P.mis + P.x_begin || ua >= P.mis + P.x_end) return;
    const uint64_t x = ua - P.mis;
    const DevTable &T = P.tab;
    if (MODE == kFilterNone) {
        for (uint32_t i = 0; i < T.n_lengths; ++i) {
            const uint32_t L = s2.lengths[i];
            if (x + L > P.n) break;
            probe_length(s2, T.base_log2, w, buf, pos, x, L);
        }
        return;
    }
    const uint64_t v = ld8(buf, pos);  // window bytes 0..7, little-endian
    const uint32_t key = T.q == 4 ? (uint32_t)v : (uint32_t)v & ((1u << (8u * T.q)) - 1u);
    const uint32_t gmask = (1u << T.gram_bits) - 1u;
    uint32_t idx = (key * kGramMult) >> (32u - T.gram_bits);
    for (;;) {
        const GramSlot g = s2.grams[idx];
        if (g.count == 0) return;  // a false positive of the bit set
        if (g.key == key) {
            // patterns of length >= q + 4 need bytes q..q+3 in the fingerprint set
            const bool ext_ok = (g.ext >> ext_bit((uint32_t)(v >> (8u * T.q)))) & 1u;
            for (uint32_t j = 0; j < g.count; ++j) {
                const uint32_t L = s2.gram_lens[g.first + j];
                if (x + L > P.n) break;  // lengths ascend
                if (L >= T.q + 4 && !ext_ok) break;
                probe_length(s2, T.base_log2, w, buf, pos, x, L);
            }
            return;
        }
        idx = (idx + 1) & gmask;
    }
}

// Stage 1 for one 16-byte chunk, given its words v and the next chunk's first
// word v4: bit (15 - j) of the result is set when window j may start a match.
template <int MODE, bool Q4>
__device__ __forceinline__ uint32_t stage1(const uint4 v, const uint32_t v4, const uint8_t *sfilt,
                                           uint32_t fmask, uint32_t lane4, uint32_t qmask) {
    if (MODE == kFilterNone) return 0xFFFFu;
    const uint32_t wd[5] = {v.x, v.y, v.z, v.w, v4};
    // four independent 4-bit accumulators keep the dependency chains short
    uint32_t acc[4] = {0, 0, 0, 0};
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        // bytes j..j+3 of the chunk as a little-endian word: the window's prefix
        uint32_t g = (j & 3) == 0 ? wd[j >> 2]
                                  : __funnelshift_r(wd[j >> 2], wd[(j >> 2) + 1], 8 * (j & 3));
        if (!Q4) g &= qmask;
        const uint32_t hh = __umulhi(g, kFilterMult);
        const uint32_t a = MODE == kFilterReplicated ? ((hh & fmask) | lane4) : ((hh >> 3) & fmask);
        const uint32_t word = *reinterpret_cast<const uint32_t *>(sfilt + a);
        const uint32_t rot = __funnelshift_r(word, word, hh);  // bucket bit -> bit 31
        acc[j >> 2] = __funnelshift_l(rot, acc[j >> 2], 1);    // acc = acc << 1 | bit
    }
    return (acc[0] << 12) | (acc[1] << 8) | (acc[2] << 4) | acc[3];
}

struct Chunk {
    uint4 v;
    uint32_t v4;
};

// Words of chunk c (clamped into the tile so the read stays in its buffer).
__device__ __forceinline__ Chunk load_chunk(const uint8_t *buf, uint32_t c, uint32_t last) {
    c = min(c, last);
    Chunk k;
    k.v = *reinterpret_cast<const uint4 *>(buf + 16u * c);
    k.v4 = *reinterpret_cast<const uint32_t *>(buf + 16u * c + 16u);
    return k;
}

// MAXW: most consumer warps this instance is launched with; the register
// budget per thread follows from (MAXW + 1) warps per SM.  S2S: the
// survivor-stage tables are staged in shared memory (their loads then
// compile to shared-memory loads).
template <int MODE, bool Q4, int MAXW, bool S2S>
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
        if (lane != 0) return;
        uint64_t issued = 0;
        for (uint64_t i = 0; i < my_tiles; ++i) {
            const uint32_t s = (uint32_t)(i % P.stages);
            if (i >= P.stages &&
                !mbar_wait_bounded(&empty[s], (uint32_t)((i / P.stages) + 1) & 1u, kWaitTimeoutNs)) {
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
            mbar_wait_bounded(&full[i % P.stages], (uint32_t)(i / P.stages) & 1u, kWaitTimeoutNs);
        return;
    }

    // -------------------------------------- consumer warps
    S2 s2;
    {
        const DevTable &T = P.tab;
        const uint8_t *from = T.s2_base;
        const uint8_t *to = S2S ? ss2 : T.s2_base;
        s2.grams = rebase(T.grams, from, to);
        s2.gram_lens = rebase(T.gram_lens, from, to);
        s2.group_hdr = rebase(T.group_hdr, from, to);
        s2.slots = rebase(T.slots, from, to);
        s2.group_pids = rebase(T.group_pids, from, to);
        s2.pbytes = rebase(T.pbytes, from, to);
        s2.poff = rebase(T.poff, from, to);
        s2.lengths = rebase(T.lengths, from, to);
    }
    uint16_t *q = queues + warp * kQueueCap;
    WarpCtx w{mcount + warp, mbuf + (size_t)warp * kMatchCap, P.keys, P.capacity, P.info};
    const uint32_t lane4 = lane << 2;
    const uint32_t fmask = P.tab.filter_mask;
    const uint32_t qmask = P.tab.q == 4 ? 0xFFFFFFFFu : (1u << (8u * P.tab.q)) - 1u;

    for (uint64_t i = 0; i < my_tiles; ++i) {
        const uint32_t s = (uint32_t)(i % P.stages);
        if (!mbar_wait_bounded(&full[s], (uint32_t)(i / P.stages) & 1u, kWaitTimeoutNs)) {
            s_abort = 1;
            P.info[1] = RK_ETIMEOUT;
            break;
        }
        const uint8_t *buf = stage0 + (size_t)s * lay.stage_stride;
        const uint64_t t = blockIdx.x + i * gridDim.x;
        const uint64_t u0 = P.u_first + t * P.tile;
        const uint64_t wend = min(u0 + P.tile, P.mis + P.x_end);
        const uint32_t nchunks = (uint32_t)((wend - u0 + 15) / 16);

        uint32_t qn = 0;  // warp-uniform queue length (< 32 between rounds)
        // Each lane takes chunks c0 + lane and c0 + 32 + lane (32 windows);
        // the next pair's words are loaded before this pair is tested.
        const uint32_t last = P.tile / 16u - 1u;
        const uint32_t step = nw * 64u;
        uint32_t c0 = warp * 64u;
        Chunk ka = load_chunk(buf, c0 + lane, last), kb = load_chunk(buf, c0 + 32u + lane, last);
        while (c0 < nchunks) {
            const uint32_t ca = c0 + lane, cb = c0 + 32u + lane;
            const Chunk na = load_chunk(buf, ca + step, last), nb = load_chunk(buf, cb + step, last);
            uint32_t m = 0;
            if (ca < nchunks) m = stage1<MODE, Q4>(ka.v, ka.v4, sfilt, fmask, lane4, qmask);
            if (cb < nchunks) m |= stage1<MODE, Q4>(kb.v, kb.v4, sfilt, fmask, lane4, qmask) << 16;
            ka = na;
            kb = nb;
            c0 += step;
            if (__ballot_sync(0xffffffffu, m != 0) == 0) continue;
            // bit b of m: window 15 - (b & 15) of chunk (b < 16 ? ca : cb)
            const uint32_t cnt = __popc(m);
            uint32_t incl = cnt;
#pragma unroll
            for (uint32_t d = 1; d < 32; d <<= 1) {
                const uint32_t o = __shfl_up_sync(0xffffffffu, incl, d);
                if (lane >= d) incl += o;
            }
            const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
            if (qn + total <= kQueueCap) {
                uint32_t at = qn + incl - cnt;
                while (m) {
                    const uint32_t b = 31u - __clz(m);
                    m &= ~(1u << b);
                    q[at++] = (uint16_t)(16u * (b < 16 ? ca : cb) + (15u - (b & 15u)));
                }
                qn += total;
                __syncwarp();
                // full rounds: one queued window per lane
                while (qn >= 32) {
                    qn -= 32;
                    process_window<MODE>(P, s2, w, buf, q[qn + lane], u0);
                    __syncwarp();
                    if (*reinterpret_cast<volatile uint32_t *>(w.mcount) >= kMatchCap - 32)
                        flush(w, lane);
                }
            } else {
                // more survivors than the queue holds (very dense matches):
                // each lane works through its own
                while (m) {
                    const uint32_t b = 31u - __clz(m);
                    m &= ~(1u << b);
                    process_window<MODE>(P, s2, w, buf,
                                         16u * (b < 16 ? ca : cb) + (15u - (b & 15u)), u0);
                }
                flush(w, lane);
            }
        }
        if (lane < qn) process_window<MODE>(P, s2, w, buf, q[lane], u0);
        flush(w, lane);
        if (lane == 0) mbar_arrive(&empty[s]);
    }
    flush(w, lane);
}

template <int MODE, bool Q4, int MAXW>
cudaError_t launch_w(const ScanParams &p, uint32_t grid, uint32_t threads, uint32_t smem,
                     cudaStream_t st) {
    auto fn = p.s2_smem ? rk_scan_tiles_kernel<MODE, Q4, MAXW, true>
                        : rk_scan_tiles_kernel<MODE, Q4, MAXW, false>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    fn<<<grid, threads, smem, st>>>(p);
    return cudaGetLastError();
}

template <int MODE, bool Q4>
cudaError_t launch_one(const ScanParams &p, uint32_t grid, uint32_t threads, uint32_t smem,
                       cudaStream_t st) {
    if (p.warps <= 8) return launch_w<MODE, Q4, 8>(p, grid, threads, smem, st);
    if (p.warps <= 16) return launch_w<MODE, Q4, 16>(p, grid, threads, smem, st);
    return launch_w<MODE, Q4, 31>(p, grid, threads, smem, st);
}

}  // namespace

int launch_scan(const rk_table *t, const uint8_t *d_text, uint64_t n, uint64_t x_begin,
                uint64_t x_end, uint64_t *d_keys, uint64_t capacity, uint64_t *d_info,
                cudaStream_t stream) {
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
    p.n_tiles = (p.mis + x_end - p.u_first + tu.tile_bytes - 1) / tu.tile_bytes;
    p.keys = d_keys;
    p.capacity = capacity;
    p.info = reinterpret_cast<unsigned long long *>(d_info);
    p.tile = tu.tile_bytes;
    p.stages = tu.stages;
    p.halo = tu.halo;
    p.warps = tu.warps;
    p.s2_smem = tu.s2_smem;
    uint64_t max_ctas = (uint64_t)t->sm_count * tu.ctas_per_sm;
    uint32_t grid = (uint32_t)(p.n_tiles < max_ctas ? p.n_tiles : max_ctas);
    uint32_t threads = (tu.warps + 1) * 32;
    bool q4 = t->dev.q == 4;
    cudaError_t e;
    switch (t->dev.filter_mode) {
        case kFilterNone:
            e = q4 ? launch_one<kFilterNone, true>(p, grid, threads, tu.smem_bytes, stream)
                   : launch_one<kFilterNone, false>(p, grid, threads, tu.smem_bytes, stream);
            break;
        case kFilterReplicated:
            e = q4 ? launch_one<kFilterReplicated, true>(p, grid, threads, tu.smem_bytes, stream)
                   : launch_one<kFilterReplicated, false>(p, grid, threads, tu.smem_bytes, stream);
            break;
        default:
            e = q4 ? launch_one<kFilterFlat, true>(p, grid, threads, tu.smem_bytes, stream)
                   : launch_one<kFilterFlat, false>(p, grid, threads, tu.smem_bytes, stream);
            break;
    }
    return e == cudaSuccess ? RK_OK : RK_ECUDA;
}

}  // namespace rk
