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
//  A2 hash    every window's Rabin hash at the prefix length q (q = min(4,
//             shortest pattern)) is its big-endian q-byte value (B = 256,
//             256^q < 2^61 - 1), obtained from registers by one byte permute;
//             it is tested against a shared-memory bit set of the patterns'
//             prefix hashes.  Windows that pass (and only those) get the
//             full-length Rabin hash mod 2^61 - 1 for each pattern length
//             that starts with their prefix.
//  A3 probe   that hash is looked up in the table of its length group.
//  A4 verify  each pattern of the matching slot is compared byte for byte
//             (Section 3.1's compare(P, T + x, m) after hx == hy).
//  A5 emit    matches collect in a per-warp shared buffer and are appended
//             to the output with one atomic per warp flush.
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
    uint32_t tile, stages, halo, warps;
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

__device__ __forceinline__ bool verify(const uint8_t *buf, uint32_t pos, const uint8_t *pat,
                                       uint32_t L) {
    for (uint32_t i = 0; i < L; i += 8) {
        uint64_t d = ld8(buf, pos + i) ^ __ldg(reinterpret_cast<const uint64_t *>(pat + i));
        uint32_t rem = L - i;
        if (rem < 8) d &= (1ull << (8u * rem)) - 1ull;
        if (d) return false;
    }
    return true;
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
__device__ __forceinline__ void probe_length(const ScanParams &P, const WarpCtx &w,
                                             const uint8_t *buf, uint32_t pos, uint64_t x,
                                             uint32_t L) {
    const DevTable &T = P.tab;
    uint2 hdr = __ldg(&T.group_hdr[L]);
    if (hdr.y == 0) return;
    uint64_t h = window_hash(buf, pos, L, T.base_log2);
    uint64_t mask = (1ull << hdr.y) - 1ull;
    uint64_t idx = (h * kGroupMult) >> (64u - hdr.y);
    for (;;) {
        const GroupSlot *s = &T.slots[hdr.x + idx];
        uint32_t cnt = __ldg(&s->count);
        if (cnt == 0) return;
        if (__ldg(&s->h) == h) {
            uint32_t first = __ldg(&s->first);
            for (uint32_t j = 0; j < cnt; ++j) {
                uint32_t pid = __ldg(&T.group_pids[first + j]);
                if (verify(buf, pos, T.pbytes + __ldg(&T.poff[pid]), L))
                    emit(w, ((uint64_t)pid << RK_KEY_OFFSET_BITS) | x);
            }
            return;
        }
        idx = (idx + 1) & mask;
    }
}

// Stage 2 for one window at buffer position pos.
template <int MODE>
__device__ __forceinline__ void process_window(const ScanParams &P, const WarpCtx &w,
                                               const uint8_t *buf, uint32_t pos, uint64_t u0) {
    uint64_t ua = u0 + pos;
    if (ua < P.mis + P.x_begin || ua >= P.mis + P.x_end) return;
    uint64_t x = ua - P.mis;
    const DevTable &T = P.tab;
    if (MODE == kFilterNone) {
        for (uint32_t i = 0; i < T.n_lengths; ++i) {
            uint32_t L = __ldg(&T.lengths[i]);
            if (x + L > P.n) break;
            probe_length(P, w, buf, pos, x, L);
        }
        return;
    }
    uint32_t key = (uint32_t)(bswap64(ld8(buf, pos)) >> (64u - 8u * T.q));
    uint32_t gmask = (1u << T.gram_bits) - 1u;
    uint32_t idx = (key * kGramMult) >> (32u - T.gram_bits);
    for (;;) {
        const GramSlot *g = &T.grams[idx];
        uint32_t cnt = __ldg(&g->count);
        if (cnt == 0) return;  // a false positive of the bit set
        if (__ldg(&g->key) == key) {
            uint32_t first = __ldg(&g->first);
            for (uint32_t j = 0; j < cnt; ++j) {
                uint32_t L = __ldg(&T.gram_lens[first + j]);
                if (x + L > P.n) break;  // lengths ascend
                probe_length(P, w, buf, pos, x, L);
            }
            return;
        }
        idx = (idx + 1) & gmask;
    }
}

// Stage 1 for one 16-byte chunk: bit (15 - j) of the result is set when
// window j of the chunk may start a match.
template <int MODE, bool Q4>
__device__ __forceinline__ uint32_t stage1(const uint8_t *buf, uint32_t c, const uint8_t *sfilt,
                                           uint32_t fmask, uint32_t lane4, uint32_t qshift) {
    if (MODE == kFilterNone) return 0xFFFFu;
    const uint4 v = *reinterpret_cast<const uint4 *>(buf + 16u * c);
    const uint32_t v4 = *reinterpret_cast<const uint32_t *>(buf + 16u * c + 16u);
    const uint32_t wd[5] = {v.x, v.y, v.z, v.w, v4};
    uint32_t m = 0;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        // big-endian bytes j..j+3 of the chunk: the window's q-byte prefix
        const uint32_t sel = (j & 3) == 0 ? 0x0123u : (j & 3) == 1 ? 0x1234u
                             : (j & 3) == 2 ? 0x2345u : 0x3456u;
        uint32_t g = __byte_perm(wd[j >> 2], wd[(j >> 2) + 1], sel);
        if (!Q4) g >>= qshift;
        const uint32_t hh = __umulhi(g, kFilterMult);
        uint32_t a = MODE == kFilterReplicated ? ((hh & fmask) | lane4) : ((hh >> 3) & fmask);
        const uint32_t word = *reinterpret_cast<const uint32_t *>(sfilt + a);
        const uint32_t rot = __funnelshift_r(word, word, hh);  // bucket bit -> bit 31
        m = __funnelshift_l(rot, m, 1);                        // m = m << 1 | bit
    }
    return m;
}

template <int MODE, bool Q4>
__global__ void __launch_bounds__(1024, 1) rk_scan_tiles_kernel(const __grid_constant__ ScanParams P) {
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ volatile uint32_t s_abort;
    const SmemLayout lay = smem_layout(P.tab.filter_bytes, P.warps, P.stages, P.tile, P.halo);
    uint8_t *sfilt = smem + lay.filter_off;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + lay.bar_off);
    uint64_t *empty = full + P.stages;
    uint32_t *queues = reinterpret_cast<uint32_t *>(smem + lay.queue_off);
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
    uint32_t *q = queues + warp * kQueueCap;
    WarpCtx w{mcount + warp, mbuf + (size_t)warp * kMatchCap, P.keys, P.capacity, P.info};
    const uint32_t lane4 = lane << 2;
    const uint32_t fmask = P.tab.filter_mask;
    const uint32_t qshift = 8u * (4u - P.tab.q);
    const uint32_t lt_mask = (1u << lane) - 1u;

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

        uint32_t qn = 0;  // warp-uniform queue length
        auto drain = [&]() {
            __syncwarp();
            for (uint32_t e = lane; e < qn; e += 32) {
                const uint32_t ent = q[e];
                const uint32_t c = ent >> 16;
                uint32_t m = ent & 0xFFFFu;
                while (m) {
                    const uint32_t b = 31u - __clz(m);
                    m &= ~(1u << b);
                    process_window<MODE>(P, w, buf, 16u * c + (15u - b), u0);
                }
            }
            qn = 0;
            flush(w, lane);
        };

        for (uint32_t c0 = warp * 32; c0 < nchunks; c0 += nw * 32) {
            const uint32_t c = c0 + lane;
            uint32_t m = 0;
            if (c < nchunks) m = stage1<MODE, Q4>(buf, c, sfilt, fmask, lane4, qshift);
            const uint32_t bal = __ballot_sync(0xffffffffu, m != 0);
            if (bal) {
                const uint32_t cnt = __popc(bal);
                if (qn + cnt > kQueueCap) drain();
                if (m) q[qn + __popc(bal & lt_mask)] = (c << 16) | m;
                qn += cnt;
                if (qn >= 32) drain();
            }
        }
        if (qn) drain();
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
    }
    flush(w, lane);
}

template <int MODE, bool Q4>
cudaError_t launch_one(const ScanParams &p, uint32_t grid, uint32_t threads, uint32_t smem,
                       cudaStream_t st) {
    auto fn = rk_scan_tiles_kernel<MODE, Q4>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    fn<<<grid, threads, smem, st>>>(p);
    return cudaGetLastError();
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
