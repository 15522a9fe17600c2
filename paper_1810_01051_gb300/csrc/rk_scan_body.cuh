// Device code that processes one staged text tile: the per-window prefilter
// (stage 1), the per-warp survivor queue, and for survivors the Rabin hash
// mod 2^61 - 1 at each candidate pattern length (A2), the probe of that
// length's table (A3), the byte comparison (A4) and buffered emission (A5).
// Shared by the single-text scan kernel and the batch kernel.
#pragma once

#include "rk_internal.cuh"
#include "rk_layout.cuh"

namespace rk {

// 8 bytes starting at any position of a 16-byte aligned shared buffer,
// little-endian (byte i of the window in bits 8i..8i+7): three aligned words
// and two funnel shifts (reads at most 4 bytes past the 8).
__device__ __forceinline__ uint64_t ld8(const uint8_t *buf, uint32_t pos) {
    const uint32_t *w = reinterpret_cast<const uint32_t *>(buf + (pos & ~3u));
    const uint32_t s = (pos & 3u) * 8u;
    const uint32_t w0 = w[0], w1 = w[1], w2 = w[2];
    const uint32_t lo = __funnelshift_r(w0, w1, s), hi = __funnelshift_r(w1, w2, s);
    return ((uint64_t)hi << 32) | lo;
}

__device__ __forceinline__ uint32_t ld1(const uint8_t *buf, uint32_t pos) { return buf[pos]; }

// The text in global memory, for windows read outside a staged tile:
// positions from a 16-byte aligned base; words at or past `end` (the text
// end rounded up to 16 bytes) are never read.
struct GText {
    const uint8_t *base;
    uint64_t end;
};

// As above from global memory.  A word starting at or past `end` holds no
// text byte; the last word before `end` is read in its place (those bytes
// lie past the window, and every caller masks or ignores them).
__device__ __forceinline__ uint64_t ld8(const GText &g, uint64_t pos) {
    const uint64_t a = pos & ~uint64_t(3), last = g.end - 4;
    const uint32_t *w = reinterpret_cast<const uint32_t *>(g.base);
    const uint32_t w0 = __ldg(w + (min(a, last) >> 2)), w1 = __ldg(w + (min(a + 4, last) >> 2)),
                   w2 = __ldg(w + (min(a + 8, last) >> 2));
    const uint32_t s = (uint32_t)(pos & 3u) * 8u;
    const uint32_t lo = __funnelshift_r(w0, w1, s), hi = __funnelshift_r(w1, w2, s);
    return ((uint64_t)hi << 32) | lo;
}

__device__ __forceinline__ uint32_t ld1(const GText &g, uint64_t pos) { return __ldg(g.base + pos); }

// A listed window: its first 8 bytes came with the candidate, anything else
// is read from the text.
struct WText {
    GText g;
    uint64_t pos0;    // the window's position
    uint64_t first8;  // bytes pos0 .. pos0 + 7, little-endian
};

__device__ __forceinline__ uint64_t ld8(const WText &w, uint64_t pos) {
    return pos == w.pos0 ? w.first8 : ld8(w.g, pos);
}

__device__ __forceinline__ uint32_t ld1(const WText &w, uint64_t pos) {
    const uint64_t d = pos - w.pos0;
    return d < 8 ? (uint32_t)(w.first8 >> (8u * d)) & 0xFFu : ld1(w.g, pos);
}

// Rabin hash of src[pos .. pos+L) mod 2^61-1 with B = 2^k.
template <class Src, class Pos>
__device__ __forceinline__ uint64_t window_hash(const Src &src, Pos pos, uint32_t L, uint32_t k) {
    if (k == 8) {
        // 8-byte blocks: the block's big-endian value, and 256^8 = 2^64 = 2^3 (mod p).
        uint32_t r = ((L - 1u) & 7u) + 1u;  // leading partial block, 1..8 bytes
        uint64_t h = fold61(bswap64(ld8(src, pos)) >> (64u - 8u * r));
        for (uint32_t i = r; i < L; i += 8)
            h = addmod61(rotl61(h, 3), fold61(bswap64(ld8(src, pos + i))));
        return h;
    }
    uint64_t h = 0;
    for (uint32_t i = 0; i < L; ++i) {
        h = rotl61(h, k) + ld1(src, pos + i);
        if (h >= kP61) h -= kP61;
    }
    return h;
}

// pat: 8-byte aligned, zero padded to a multiple of 8 (shared or global).
template <class Src, class Pos>
__device__ __forceinline__ bool verify(const Src &src, Pos pos, const uint8_t *pat, uint32_t L) {
    for (uint32_t i = 0; i < L; i += 8) {
        uint64_t d = ld8(src, pos + i) ^ *reinterpret_cast<const uint64_t *>(pat + i);
        uint32_t rem = L - i;
        if (rem < 8) d &= (1ull << (8u * rem)) - 1ull;
        if (d) return false;
    }
    return true;
}

// Survivor-stage tables, as pointers into shared or global memory.
struct S2 {
    const GramSlot *grams;
    const uint32_t *gram_lens;
    const uint2 *group_hdr;
    const GroupSlot *slots;
    const uint32_t *group_pids;
    const uint8_t *pbytes;
    const uint64_t *poff;
    const uint32_t *lengths;
    const SampSlot *smap;  // sampled tables only
};

template <class T>
__device__ __forceinline__ const T *rebase(const T *p, const uint8_t *from, const uint8_t *to) {
    return reinterpret_cast<const T *>(to + (reinterpret_cast<const uint8_t *>(p) - from));
}

// The survivor tables of `T`, moved to `to` when they were copied there.
__device__ __forceinline__ S2 make_s2(const DevTable &T, const uint8_t *to) {
    S2 s;
    const uint8_t *from = T.s2_base;
    s.grams = rebase(T.grams, from, to);
    s.gram_lens = rebase(T.gram_lens, from, to);
    s.group_hdr = rebase(T.group_hdr, from, to);
    s.slots = rebase(T.slots, from, to);
    s.group_pids = rebase(T.group_pids, from, to);
    s.pbytes = rebase(T.pbytes, from, to);
    s.poff = rebase(T.poff, from, to);
    s.lengths = rebase(T.lengths, from, to);
    s.smap = rebase(T.smap, from, to);
    return s;
}

// What the survivor stage needs to know about the text being scanned.
struct WinCtx {
    S2 s2;
    uint64_t lo, hi;      // buffer positions (from the aligned base) of the windows scanned
    uint64_t mis;         // buffer position of text byte 0
    uint64_t n;           // text length
    uint64_t key_prefix;  // or-ed into every key
    uint32_t pid_shift;   // bit position of the pattern id in a key
    uint32_t q, gram_bits, base_log2, n_lengths;
    uint32_t smap_bits;   // sampled tables: sample map size (log2 slots)
};

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

// A match appended straight to the output (one global atomic).
__device__ __forceinline__ void emit_global(const WarpCtx &w, uint64_t key) {
    const unsigned long long g = atomicAdd(&w.info[0], 1ull);
    if (g < w.capacity) w.keys[g] = key;
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

// Probe the length-L group with the window's hash; verify and emit (DIRECT:
// straight to the output, not through the warp's buffer).
template <bool DIRECT = false, class Src, class Pos>
__device__ __forceinline__ void probe_length(const WinCtx &C, const WarpCtx &w, const Src &buf,
                                             Pos pos, uint64_t x, uint32_t L) {
    const uint2 hdr = C.s2.group_hdr[L];
    if (hdr.y == 0) return;
    const uint64_t h = window_hash(buf, pos, L, C.base_log2);
    const uint64_t mask = (1ull << hdr.y) - 1ull;
    uint64_t idx = (h * kGroupMult) >> (64u - hdr.y);
    for (;;) {
        const GroupSlot s = C.s2.slots[hdr.x + idx];
        if (s.count == 0) return;
        if (s.h == h) {
            for (uint32_t j = 0; j < s.count; ++j) {
                const uint32_t pid = C.s2.group_pids[s.first + j];
                if (verify(buf, pos, C.s2.pbytes + C.s2.poff[pid], L)) {
                    const uint64_t key = C.key_prefix | ((uint64_t)pid << C.pid_shift) | x;
                    if (DIRECT) emit_global(w, key);
                    else emit(w, key);
                }
            }
            return;
        }
        idx = (idx + 1) & mask;
    }
}

// Stage 2 for one window at buffer position pos of the tile starting at u0.
template <int MODE>
__device__ __forceinline__ void process_window(const WinCtx &C, const WarpCtx &w,
                                               const uint8_t *buf, uint32_t pos, uint64_t u0) {
    const uint64_t ua = u0 + pos;
    if (ua < C.lo || ua >= C.hi) return;
    const uint64_t x = ua - C.mis;
    if (MODE == kFilterNone) {
        for (uint32_t i = 0; i < C.n_lengths; ++i) {
            const uint32_t L = C.s2.lengths[i];
            if (x + L > C.n) break;
            probe_length(C, w, buf, pos, x, L);
        }
        return;
    }
    const uint64_t v = ld8(buf, pos);  // window bytes 0..7, little-endian
    const uint32_t key = C.q == 4 ? (uint32_t)v : (uint32_t)v & ((1u << (8u * C.q)) - 1u);
    const uint32_t gmask = (1u << C.gram_bits) - 1u;
    uint32_t idx = (key * kGramMult) >> (32u - C.gram_bits);
    for (;;) {
        const GramSlot g = C.s2.grams[idx];
        if (g.count == 0) return;  // a false positive of the bit set
        if (g.key == key) {
            // patterns of length >= q + 4 need bytes q..q+3 in the fingerprint set
            const bool ext_ok = (g.ext >> ext_bit((uint32_t)(v >> (8u * C.q)))) & 1u;
            if (!ext_ok && !(g.count & kGramShort)) return;  // every length is >= q + 4
            const uint32_t cnt = g.count & ~kGramShort;
            for (uint32_t j = 0; j < cnt; ++j) {
                const uint32_t L = C.s2.gram_lens[g.first + j];
                if (x + L > C.n) break;  // lengths ascend
                if (L >= C.q + 4 && !ext_ok) break;
                probe_length(C, w, buf, pos, x, L);
            }
            return;
        }
        idx = (idx + 1) & gmask;
    }
}

// Deferred verification (filtered modes).  Stage 2a below only finds the
// prefix-map slot whose lengths apply to a window; the candidate {offset |
// slot << 40, window bytes 0..7} goes to a global list, and a separate
// kernel hashes, probes and verifies the whole list 32 candidates per warp
// (rk_verify.cu), reading longer windows' other bytes from the text.  With a
// role filter's side table a candidate also carries a length class.
constexpr uint32_t kCandSlotShift = 40;          // text offsets are below 2^40
constexpr uint32_t kCandClassShift = 62;         // slots are below 2^22: two bits for a class
constexpr uint64_t kCandSlotMask = (1ull << (kCandClassShift - kCandSlotShift)) - 1ull;

// Pattern-length class of a window: every length, or only those from
// kRfSplit on, or only those below it (a role filter with a side table finds
// the two kinds of a window through different sampled positions).
enum LenClass : uint32_t { kLenAll = 0, kLenLong = 1, kLenShort = 2 };
constexpr uint32_t kRfSplit = 7;

__device__ __forceinline__ bool len_in_class(uint32_t L, uint32_t cls) {
    return cls == kLenAll || ((L >= kRfSplit) == (cls == kLenLong));
}

// A candidate's parts: text offset, prefix-map slot, length class.
__device__ __forceinline__ uint64_t cand_x(uint64_t e) {
    return e & ((1ull << kCandSlotShift) - 1ull);
}
__device__ __forceinline__ uint32_t cand_slot(uint64_t e) {
    return (uint32_t)((e >> kCandSlotShift) & kCandSlotMask);
}
__device__ __forceinline__ uint32_t cand_class(uint64_t e) { return (uint32_t)(e >> kCandClassShift); }
__device__ __forceinline__ uint64_t cand_pack(uint64_t x, uint32_t slot, uint32_t cls) {
    return x | ((uint64_t)slot << kCandSlotShift) | ((uint64_t)cls << kCandClassShift);
}
constexpr uint32_t kCandBuf = kMatchCap / 2;     // 16-byte candidates in a warp's match buffer

// The prefix-map slot whose lengths apply to a window whose bytes 0..7 are v
// (little-endian): exact prefix, and a length below q + 4 or the next four
// bytes in the slot's fingerprint set; -1 if none.
__device__ __forceinline__ int gram_lookup_v8(const WinCtx &C, uint64_t v) {
    const uint32_t key = C.q == 4 ? (uint32_t)v : (uint32_t)v & ((1u << (8u * C.q)) - 1u);
    const uint32_t gmask = (1u << C.gram_bits) - 1u;
    uint32_t idx = (key * kGramMult) >> (32u - C.gram_bits);
    for (;;) {
        const GramSlot g = C.s2.grams[idx];
        if (g.count == 0) return -1;
        if (g.key == key) {
            const bool ext_ok = (g.ext >> ext_bit((uint32_t)(v >> (8u * C.q)))) & 1u;
            return ext_ok || (g.count & kGramShort) ? (int)idx : -1;
        }
        idx = (idx + 1) & gmask;
    }
}

template <class Src, class Pos>
__device__ __forceinline__ int gram_lookup(const WinCtx &C, const Src &src, Pos pos,
                                           uint64_t *v8) {
    const uint64_t v = ld8(src, pos);  // window bytes 0..7, little-endian
    *v8 = v;
    return gram_lookup_v8(C, v);
}

// Probe every length of prefix-map slot gi that applies to the window at pos
// (text offset x): A2 hash, A3 probe, A4 verify, A5 emit.
template <bool DIRECT = false, class Src, class Pos>
__device__ __forceinline__ void probe_slot(const WinCtx &C, const WarpCtx &w, const Src &src,
                                           Pos pos, uint64_t x, uint32_t gi,
                                           uint32_t cls = kLenAll) {
    const GramSlot g = C.s2.grams[gi];
    const bool ext_ok = (g.ext >> ext_bit((uint32_t)(ld8(src, pos) >> (8u * C.q)))) & 1u;
    const uint32_t cnt = g.count & ~kGramShort;
    for (uint32_t j = 0; j < cnt; ++j) {
        const uint32_t L = C.s2.gram_lens[g.first + j];
        if (x + L > C.n) break;  // lengths ascend
        if (L >= C.q + 4 && !ext_ok) break;
        if (len_in_class(L, cls)) probe_length<DIRECT>(C, w, src, pos, x, L);
    }
}

// A candidate for which the list has no room is probed at once, with its
// matches appended straight to the output (the warp's buffer holds
// candidates).
__device__ __forceinline__ void cand_overflow(const WinCtx &C, const WarpCtx &w, const uint8_t *buf,
                                              uint64_t u0, uint64_t e) {
    const uint64_t x = cand_x(e);
    probe_slot<true>(C, w, buf, (uint32_t)(x + C.mis - u0), x, cand_slot(e), cand_class(e));
}

// Stage 2a for the window at pos of the tile at u0; a candidate is queued in
// the warp's buffer (w.mbuf as kCandBuf 16-byte entries), or offered to the
// list when that is full.
__device__ __forceinline__ void cand_window(const WinCtx &C, const WarpCtx &w, const CandList &cc,
                                            const uint8_t *buf, uint32_t pos, uint64_t u0) {
    const uint64_t ua = u0 + pos;
    if (ua < C.lo || ua >= C.hi) return;
    uint64_t v8;
    const int gi = gram_lookup(C, buf, pos, &v8);
    if (gi < 0) return;
    const ulonglong2 c = make_ulonglong2(cand_pack(ua - C.mis, (uint32_t)gi, kLenAll), v8);
    const uint32_t s = atomicAdd(w.mcount, 1u);
    if (s < kCandBuf) {
        reinterpret_cast<ulonglong2 *>(w.mbuf)[s] = c;
        return;
    }
    const unsigned long long g = atomicAdd(cc.count, 1ull);
    if (g < cc.cap) cc.list[g] = c;
    else cand_overflow(C, w, buf, u0, c.x);
}

// Warp-converged: move the buffered candidates to the list with one atomic;
// those beyond its capacity are probed here (the tile is still staged).
__device__ __forceinline__ void cand_flush(const WinCtx &C, const WarpCtx &w, const CandList &cc,
                                           const uint8_t *buf, uint64_t u0, uint32_t lane) {
    __syncwarp();
    const uint32_t cnt = min(*reinterpret_cast<volatile uint32_t *>(w.mcount), kCandBuf);
    if (cnt) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(cc.count, (unsigned long long)cnt);
        base = __shfl_sync(0xffffffffu, base, 0);
        const ulonglong2 *cb = reinterpret_cast<const ulonglong2 *>(w.mbuf);
        for (uint32_t i = lane; i < cnt; i += 32) {
            if (base + i < cc.cap) cc.list[base + i] = cb[i];
            else cand_overflow(C, w, buf, u0, cb[i].x);
        }
    }
    __syncwarp();
    if (lane == 0) *reinterpret_cast<volatile uint32_t *>(w.mcount) = 0;
    __syncwarp();
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

// One consumer warp's share of a staged tile: chunks warp*64 + {lane, 32 +
// lane} + k * nw * 64 (32 windows per lane per round), survivors queued per
// warp and processed one window per lane, matches flushed at the end.
//   buf: the tile's shared buffer; u0: its buffer position; nchunks: 16-byte
//   chunks holding window starts; last: highest chunk index of a full tile.
// DEFER (filtered modes): survivors only go through stage 2a, candidates to
// the list `cc` (w's buffer then holds candidates).
template <int MODE, bool Q4, bool DEFER = false>
__device__ __forceinline__ void consume_tile(const WinCtx &C, const WarpCtx &w, uint16_t *q,
                                             const uint8_t *buf, uint64_t u0, uint32_t nchunks,
                                             uint32_t last, const uint8_t *sfilt, uint32_t fmask,
                                             uint32_t lane4, uint32_t qmask, uint32_t warp,
                                             uint32_t nw, uint32_t lane,
                                             const CandList *cc = nullptr) {
    uint32_t qn = 0;  // warp-uniform queue length (< 32 between rounds)
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
                if (DEFER) {
                    cand_window(C, w, *cc, buf, q[qn + lane], u0);
                    __syncwarp();
                    if (*reinterpret_cast<volatile uint32_t *>(w.mcount) >= kCandBuf - 32)
                        cand_flush(C, w, *cc, buf, u0, lane);
                    continue;
                }
                process_window<MODE>(C, w, buf, q[qn + lane], u0);
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
                const uint32_t pos = 16u * (b < 16 ? ca : cb) + (15u - (b & 15u));
                if (DEFER) cand_window(C, w, *cc, buf, pos, u0);
                else process_window<MODE>(C, w, buf, pos, u0);
            }
            if (DEFER) cand_flush(C, w, *cc, buf, u0, lane);
            else flush(w, lane);
        }
    }
    if (DEFER) {
        if (lane < qn) cand_window(C, w, *cc, buf, q[lane], u0);
        cand_flush(C, w, *cc, buf, u0, lane);
        return;
    }
    if (lane < qn) process_window<MODE>(C, w, buf, q[lane], u0);
    flush(w, lane);
}

// ------------------------------------------------------------ sampled scan
// Stage 1 over sampled positions only (tables with sample == 4, deferred
// scans): bit i of the result is set when the word at position 4i of the
// 16-byte chunk may be the gram at offset j < 4 of some pattern.  The flat
// bit set of the grams has three bits per gram in one word (the second and
// third from the hash's bits 27..31 and 22..26): all must be set.
template <int MODE>
__device__ __forceinline__ uint32_t stage1_s4(const uint4 v, const uint8_t *sfilt, uint32_t fmask,
                                              uint32_t lane4) {
    const uint32_t wd[4] = {v.x, v.y, v.z, v.w};
    uint32_t acc = 0;
#pragma unroll
    for (int i = 3; i >= 0; --i) {
        const uint32_t hh = __umulhi(wd[i], kFilterMult);
        const uint32_t a = MODE == kFilterReplicated ? ((hh & fmask) | lane4) : ((hh >> 3) & fmask);
        const uint32_t word = *reinterpret_cast<const uint32_t *>(sfilt + a);
        uint32_t rot = __funnelshift_r(word, word, hh);  // bucket bit -> bit 31
        if (MODE == kFilterFlat)
            rot &= __funnelshift_r(word, word, hh >> 27) & __funnelshift_r(word, word, hh >> 22);
        acc = __funnelshift_l(rot, acc, 1);  // word i ends in bit i
    }
    return acc;
}

// A sampled position pos (a multiple of 4) that passed stage 1: each offset
// j of its gram in the sample map gives the window pos - j, which is offered
// to stage 2a when it belongs to this tile (windows before the tile were
// offered by the previous tile, whose last sampled position is this tile's
// first).
__device__ __forceinline__ void samp_window(const WinCtx &C, const WarpCtx &w, const CandList &cc,
                                            const uint8_t *buf, uint32_t pos, uint64_t u0,
                                            uint32_t tile) {
    const uint32_t key = *reinterpret_cast<const uint32_t *>(buf + pos);
    const uint32_t smask = (1u << C.smap_bits) - 1u;
    uint32_t idx = (key * kGramMult) >> (32u - C.smap_bits);
    uint32_t offs = 0;
    for (;;) {
        const SampSlot e = C.s2.smap[idx];
        if (e.mask == 0) return;  // a false positive of the bit set
        if (e.key == key) {
            offs = e.mask;
            break;
        }
        idx = (idx + 1) & smask;
    }
    for (uint32_t j = 0; j < 4; ++j)
        if (((offs >> j) & 1u) && pos >= j && pos - j < tile) cand_window(C, w, cc, buf, pos - j, u0);
}

// One consumer warp's share of a staged tile in a sampled, deferred scan:
// chunks warp*128 + lane + 32k (k < 4) + r * nw * 128, four sampled
// positions per chunk (16 per lane per round), the positions that pass
// queued and handled one per lane.  Chunk nchunks (the next tile's first,
// in the halo) is tested too: its words start the windows at the tile's end.
template <int MODE>
__device__ __forceinline__ void consume_tile_s4(const WinCtx &C, const WarpCtx &w, uint16_t *q,
                                                const uint8_t *buf, uint64_t u0, uint32_t nchunks,
                                                uint32_t tile, const uint8_t *sfilt,
                                                uint32_t fmask, uint32_t lane4, uint32_t warp,
                                                uint32_t nw, uint32_t lane, const CandList &cc) {
    const uint32_t nch = nchunks + 1, lastc = tile / 16u;  // chunk tile/16 lies in the halo
    uint32_t qn = 0;  // warp-uniform queue length (< 32 between rounds)
    const uint32_t step = nw * 128u;
    uint32_t c0 = warp * 128u;
    uint4 k[4];
#pragma unroll
    for (uint32_t i = 0; i < 4; ++i)
        k[i] = *reinterpret_cast<const uint4 *>(buf + 16u * min(c0 + lane + 32u * i, lastc));
    while (c0 < nch) {
        uint4 nk[4];
#pragma unroll
        for (uint32_t i = 0; i < 4; ++i)
            nk[i] = *reinterpret_cast<const uint4 *>(buf + 16u * min(c0 + step + lane + 32u * i, lastc));
        uint32_t m = 0;
#pragma unroll
        for (uint32_t i = 0; i < 4; ++i)
            if (c0 + lane + 32u * i < nch) m |= stage1_s4<MODE>(k[i], sfilt, fmask, lane4) << (4u * i);
#pragma unroll
        for (uint32_t i = 0; i < 4; ++i) k[i] = nk[i];
        const uint32_t cbase = c0 + lane;
        c0 += step;
        if (__ballot_sync(0xffffffffu, m != 0) == 0) continue;
        // bit b of m: word b & 3 of chunk cbase + 32 * (b >> 2)
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
                q[at++] = (uint16_t)(16u * (cbase + 32u * (b >> 2)) + 4u * (b & 3u));
            }
            qn += total;
            __syncwarp();
            while (qn >= 32) {  // full rounds: one queued position per lane
                qn -= 32;
                samp_window(C, w, cc, buf, q[qn + lane], u0, tile);
                __syncwarp();
                if (*reinterpret_cast<volatile uint32_t *>(w.mcount) >= kCandBuf - 32)
                    cand_flush(C, w, cc, buf, u0, lane);
            }
        } else {
            while (m) {  // more than the queue holds: each lane works through its own
                const uint32_t b = 31u - __clz(m);
                m &= ~(1u << b);
                samp_window(C, w, cc, buf, 16u * (cbase + 32u * (b >> 2)) + 4u * (b & 3u), u0,
                            tile);
            }
            cand_flush(C, w, cc, buf, u0, lane);
        }
    }
    if (lane < qn) samp_window(C, w, cc, buf, q[lane], u0, tile);
    cand_flush(C, w, cc, buf, u0, lane);
}

// ------------------------------------------------------------ role filter
// Stage 1 with a role filter (DevTable::rf_step): only every STEP-th
// position p is looked up, with its gram G(p) (4 bytes, little-endian).

// G's word of the bit set, rotated so that G's roles S, L, B sit at bits
// 31, 30, 29.
__device__ __forceinline__ uint32_t rf_probe(uint32_t g, const uint8_t *rfilt, uint32_t rshift) {
    const uint32_t lo = g * kRoleMult;
    const uint32_t word = *reinterpret_cast<const uint32_t *>(rfilt + ((lo >> rshift) & ~3u));
    return __funnelshift_r(word, word, lo);
}

// G's word of a side set (replicated into the 32 banks: the lane reads its
// own bank's copy), chosen by G's low three bytes, rotated by G's top byte so
// that the bit pair a gram with that top byte sets sits at bits 31 and 28.
__device__ __forceinline__ uint32_t rf_side_probe(uint32_t g, const uint8_t *side,
                                                  uint32_t lane4) {
    const uint32_t lo = (g & 0x00FFFFFFu) * kRoleMult;
    const uint32_t word =
        *reinterpret_cast<const uint32_t *>(side + (((lo >> 16) & 0xFF80u) | lane4));
    return __funnelshift_r(word, word, g >> 24);
}

// Kinds of role filter: 2 and 4, the sampling step; 6, step 4 with a side
// set tested at the positions 2 mod 4.  Kinds 2 and 6 sample every even
// position of a chunk and share its layout (rf_step_of).
__host__ __device__ constexpr int rf_step_of(int kind) { return kind == 4 ? 4 : 2; }

// Roles of the sampled positions of one 16-byte chunk (words v; v4: the next
// chunk's first word), one nibble per position i (bit 3 S, bit 2 L, bit 1 B,
// bit 0 S's second bit):
//   kinds 2, 6: positions 2i, i < 8, in nibble 7 - i of the 32-bit result
//     (kind 6: even i from the main set, odd i from the side set);
//   kind 4: positions 4i, i < 4, in nibble 3 - i of the low 16 bits.
template <int KIND>
__device__ __forceinline__ uint32_t rf_chunk(const uint4 v, uint32_t v4, const uint8_t *rfilt,
                                             uint32_t rshift, const uint8_t *side,
                                             uint32_t lane4) {
    const uint32_t wd[5] = {v.x, v.y, v.z, v.w, v4};
    uint32_t a = 0, b = 0;  // two independent accumulators
    if constexpr (rf_step_of(KIND) == 2) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const uint32_t g =
                (i & 1) ? __funnelshift_r(wd[i >> 1], wd[(i >> 1) + 1], 16) : wd[i >> 1];
            const uint32_t r = (KIND == 6 && (i & 1)) ? rf_side_probe(g, side, lane4)
                                                      : rf_probe(g, rfilt, rshift);
            if (i < 4) a = __funnelshift_l(r, a, 4);  // a = a << 4 | r >> 28
            else b = __funnelshift_l(r, b, 4);
        }
        const uint32_t acc = __byte_perm(b, a, 0x5410);  // a << 16 | b
        // a side nibble keeps only S's bits: its other bits carry no role
        return KIND == 6 ? acc & 0xF9F9F9F9u : acc;
    } else {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const uint32_t r = rf_probe(wd[i], rfilt, rshift);
            if (i < 2) a = __funnelshift_l(r, a, 4);
            else b = __funnelshift_l(r, b, 4);
        }
        return (a << 8) | b;
    }
}

// Candidate positions of a chunk from its role nibbles and the next chunk's
// (whose first positions hold the second grams of the last ones): bit 0 of
// nibble 7 - i is set when sampled position i of the chunk makes its windows
// candidates: both S bits, or L with B at the position 4 bytes on.
template <int STEP>
__device__ __forceinline__ uint32_t rf_cands(uint32_t acc, uint32_t accn) {
    uint32_t x, comb, keep;
    if constexpr (STEP == 2) {
        x = acc;
        comb = __funnelshift_l(accn, acc, 9);  // B of position i + 2 under L of i
        keep = 0x11111111u;
    } else {
        x = __byte_perm(accn, acc, 0x5410);    // acc << 16 | accn
        comb = x << 5;                         // B of position i + 1 under L of i
        keep = 0x11110000u;
    }
    return ((x & (x >> 3)) | ((x & comb) >> 2)) & keep;
}

// A lane's candidates of one round in one word: the mask of its chunk k
// (bits 4n) shifted left by k, so bit b belongs to chunk b mod 4, position
// 7 - b / 4 of it.  Buffer position of the sampled position named by bit b,
// for the lane's first chunk cbase (its chunk k is cbase + 32k).
template <int STEP>
__device__ __forceinline__ uint32_t rf_pos(uint32_t cbase, uint32_t b) {
    return 16u * (cbase + 32u * (b & 3u)) + (uint32_t)STEP * (7u - (b >> 2));
}

// A window (buffer position ua, bytes 0..7 in v8) of a role-filter
// survivor: stage 2a (DEFER: the candidate to the warp's buffer, or to the
// list when that is full, or probed at once when the list is full too) or
// stage 2 (the rest of a longer window read from the text in global memory).
template <bool DEFER>
__device__ __forceinline__ void rf_window_g(const WinCtx &C, const WarpCtx &w, const CandList *cc,
                                            const GText &g, uint64_t ua, uint64_t v8,
                                            uint32_t cls) {
    if (ua < C.lo || ua >= C.hi) return;
    const int gi = gram_lookup_v8(C, v8);
    if (gi < 0) return;
    const uint64_t x = ua - C.mis;
    const WText win{g, ua, v8};
    if (!DEFER) {
        probe_slot(C, w, win, ua, x, (uint32_t)gi, cls);
        return;
    }
    const ulonglong2 c = make_ulonglong2(cand_pack(x, (uint32_t)gi, cls), v8);
    const uint32_t s = atomicAdd(w.mcount, 1u);
    if (s < kCandBuf) {
        reinterpret_cast<ulonglong2 *>(w.mbuf)[s] = c;
        return;
    }
    const unsigned long long k = atomicAdd(cc->count, 1ull);
    if (k < cc->cap) cc->list[k] = c;
    else probe_slot<true>(C, w, win, ua, x, (uint32_t)gi, cls);
}

// Warp-converged: the warp's buffered candidates to the list with one
// atomic; those beyond its capacity are probed here from global memory.
__device__ __forceinline__ void rf_cand_flush(const WinCtx &C, const WarpCtx &w,
                                              const CandList &cc, const GText &g, uint32_t lane) {
    __syncwarp();
    const uint32_t cnt = min(*reinterpret_cast<volatile uint32_t *>(w.mcount), kCandBuf);
    if (cnt) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(cc.count, (unsigned long long)cnt);
        base = __shfl_sync(0xffffffffu, base, 0);
        const ulonglong2 *cb = reinterpret_cast<const ulonglong2 *>(w.mbuf);
        for (uint32_t i = lane; i < cnt; i += 32) {
            const ulonglong2 c = cb[i];
            if (base + i < cc.cap) {
                cc.list[base + i] = c;
            } else {
                const uint64_t x = cand_x(c.x);
                probe_slot<true>(C, w, g, x + C.mis, x, cand_slot(c.x), cand_class(c.x));
            }
        }
    }
    __syncwarp();
    if (lane == 0) *reinterpret_cast<volatile uint32_t *>(w.mcount) = 0;
    __syncwarp();
}

}  // namespace rk
