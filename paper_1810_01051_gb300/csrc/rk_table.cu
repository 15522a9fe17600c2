// Pattern-table builder (host side of rk_build) and table bookkeeping.
//
// Section 3.1 computes the pattern hash once on the host and passes it to the
// kernel.  For a pattern set the host builds, in one device allocation:
//   - stage-1 bit set over the q-byte prefixes of all patterns (q = min(4,
//     shortest length)), keyed by the prefix read as a little-endian word;
//   - prefix map: exact q-byte prefix -> distinct lengths of the patterns
//     that start with it, plus a 32-bit fingerprint set of their next four
//     bytes;
//   - one open-addressing table per pattern length L, keyed by the Rabin
//     hash h_B(P) = sum_i P[i] * B^(L-1-i) mod (2^61 - 1), B = 2^base_log2,
//     each slot naming the ids of the patterns of that length and hash;
//   - the pattern bytes, each pattern 8-byte aligned and zero padded.
#include <algorithm>
#include <cstring>
#include <new>
#include <unordered_map>
#include <utility>

#include "rk_internal.cuh"
#include "rk_layout.cuh"

namespace rk {
namespace {

uint64_t host_rotl61(uint64_t x, uint32_t s) { return ((x << s) | (x >> (61 - s))) & kP61; }

// Rabin hash mod 2^61-1 with B = 2^k: Horner's rule, multiplication by B
// being a 61-bit rotation by k.
uint64_t host_rabin(const uint8_t *s, uint32_t L, uint32_t k) {
    uint64_t h = 0;
    for (uint32_t i = 0; i < L; ++i) {
        h = host_rotl61(h, k) + s[i];
        if (h >= kP61) h -= kP61;
    }
    return h;
}

uint32_t ceil_log2(uint64_t x) {
    uint32_t b = 0;
    while ((1ull << b) < x) ++b;
    return b;
}

// The first q bytes as a little-endian integer.
uint32_t prefix_key(const uint8_t *s, uint32_t q) {
    uint32_t v = 0;
    for (uint32_t i = 0; i < q; ++i) v |= (uint32_t)s[i] << (8 * i);
    return v;
}

struct Blob {  // host staging of the device allocation
    std::vector<uint8_t> bytes;
    size_t add(size_t n, size_t align = 256) {
        size_t off = (bytes.size() + align - 1) / align * align;
        bytes.resize(off + n);
        return off;
    }
};

}  // namespace

int check_device(const rk_table *t) {
    int d = -1;
    if (cudaGetDevice(&d) != cudaSuccess) return RK_ECUDA;
    return d == t->device ? RK_OK : RK_EINVAL;
}

}  // namespace rk

using namespace rk;

extern "C" const char *rk_strerror(int status) {
    switch (status) {
        case RK_OK: return "ok";
        case RK_EINVAL: return "invalid argument";
        case RK_ENOMEM: return "out of memory";
        case RK_ECAPACITY: return "output capacity too small";
        case RK_ECUDA: return "CUDA error";
        case RK_ETIMEOUT: return "device wait timed out";
        default: return "unknown status";
    }
}

namespace rk {

namespace {

// Stage-1 bit set of `keys` (4-byte little-endian values or q-byte prefixes):
// the layout (replicated into 32 banks or flat), its size and the device
// image.  Returns false for an invalid forced size.
// three_bits (flat layout): each key also sets two more bits of the same
// word, at the hash's bits 27..31 and 22..26, and a key passes only when all
// three are set.
bool make_filter(const std::vector<uint32_t> &keys, uint32_t filter_opt, uint32_t bits_opt,
                 bool three_bits, uint32_t *mode, uint32_t *fbits, std::vector<uint32_t> *img,
                 uint32_t *fmask) {
    const uint64_t D = keys.size();
    *fbits = bits_opt;
    if (filter_opt == RK_FILTER_NONE) {
        *mode = kFilterNone;
    } else if (filter_opt == RK_FILTER_REPLICATED ||
               (filter_opt == RK_FILTER_AUTO && D <= 256 && !bits_opt)) {
        *mode = kFilterReplicated;
        if (!*fbits) *fbits = 14;
        if (*fbits < 10 || *fbits > 15) return false;
    } else {
        *mode = kFilterFlat;
        // about 1 in 32 bits set (three bits per key: at most 2^19 bits,
        // 64 KiB, so that two 48 KiB tiles still fit beside it)
        if (!*fbits)
            *fbits = std::min<uint32_t>(three_bits ? 19 : 20,
                                        std::max<uint32_t>(15, ceil_log2(32ull * D)));
        if (*fbits < 10 || *fbits > 20) return false;
    }
    img->clear();
    *fmask = 0;
    if (*mode == kFilterNone) return true;
    const uint32_t W = 1u << (*fbits - 5);
    std::vector<uint32_t> bm(W, 0);
    for (uint32_t key : keys) {
        const uint32_t hi = (uint32_t)(((uint64_t)key * kFilterMult) >> 32);
        const uint32_t word = (*mode == kFilterReplicated ? (hi >> 7) : (hi >> 5)) & (W - 1);
        const uint32_t r = hi & 31;
        // stored one place below r: a right rotation by r moves it to bit 31
        bm[word] |= 1u << ((r + 31) & 31);
        if (three_bits && *mode == kFilterFlat)
            bm[word] |= (1u << (((hi >> 27) + 31) & 31)) | (1u << (((hi >> 22) + 31) & 31));
    }
    if (*mode == kFilterReplicated) {
        img->resize((size_t)W * 32);
        for (uint32_t w = 0; w < W; ++w)
            for (uint32_t l = 0; l < 32; ++l) (*img)[(size_t)w * 32 + l] = bm[w];
        *fmask = (W - 1) << 7;
    } else {
        *img = bm;
        *fmask = (W - 1) << 2;
    }
    return true;
}

// Role filter of the patterns for sampling step `step` (see DevTable): the
// grams at offsets j < step of every pattern with their roles, in a flat bit
// set of 2^bits bits.  Role S sets two bits of the gram's word (at lo + 31
// and lo + 28, the slot of a fourth role), and the scan asks for both, so a
// text gram that is no key passes as S about as often as two set bits line
// up, like L with B.  Step 2 needs every pattern to have at least 5 bytes,
// or 4: a 4-byte pattern P has no gram at offset 1, so for an occurrence at
// an odd x the gram at p = x + 1 holds P[1..4) and one text byte; every such
// gram (256 of them) gets role S.  Step 4 needs at least 7 bytes, or a side
// table: the patterns shorter than kRfSplit (7) go into the main set only
// at offsets 0 and 1 (their windows at positions 0 and 3 mod 4), and into a
// small set tested at the positions 2 mod 4 (*side), where the same offsets
// find their windows at positions 2 and 1 mod 4; the scan then looks at
// windows 2 and 3 bytes before a main position only for longer patterns.
// The side set (2^14 bits, replicated) picks a word by a gram's low three
// bytes and the bit pair by its top byte (side_word).
// Returns false when the patterns do not allow the step or a set would be
// too dense (more than one key per 16 bits at the largest size).
constexpr uint32_t kRoleMaxLog2Bits = 19;   // 64 KiB of shared memory
constexpr uint32_t kRoleMaxWild = 64;       // 4-byte patterns a filter takes
constexpr uint32_t kRoleBitsPerKey = 16;    // least bits per key
constexpr uint32_t kRfSurvivorWarps = 6;    // survivor warps of the role-filter scan kernel
constexpr uint32_t kRfSplitLen = 7;         // shorter patterns use the side table (step 4)
constexpr uint32_t kSideWords = 512;        // side table: 2^14 bits, replicated into 32 banks
constexpr uint32_t kSideMaxKeys = 1024;

// The grams of pattern p (length L) at offsets 0 and 1 (or its wildcard
// grams), role S, appended to keys.
void short_keys(const uint8_t *p, uint32_t L,
                std::vector<std::pair<uint32_t, uint32_t>> *keys) {
    keys->emplace_back(prefix_key(p, 4), 0u);
    if (L >= 5) {
        keys->emplace_back(prefix_key(p + 1, 4), 0u);
    } else {
        const uint32_t g3 = prefix_key(p + 1, 3);
        for (uint32_t c = 0; c < 256; ++c) keys->emplace_back(g3 | (c << 24), 0u);
    }
}

// The side set's word for a gram: chosen by its low three bytes (so that the
// wildcard grams of a 4-byte pattern, P[1..4) and any fourth byte, share one
// word), the bit pair by its top byte.
uint32_t side_word(uint32_t g) { return ((g & 0x00FFFFFFu) * kRoleMult) >> 23; }

bool make_role_filter(const uint8_t *patterns, const std::vector<uint64_t> &src_off,
                      const std::vector<uint32_t> &plen, uint32_t step,
                      std::vector<uint32_t> *img, uint32_t *log2_bits,
                      std::vector<uint32_t> *side) {
    const uint32_t k = (uint32_t)plen.size();
    uint32_t lmin = UINT32_MAX, n4 = 0;
    for (uint32_t L : plen) {
        lmin = std::min(lmin, L);
        n4 += L == 4;
    }
    side->clear();
    if (lmin < 4 || n4 > kRoleMaxWild) return false;
    const bool with_side = step == 4 && lmin < kRfSplitLen;
    std::vector<std::pair<uint32_t, uint32_t>> keys;  // (gram, role 0 S / 1 L / 2 B)
    std::vector<std::pair<uint32_t, bool>> skeys;      // side set: (gram, any top byte)
    keys.reserve((size_t)k * step * 2 + (size_t)n4 * 256);
    for (uint32_t i = 0; i < k; ++i) {
        const uint8_t *p = patterns + src_off[i];
        const uint32_t L = plen[i];
        if (with_side && L < kRfSplitLen) {
            short_keys(p, L, &keys);
            skeys.emplace_back(prefix_key(p, 4), false);
            if (L >= 5) skeys.emplace_back(prefix_key(p + 1, 4), false);
            else skeys.emplace_back(prefix_key(p + 1, 3), true);
            continue;
        }
        for (uint32_t j = 0; j < step; ++j) {
            if (j + 4 <= L) {
                const bool longer = L >= j + 8;  // a second gram follows
                keys.emplace_back(prefix_key(p + j, 4), longer ? 1u : 0u);
                if (longer) keys.emplace_back(prefix_key(p + j + 4, 4), 2u);
            } else {  // step 2, L = 4, j = 1: P[1..4) and any byte
                const uint32_t g3 = prefix_key(p + 1, 3);
                for (uint32_t c = 0; c < 256; ++c) keys.emplace_back(g3 | (c << 24), 0u);
            }
        }
    }
    if (skeys.size() > kSideMaxKeys) return false;
    const uint64_t nk = keys.size();
    const uint32_t bits =
        std::min<uint32_t>(kRoleMaxLog2Bits, std::max<uint32_t>(15, ceil_log2(nk * 512)));
    if (nk * kRoleBitsPerKey > (1ull << bits)) return false;
    const uint32_t wbits = bits - 5;
    img->assign(1u << wbits, 0u);
    for (const auto &kr : keys) {
        const uint32_t lo = kr.first * kRoleMult;
        uint32_t &word = (*img)[lo >> (32 - wbits)];
        word |= 1u << ((lo + 31u - kr.second) & 31u);
        if (kr.second == 0) word |= 1u << ((lo + 28u) & 31u);  // S's second bit
    }
    if (with_side) {
        // word w of the side set at byte (w << 7) | (bank << 2), every bank a
        // copy; a gram's bits at its top byte + 31 and + 28 (mod 32), a
        // wildcard gram's every bit
        std::vector<uint32_t> bm(kSideWords, 0u);
        for (const auto &kw : skeys) {
            const uint32_t t = kw.first >> 24;
            bm[side_word(kw.first)] |=
                kw.second ? 0xFFFFFFFFu : (1u << ((t + 31u) & 31u)) | (1u << ((t + 28u) & 31u));
        }
        side->resize((size_t)kSideWords * 32);
        for (uint32_t w = 0; w < kSideWords; ++w)
            for (uint32_t b = 0; b < 32; ++b) (*side)[(size_t)w * 32 + b] = bm[w];
    }
    *log2_bits = bits;
    return true;
}

}  // namespace

// Serialise the pattern table of one pattern set into a host image; every
// part is 256-byte aligned and the image ends on a 256-byte boundary.
int build_blob(const uint8_t *patterns, const uint32_t *lens, uint32_t k, uint32_t base_log2,
               uint32_t filter_opt, uint32_t filter_bits_opt, uint32_t sample_opt,
               uint32_t role_opt, TableBlob *out) {
    // ---- patterns ---------------------------------------------------------
    std::vector<uint64_t> src_off(k), poff(k);
    std::vector<uint32_t> plen(k);
    uint64_t acc = 0, packed = 0;
    uint32_t lmin = UINT32_MAX, lmax = 0;
    for (uint32_t i = 0; i < k; ++i) {
        uint32_t L = lens[i];
        if (L < 1 || L > RK_MAX_PATTERN_LEN) return RK_EINVAL;
        src_off[i] = acc;
        acc += L;
        plen[i] = L;
        poff[i] = packed;
        packed += (L + 7) / 8 * 8;
        lmin = std::min(lmin, L);
        lmax = std::max(lmax, L);
    }
    if (k == 0) { lmin = 1; lmax = 1; }
    uint32_t q = std::min<uint32_t>(4, lmin);

    std::vector<uint32_t> lengths(plen);
    std::sort(lengths.begin(), lengths.end());
    lengths.erase(std::unique(lengths.begin(), lengths.end()), lengths.end());

    // ---- prefix map: q-byte prefix -> distinct lengths ----------------------
    std::unordered_map<uint32_t, std::vector<uint32_t>> gram_to_lens;
    std::unordered_map<uint32_t, uint32_t> gram_ext;
    gram_to_lens.reserve(k * 2 + 1);
    for (uint32_t i = 0; i < k; ++i) {
        const uint8_t *p = patterns + src_off[i];
        uint32_t key = prefix_key(p, q);
        gram_to_lens[key].push_back(plen[i]);
        uint32_t &ext = gram_ext[key];
        if (plen[i] >= q + 4) ext |= 1u << ext_bit(prefix_key(p + q, 4));
    }
    std::vector<uint32_t> gram_keys;
    gram_keys.reserve(gram_to_lens.size());
    for (auto &kv : gram_to_lens) {
        auto &v = kv.second;
        std::sort(v.begin(), v.end());
        v.erase(std::unique(v.begin(), v.end()), v.end());
        gram_keys.push_back(kv.first);
    }
    std::sort(gram_keys.begin(), gram_keys.end());  // deterministic layout
    uint32_t D = (uint32_t)gram_keys.size();
    uint32_t gram_bits = std::max<uint32_t>(4, ceil_log2(2ull * D));
    std::vector<GramSlot> grams(1ull << gram_bits, GramSlot{0, 0, 0, 0});
    std::vector<uint32_t> gram_lens;
    for (uint32_t key : gram_keys) {
        const auto &v = gram_to_lens[key];
        uint32_t idx = (key * kGramMult) >> (32 - gram_bits);
        uint32_t mask = (1u << gram_bits) - 1;
        while (grams[idx].count) idx = (idx + 1) & mask;
        const uint32_t shorts = v.front() < q + 4 ? kGramShort : 0u;  // v ascends
        grams[idx] = GramSlot{key, (uint32_t)gram_lens.size(), (uint32_t)v.size() | shorts,
                              gram_ext[key]};
        gram_lens.insert(gram_lens.end(), v.begin(), v.end());
    }

    // ---- stage-1 bit set ---------------------------------------------------
    uint32_t mode, fbits, fmask;
    std::vector<uint32_t> fimg;
    if (!make_filter(gram_keys, filter_opt, filter_bits_opt, false, &mode, &fbits, &fimg, &fmask))
        return RK_EINVAL;

    // ---- role filter: sampled grams with their roles ------------------------
    std::vector<uint32_t> rimg, rside;
    uint32_t rstep = 0, rbits = 0;
    // chosen by the builder only when the prefilter is too (RK_FILTER_AUTO)
    const bool role_ok = role_opt > 1 || (role_opt == 0 && filter_opt == RK_FILTER_AUTO);
    if (role_ok && mode != kFilterNone && q == 4 && k > 0) {
        for (uint32_t step : {4u, 2u}) {
            if (role_opt > 1 && role_opt != step) continue;
            // the builder's own choice takes step 4 only without a side set:
            // with one, every main-position survivor stands for four windows
            // of survivor-warp work, and step 2 measured faster
            if (role_opt == 0 && step == 4 && lmin < kRfSplitLen) continue;
            if (make_role_filter(patterns, src_off, plen, step, &rimg, &rbits, &rside)) {
                rstep = step;
                break;
            }
        }
    }

    // ---- sampled stage 1: 4-byte grams at offsets 0..3, their offset sets --
    const bool sampled = !rstep && sample_opt != 1 && mode != kFilterNone && q == 4 && lmin >= 7;
    std::vector<SampSlot> smap;
    std::vector<uint32_t> simg;
    uint32_t smap_bits = 0, smode = 0, sbits = 0, smask_addr = 0;
    if (sampled) {
        std::unordered_map<uint32_t, uint32_t> offs;
        offs.reserve(k * 8 + 1);
        for (uint32_t i = 0; i < k; ++i)
            for (uint32_t j = 0; j < 4; ++j)
                offs[prefix_key(patterns + src_off[i] + j, 4)] |= 1u << j;
        std::vector<uint32_t> skeys;
        skeys.reserve(offs.size());
        for (auto &kv : offs) skeys.push_back(kv.first);
        std::sort(skeys.begin(), skeys.end());
        smap_bits = std::max<uint32_t>(4, ceil_log2(2ull * skeys.size()));
        smap.assign(1ull << smap_bits, SampSlot{0, 0});
        const uint32_t smask = (1u << smap_bits) - 1;
        for (uint32_t key : skeys) {
            uint32_t idx = (key * kGramMult) >> (32 - smap_bits);
            while (smap[idx].mask) idx = (idx + 1) & smask;
            smap[idx] = SampSlot{key, offs[key]};
        }
        // the same layout choice as the prefix bit set, for this key set; a
        // flat one tests three bits per gram (stage 1 tests 4x fewer positions)
        if (!make_filter(skeys, filter_opt, filter_bits_opt, true, &smode, &sbits, &simg,
                         &smask_addr))
            return RK_EINVAL;
    }

    // ---- per-length hash tables -------------------------------------------
    std::vector<uint2> group_hdr(lmax + 1, make_uint2(0, 0));
    std::vector<GroupSlot> slots;
    std::vector<uint32_t> group_pids;
    group_pids.reserve(k);
    {
        std::vector<std::vector<uint32_t>> by_len(lmax + 1);
        for (uint32_t i = 0; i < k; ++i) by_len[plen[i]].push_back(i);
        for (uint32_t L : lengths) {
            auto &ids = by_len[L];
            std::vector<std::pair<uint64_t, uint32_t>> hp;
            hp.reserve(ids.size());
            for (uint32_t id : ids) hp.emplace_back(host_rabin(patterns + src_off[id], L, base_log2), id);
            std::sort(hp.begin(), hp.end());
            uint32_t uniq = 0;
            for (size_t i = 0; i < hp.size(); ++i)
                if (i == 0 || hp[i].first != hp[i - 1].first) ++uniq;
            uint32_t bits = std::max<uint32_t>(1, ceil_log2(2ull * uniq));
            uint32_t first_slot = (uint32_t)slots.size();
            slots.resize(slots.size() + (1ull << bits), GroupSlot{0, 0, 0});
            group_hdr[L] = make_uint2(first_slot, bits);
            uint64_t mask = (1ull << bits) - 1;
            for (size_t i = 0; i < hp.size();) {
                size_t j = i;
                while (j < hp.size() && hp[j].first == hp[i].first) ++j;
                uint64_t h = hp[i].first;
                uint64_t idx = (h * kGroupMult) >> (64 - bits);
                while (slots[first_slot + idx].count) idx = (idx + 1) & mask;
                slots[first_slot + idx] = GroupSlot{h, (uint32_t)group_pids.size(), (uint32_t)(j - i)};
                for (size_t m = i; m < j; ++m) group_pids.push_back(hp[m].second);
                i = j;
            }
        }
    }

    // ---- one device allocation --------------------------------------------
    Blob b;
    size_t o_filter = b.add(fimg.size() * 4 + 16);
    size_t o_grams = b.add(grams.size() * sizeof(GramSlot));
    size_t o_glens = b.add(gram_lens.size() * 4 + 4);
    size_t o_ghdr = b.add(group_hdr.size() * sizeof(uint2));
    size_t o_slots = b.add(slots.size() * sizeof(GroupSlot) + sizeof(GroupSlot));
    size_t o_gpids = b.add(group_pids.size() * 4 + 4);
    size_t o_pbytes = b.add(packed + 16);
    size_t o_poff = b.add(k * 8 + 8);
    size_t o_plen = b.add(k * 4 + 4);
    size_t o_lens = b.add(lengths.size() * 4 + 4);
    size_t o_smap = b.add(smap.size() * sizeof(SampSlot) + 8);
    size_t o_sfilter = b.add(simg.size() * 4 + 16);  // after the survivor tables: not staged with them
    // the side set right after the main one: the scan stages both with one copy
    size_t o_rfilter = b.add((rimg.size() + rside.size()) * 4 + 16);
    b.add(0);  // the blob ends on a 256-byte boundary: whole 16-byte copies stay inside
    uint8_t *hb = b.bytes.data();
    if (!fimg.empty()) memcpy(hb + o_filter, fimg.data(), fimg.size() * 4);
    memcpy(hb + o_grams, grams.data(), grams.size() * sizeof(GramSlot));
    if (!gram_lens.empty()) memcpy(hb + o_glens, gram_lens.data(), gram_lens.size() * 4);
    memcpy(hb + o_ghdr, group_hdr.data(), group_hdr.size() * sizeof(uint2));
    if (!slots.empty()) memcpy(hb + o_slots, slots.data(), slots.size() * sizeof(GroupSlot));
    if (!group_pids.empty()) memcpy(hb + o_gpids, group_pids.data(), group_pids.size() * 4);
    for (uint32_t i = 0; i < k; ++i) memcpy(hb + o_pbytes + poff[i], patterns + src_off[i], plen[i]);
    if (k) memcpy(hb + o_poff, poff.data(), k * 8);
    if (k) memcpy(hb + o_plen, plen.data(), k * 4);
    if (!lengths.empty()) memcpy(hb + o_lens, lengths.data(), lengths.size() * 4);
    if (!smap.empty()) memcpy(hb + o_smap, smap.data(), smap.size() * sizeof(SampSlot));
    if (!simg.empty()) memcpy(hb + o_sfilter, simg.data(), simg.size() * 4);
    if (!rimg.empty()) memcpy(hb + o_rfilter, rimg.data(), rimg.size() * 4);
    if (!rside.empty()) memcpy(hb + o_rfilter + rimg.size() * 4, rside.data(), rside.size() * 4);

    if (b.bytes.size() - o_grams > 0xFFFFFFFFull) return RK_EINVAL;  // tables above 4 GiB
    TableBlob &tb = *out;
    tb.o_filter = o_filter;
    tb.o_grams = o_grams;
    tb.o_glens = o_glens;
    tb.o_ghdr = o_ghdr;
    tb.o_slots = o_slots;
    tb.o_gpids = o_gpids;
    tb.o_pbytes = o_pbytes;
    tb.o_poff = o_poff;
    tb.o_plen = o_plen;
    tb.o_lens = o_lens;
    tb.o_smap = o_smap;
    tb.o_sfilter = o_sfilter;
    tb.o_rfilter = o_rfilter;
    DevTable &d = tb.meta;
    d = DevTable{};
    d.filter_bytes = (uint32_t)(fimg.size() * 4);
    d.filter_mode = mode;
    d.filter_mask = fmask;
    d.q = q;
    d.gram_bits = gram_bits;
    d.n_lengths = (uint32_t)lengths.size();
    d.n_patterns = k;
    d.lmin = lmin;
    d.lmax = lmax;
    d.base_log2 = base_log2;
    d.sample = sampled ? 4u : 1u;
    d.sfilter_bytes = (uint32_t)(simg.size() * 4);
    d.sfilter_mode = smode;
    d.sfilter_mask = smask_addr;
    d.smap_bits = smap_bits;
    d.rf_step = rstep;
    d.rfilter_bytes = (uint32_t)((rimg.size() + rside.size()) * 4);
    d.rf_side_off = rside.empty() ? 0u : (uint32_t)(rimg.size() * 4);
    d.rf_shift = rstep ? 30 - (rbits - 5) : 0;
    d.s2_bytes = (uint32_t)(o_sfilter - o_grams);
    tb.n_grams = D;
    tb.filter_log2_bits = mode == kFilterNone ? 0 : fbits;
    tb.sfilter_log2_bits = sampled ? sbits : 0;
    tb.rfilter_log2_bits = rstep ? rbits : 0;
    tb.bytes = std::move(b.bytes);
    return RK_OK;
}

// Point the device view of a table at its image placed at device address dm.
void bind_blob(DevTable *d, const TableBlob &b, const uint8_t *dm) {
    *d = b.meta;
    d->filter = (const uint32_t *)(dm + b.o_filter);
    d->grams = (const GramSlot *)(dm + b.o_grams);
    d->gram_lens = (const uint32_t *)(dm + b.o_glens);
    d->group_hdr = (const uint2 *)(dm + b.o_ghdr);
    d->slots = (const GroupSlot *)(dm + b.o_slots);
    d->group_pids = (const uint32_t *)(dm + b.o_gpids);
    d->pbytes = dm + b.o_pbytes;
    d->poff = (const uint64_t *)(dm + b.o_poff);
    d->plen = (const uint32_t *)(dm + b.o_plen);
    d->lengths = (const uint32_t *)(dm + b.o_lens);
    d->smap = (const SampSlot *)(dm + b.o_smap);
    d->sfilter = (const uint32_t *)(dm + b.o_sfilter);
    d->rfilter = (const uint32_t *)(dm + b.o_rfilter);
    d->s2_base = dm + b.o_grams;
}

}  // namespace rk

namespace rk {
namespace {

// rk_build_opts with the defaults filled in.
struct Opts {
    uint32_t base_log2, filter, filter_log2_bits, warps, tile, stages, cps, sample, role;
};

// Check the patterns' count and lengths and the options (no CUDA call).
int read_opts(const uint8_t *patterns, const uint32_t *lens, uint32_t k,
              const rk_build_opts *opts, Opts *out) {
    if (k > RK_MAX_PATTERNS) return RK_EINVAL;
    if (k > 0 && (!patterns || !lens)) return RK_EINVAL;
    for (uint32_t i = 0; i < k; ++i)
        if (lens[i] < 1 || lens[i] > RK_MAX_PATTERN_LEN) return RK_EINVAL;
    rk_build_opts o{};
    if (opts) o = *opts;
    Opts r{};
    r.base_log2 = o.base_log2 ? o.base_log2 : 8;
    r.filter = o.filter;
    r.filter_log2_bits = o.filter_log2_bits;
    // warps, tile and stages stay 0 (default) here: plan_table picks them
    // by the kind of stage-1 filter the table gets
    r.warps = o.warps;
    r.tile = o.tile_bytes;
    r.stages = o.stages;
    r.cps = o.ctas_per_sm ? o.ctas_per_sm : 1;
    r.sample = o.sample;
    r.role = o.role_step;
    if (r.base_log2 < 1 || r.base_log2 > 60) return RK_EINVAL;
    if (r.filter > RK_FILTER_NONE) return RK_EINVAL;
    // survivor positions within a tile are 16-bit
    if (r.warps > 31 || (r.tile && (r.tile < 1024 || r.tile % 16 || r.tile > kMaxTileBytes)) ||
        (r.stages && (r.stages < 2 || r.stages > 8)) || r.cps < 1 || r.cps > 8)
        return RK_EINVAL;
    if (r.sample > 1) return RK_EINVAL;
    if (r.role != 0 && r.role != 1 && r.role != 2 && r.role != 4) return RK_EINVAL;
    *out = r;
    return RK_OK;
}

constexpr int kNoRoom = -1;  // plan_with: the shared memory cannot hold the pipeline

// plan_table with one role-filter option.
int plan_with(const uint8_t *patterns, const uint32_t *lens, uint32_t k, const Opts &o,
              uint32_t role_opt, uint32_t smem_optin, TableBlob *tb, Tuning *tune) {
    const uint32_t cps = o.cps;
    int rc = build_blob(patterns, lens, k, o.base_log2, o.filter, o.filter_log2_bits, o.sample,
                        role_opt, tb);
    if (rc) return rc;
    const bool role = tb->meta.rf_step != 0;
    // Defaults: 48 KiB tiles, two in flight; 24 warps with the prefix filter
    // (two 24 KiB rounds each), with a role filter 16 stage-1 warps (three
    // 16 KiB rounds) and kRfSurvivorWarps survivor warps (fewer when the
    // stage-1 warps leave less room under 31).
    uint32_t warps = o.warps ? o.warps : (role ? 16u : 24u);
    uint32_t tile = o.tile ? o.tile : 49152u;
    uint32_t stages = o.stages ? o.stages : 2u;
    uint32_t sv = 0;
    if (role) {
        sv = std::min<uint32_t>(kRfSurvivorWarps, std::max<uint32_t>(1, 31 - warps));
        warps = std::min<uint32_t>(warps, 31 - sv);
    }
    const uint32_t lmax = tb->meta.lmax;
    // the bit set a scan stages at offset 0: the role filter when there is
    // one, else the prefixes' or (deferred scans) the sampled grams'
    const uint32_t fbytes = tb->meta.rf_step
                                ? tb->meta.rfilter_bytes
                                : std::max(tb->meta.filter_bytes, tb->meta.sfilter_bytes);
    const uint64_t s2_total = tb->meta.s2_bytes;

    // ---- launch shape: shrink stages / tile until shared memory fits -------
    uint32_t halo = align_up(std::max<uint32_t>(lmax - 1, 1), 16);
    uint32_t limit = smem_optin / cps - 1024;
    // The survivor-stage tables go to shared memory when they fit beside the
    // requested pipeline (or beside a two-stage one); otherwise they are read
    // from global memory (L2).
    // the shared memory of either scan kernel
    auto total = [&](uint32_t s2b, uint32_t st, uint32_t tl) {
        return role ? rf_smem_layout(fbytes, s2b, sv, st, tl, halo).total
                    : smem_layout(fbytes, s2b, warps, st, tl, halo).total;
    };
    uint32_t s2 = 0;
    if (s2_total <= limit) {
        if (total((uint32_t)s2_total, stages, tile) <= limit) {
            s2 = (uint32_t)s2_total;
        } else if (total((uint32_t)s2_total, 2, tile) <= limit) {
            s2 = (uint32_t)s2_total;
            stages = 2;
        }
    }
    uint32_t bytes = total(s2, stages, tile);
    while (bytes > limit) {
        if (stages > 2) --stages;
        else if (tile > 4 * halo && tile > 4096) tile /= 2;
        else return kNoRoom;
        tile = tile / 16 * 16;
        bytes = total(s2, stages, tile);
    }
    *tune = Tuning{warps, tile, stages, cps, halo, s2, bytes, sv};
    return RK_OK;
}

// Host part of rk_build: build the host image of the table and pick the
// launch shape for a device with smem_optin bytes of opt-in shared memory per
// block.  When the builder chooses the stage-1 filter and the shared memory
// cannot hold its pipeline, the next choice is tried: step 2, then no role
// filter.  No CUDA call.
int plan_table(const uint8_t *patterns, const uint32_t *lens, uint32_t k, const Opts &o,
               uint32_t smem_optin, TableBlob *tb, Tuning *tune) {
    // room for the static shared memory of each CTA
    if (smem_optin / o.cps <= 1024) return RK_EINVAL;
    const uint32_t tries[3] = {o.role, 2u, 1u};
    const uint32_t n = o.role == 0 ? 3 : 1;
    for (uint32_t i = 0; i < n; ++i) {
        const int rc = plan_with(patterns, lens, k, o, tries[i], smem_optin, tb, tune);
        if (rc != kNoRoom) return rc;
    }
    return RK_EINVAL;
}

rk_table_info make_info(const DevTable &d, const Tuning &tune, uint32_t n_grams,
                        uint32_t filter_log2_bits, uint32_t sfilter_log2_bits,
                        uint32_t rfilter_log2_bits, uint32_t sm_count,
                        uint32_t device, uint64_t device_bytes) {
    rk_table_info r{};
    r.n_patterns = d.n_patterns;
    r.min_len = d.lmin;
    r.max_len = d.lmax;
    r.n_lengths = d.n_lengths;
    r.gram_len = d.q;
    r.base_log2 = d.base_log2;
    r.filter = d.filter_mode == kFilterNone ? RK_FILTER_NONE
               : d.filter_mode == kFilterReplicated ? RK_FILTER_REPLICATED
                                                    : RK_FILTER_FLAT;
    r.filter_log2_bits = filter_log2_bits;
    r.filter_smem_bytes = d.filter_bytes;
    r.n_grams = n_grams;
    r.warps = tune.warps;
    r.tile_bytes = tune.tile_bytes;
    r.stages = tune.stages;
    r.ctas_per_sm = tune.ctas_per_sm;
    r.halo_bytes = tune.halo;
    r.smem_bytes = tune.smem_bytes;
    r.sm_count = sm_count;
    r.device = device;
    r.s2_smem_bytes = tune.s2_smem;
    r.device_bytes = device_bytes;
    r.sample_step = d.sample;
    r.sample_filter_log2_bits = sfilter_log2_bits;
    r.role_step = d.rf_step;
    r.role_filter_log2_bits = rfilter_log2_bits;
    r.role_side_log2_bits = d.rf_side_off ? 14u : 0u;
    r.survivor_warps = tune.sv_warps;
    return r;
}

}  // namespace
}  // namespace rk

extern "C" int rk_build(const uint8_t *patterns, const uint32_t *lens, uint32_t k,
                        const rk_build_opts *opts, rk_table **out) {
    if (!out) return RK_EINVAL;
    *out = nullptr;
    // bad patterns and options are rejected before any CUDA call
    Opts o{};
    int rc = read_opts(patterns, lens, k, opts, &o);
    if (rc) return rc;

    int dev = 0, sms = 0, smem_optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return RK_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return RK_ECUDA;
    if (cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
        cudaSuccess)
        return RK_ECUDA;

    TableBlob tb;
    Tuning tune{};
    rc = plan_table(patterns, lens, k, o, (uint32_t)smem_optin, &tb, &tune);
    if (rc) return rc;

    rk_table *t = new (std::nothrow) rk_table();
    if (!t) return RK_ENOMEM;
    t->device = dev;
    t->sm_count = sms;
    if (cudaMalloc(&t->d_mem, tb.bytes.size()) != cudaSuccess) {
        delete t;
        cudaGetLastError();
        return RK_ENOMEM;
    }
    t->d_bytes = tb.bytes.size();
    if (cudaMemcpy(t->d_mem, tb.bytes.data(), tb.bytes.size(), cudaMemcpyHostToDevice) !=
        cudaSuccess) {
        cudaFree(t->d_mem);
        delete t;
        return RK_ECUDA;
    }
    bind_blob(&t->dev, tb, (const uint8_t *)t->d_mem);
    t->tune = tune;
    t->n_grams = tb.n_grams;
    t->filter_log2_bits = tb.filter_log2_bits;
    t->sfilter_log2_bits = tb.sfilter_log2_bits;
    t->rfilter_log2_bits = tb.rfilter_log2_bits;
    t->filter_opt = o.filter;
    *out = t;
    return RK_OK;
}

extern "C" int rk_plan(const uint8_t *patterns, const uint32_t *lens, uint32_t k,
                       const rk_build_opts *opts, uint32_t smem_optin, rk_table_info *info) {
    if (!info) return RK_EINVAL;
    Opts o{};
    int rc = read_opts(patterns, lens, k, opts, &o);
    if (rc) return rc;
    TableBlob tb;
    Tuning tune{};
    rc = plan_table(patterns, lens, k, o, smem_optin, &tb, &tune);
    if (rc) return rc;
    *info = make_info(tb.meta, tune, tb.n_grams, tb.filter_log2_bits, tb.sfilter_log2_bits,
                      tb.rfilter_log2_bits, 0,
                      UINT32_MAX, tb.bytes.size());
    return RK_OK;
}

extern "C" void rk_destroy(rk_table *t) {
    if (!t) return;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != t->device) cudaSetDevice(t->device);
    if (t->s_copy) cudaStreamSynchronize(t->s_copy);
    if (t->s_comp) cudaStreamSynchronize(t->s_comp);
    for (cudaEvent_t e : t->events) cudaEventDestroy(e);
    if (t->s_copy) cudaStreamDestroy(t->s_copy);
    if (t->s_comp) cudaStreamDestroy(t->s_comp);
    cudaFree(t->h_text);
    cudaFree(t->h_keys);
    cudaFree(t->h_info);
    cudaFree(t->h_ws);
    cudaFree(t->d_mem);
    if (prev >= 0 && prev != t->device) cudaSetDevice(prev);
    delete t;
}

extern "C" int rk_table_info_get(const rk_table *t, rk_table_info *info) {
    if (!t || !info) return RK_EINVAL;
    *info = make_info(t->dev, t->tune, t->n_grams, t->filter_log2_bits, t->sfilter_log2_bits,
                      t->rfilter_log2_bits,
                      (uint32_t)t->sm_count, (uint32_t)t->device, t->d_bytes);
    return RK_OK;
}
