// Internal definitions shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <vector>

#include "rk.h"

namespace rk {

// Mersenne prime modulus of the Rabin hash: p = 2^61 - 1.
constexpr uint64_t kP61 = (1ull << 61) - 1;

// Multipliers of the multiplicative hashes that place keys in tables.
constexpr uint32_t kFilterMult = 0x85EBCA77u;
constexpr uint32_t kGramMult = 0x9E3779B1u;
constexpr uint64_t kGroupMult = 0x9E3779B97F4A7C15ull;
constexpr uint32_t kRoleMult = 0x9E3779B1u;

enum FilterMode : uint32_t { kFilterNone = 0, kFilterReplicated = 1, kFilterFlat = 2 };

// One slot of a length group's hash table: the Rabin hash of some patterns of
// that length and the run [first, first+count) of their ids in group_pids.
struct GroupSlot {
    uint64_t h;
    uint32_t first;
    uint32_t count;  // 0 = empty slot
};

// One slot of the prefix map: a q-byte pattern prefix (little-endian value),
// the run [first, first+count) of distinct pattern lengths in gram_lens, and
// `ext`, a 32-bit fingerprint set of the next four bytes (bytes q..q+3) of
// the patterns with this prefix that are at least q + 4 bytes long; bit 31 of
// `count` (kGramShort) marks a prefix that also has a shorter pattern.
struct GramSlot {
    uint32_t key;
    uint32_t first;
    uint32_t count;  // 0 = empty slot; bit 31: some length is below q + 4
    uint32_t ext;
};
constexpr uint32_t kGramShort = 1u << 31;

// One slot of the sample map: a 4-byte gram (little-endian) and the set of
// offsets j (bit j, j < 4) at which it starts in some pattern; mask 0 = empty.
struct SampSlot {
    uint32_t key;
    uint32_t mask;
};

// Bit of `ext` for four bytes read as a little-endian word.
__host__ __device__ __forceinline__ uint32_t ext_bit(uint32_t w) {
    return (w * 0x9E3779B1u) >> 27;
}

// Device view of a table (pointers into one device allocation), passed to the
// scan kernel by value.
struct DevTable {
    const uint32_t *filter;   // shared-memory image of the stage-1 bit set
    uint32_t filter_bytes;    // bytes of that image
    uint32_t filter_mode;     // FilterMode
    uint32_t filter_mask;     // address mask (see scan kernel)
    uint32_t q;               // stage-1 key length in bytes, 1..4 (little-endian prefix)

    const GramSlot *grams;    // prefix map, 2^gram_bits slots
    uint32_t gram_bits;
    const uint32_t *gram_lens;

    const uint2 *group_hdr;   // per length L = 0..lmax: {first slot, log2 slots}; .y == 0: none
    const GroupSlot *slots;
    const uint32_t *group_pids;

    const uint8_t *pbytes;    // pattern bytes, each pattern 8-byte aligned, zero padded
    const uint64_t *poff;     // byte offset of each pattern in pbytes
    const uint32_t *plen;
    const uint32_t *lengths;  // distinct lengths, ascending
    uint32_t n_lengths;

    // Sampled stage 1 (sample == 4): every pattern has at least 7 bytes, so a
    // window starting at x has its position p = x + j (j < 4, p = 0 mod 4)
    // inside the pattern's first 7 bytes; stage 1 then tests only positions
    // p = 0 mod 4 against the patterns' 4-byte grams at offsets 0..3, and the
    // sample map gives each gram's offsets.
    uint32_t sample;          // 4, or 1: no sampled structures
    const uint32_t *sfilter;  // bit set of the grams (same layouts as `filter`)
    uint32_t sfilter_bytes, sfilter_mode, sfilter_mask;
    const SampSlot *smap;     // 2^smap_bits slots (in the survivor-stage tables)
    uint32_t smap_bits;

    // Role filter (rf_step 2 or 4; 0: none): stage 1 tests only positions p
    // that are multiples of rf_step, with the 4-byte gram G(p) = T[p..p+4)
    // read as a little-endian word.  The pattern grams at offsets j <
    // rf_step set role bits in a flat bit set: S, a gram that makes window
    // p - j a candidate on its own; L, a gram whose pattern continues with
    // the gram at offset j + 4; B, such a continuation.  Window p - j is a
    // candidate when G(p) has role S, or role L and G(p + 4) role B.  A word
    // of the bit set is chosen by the top bits of lo = G * kRoleMult, and
    // role i of G sits at bit (lo + 31 - i) mod 32 of it, so a rotation by
    // lo brings the roles to bits 31, 30, 29; S also sets bit 28 (both S
    // bits are tested).
    uint32_t rf_step;
    const uint32_t *rfilter;  // the bit set's shared-memory image (then the side set's)
    uint32_t rfilter_bytes;   // both images
    uint32_t rf_shift;        // byte address of G's word: (lo >> rf_shift) & ~3
    // Step 4 with patterns shorter than 7 bytes: byte offset of a side set
    // (2^14 bits replicated into the 32 banks) tested at the positions 2 mod
    // 4 for those patterns' grams at offsets 0 and 1 (0: none).
    uint32_t rf_side_off;

    uint32_t n_patterns;
    uint32_t lmin, lmax;
    uint32_t base_log2;

    // Every array above except the bit set lies in [s2_base, s2_base +
    // s2_bytes): the survivor-stage tables, which the scan kernel may copy to
    // shared memory as one block.
    const uint8_t *s2_base;
    uint32_t s2_bytes;
};

struct Tuning {
    uint32_t warps;        // consumer warps per CTA
    uint32_t tile_bytes;
    uint32_t stages;
    uint32_t ctas_per_sm;
    uint32_t halo;         // bytes staged after each tile (multiple of 16, >= 16)
    uint32_t s2_smem;      // survivor-stage table bytes copied to shared memory (0: global)
    uint32_t smem_bytes;   // dynamic shared memory per CTA
    uint32_t sv_warps;     // role-filter scans: survivor warps per CTA (0: other scans)
};

}  // namespace rk

// Host object behind the opaque handle.
struct rk_table {
    int device = 0;
    int sm_count = 0;
    rk::DevTable dev{};
    rk::Tuning tune{};
    uint32_t n_grams = 0;
    uint32_t filter_log2_bits = 0;
    uint32_t sfilter_log2_bits = 0;
    uint32_t rfilter_log2_bits = 0;
    uint32_t filter_opt = RK_FILTER_AUTO;
    void *d_mem = nullptr;
    size_t d_bytes = 0;

    // Buffers of the host-buffer search path, grown on demand.
    std::mutex host_mu;
    uint8_t *h_text = nullptr;  // device text buffer
    uint64_t h_text_cap = 0;
    uint64_t *h_keys = nullptr;
    uint64_t h_keys_cap = 0;
    uint64_t *h_info = nullptr;
    void *h_ws = nullptr;
    uint64_t h_ws_cap = 0;
    cudaStream_t s_copy = nullptr, s_comp = nullptr;
    std::vector<cudaEvent_t> events;
};

// Host object behind a table-set handle: many tables in one allocation.
struct rk_tableset {
    int device = 0, sm_count = 0;
    uint32_t n_tables = 0;
    void *d_mem = nullptr;
    size_t d_bytes = 0;
    const rk::DevTable *d_tables = nullptr;  // device array
    uint32_t filter_mode = rk::kFilterFlat;
    uint32_t max_filter_bytes = 0, max_s2_bytes = 0, max_lmax = 1, max_patterns = 0;
    bool all_q4 = true;
    uint32_t base_log2 = 8;
    std::vector<uint32_t> npat;  // patterns per table
    // host copy of the patterns (the serving loop builds plain tables from
    // them): table i's lengths start at lens[pat_first[i]], its bytes at
    // bytes[byte_first[i]]
    std::vector<uint8_t> bytes;
    std::vector<uint32_t> lens;
    std::vector<uint64_t> pat_first, byte_first;
};

namespace rk {

// Host image of one pattern table (all parts 256-byte aligned) and the
// offsets of its parts; `meta` holds the device view's non-pointer fields.
struct TableBlob {
    std::vector<uint8_t> bytes;
    size_t o_filter = 0, o_grams = 0, o_glens = 0, o_ghdr = 0, o_slots = 0, o_gpids = 0,
           o_pbytes = 0, o_poff = 0, o_plen = 0, o_lens = 0, o_sfilter = 0, o_smap = 0,
           o_rfilter = 0;
    DevTable meta{};
    uint32_t n_grams = 0, filter_log2_bits = 0, sfilter_log2_bits = 0, rfilter_log2_bits = 0;
};

// sample_opt: rk_build_opts.sample (1: no sampled structures); role_opt:
// rk_build_opts.role_step (0: chosen by the builder, 1: no role filter, 2 or
// 4: that step if the patterns allow it).
int build_blob(const uint8_t *patterns, const uint32_t *lens, uint32_t k, uint32_t base_log2,
               uint32_t filter_opt, uint32_t filter_bits_opt, uint32_t sample_opt,
               uint32_t role_opt, TableBlob *out);
void bind_blob(DevTable *d, const TableBlob &b, const uint8_t *dev_base);

// Candidate list of a scan whose survivors are verified in a second pass
// (entries: {text offset | prefix-map slot << 40, window bytes 0..7}).
struct CandList {
    ulonglong2 *list;
    uint64_t cap;
    unsigned long long *count;  // candidates offered (zeroed before the scan; may exceed cap)
};

// Scan windows whose start x lies in [x_begin, x_end) of a text of n bytes
// (bytes up to min(n, x_end + lmax - 1) must be resident); adds to d_info.
int launch_scan(const rk_table *t, const uint8_t *d_text, uint64_t n, uint64_t x_begin,
                uint64_t x_end, uint64_t *d_keys, uint64_t capacity, uint64_t *d_info,
                cudaStream_t stream, const CandList *cand = nullptr);

// launch_scan with an explicit wait limit; `withhold` makes the producer
// issue no copy (diagnostics: every consumer wait then runs out).  With a
// candidate list (can_defer(t) only), survivors stop after the prefix-map
// lookup and their candidates go to the list; launch_verify completes them.
int launch_scan_opts(const rk_table *t, const uint8_t *d_text, uint64_t n, uint64_t x_begin,
                     uint64_t x_end, uint64_t *d_keys, uint64_t capacity, uint64_t *d_info,
                     cudaStream_t stream, uint64_t timeout_ns, bool withhold,
                     const CandList *cand = nullptr);

// Tables whose survivors can be verified in a second pass: a stage-1 filter
// and prefix-map slot indices below 2^24.
bool can_defer(const rk_table *t);

// Hash, probe and verify every listed candidate of a deferred scan of
// d_text[0..n); matches are added to d_keys / d_info.
int launch_verify(const rk_table *t, const uint8_t *d_text, uint64_t n, const CandList &cand,
                  uint64_t *d_keys, uint64_t capacity, uint64_t *d_info, cudaStream_t stream);

int launch_sort(const rk_table *t, uint64_t n, uint64_t *d_keys, uint64_t capacity,
                const uint64_t *d_info, void *d_ws, uint64_t ws_bytes, cudaStream_t stream);

// Sort keys[0 .. d_info[0]) ascending over the 8-bit digits at the given bit
// shifts (least significant first).  allow_fused: outputs of up to 32 tiles
// per resident CTA may be sorted by one cooperative launch (every pass, grid
// barriers between phases) instead of one look-back kernel per pass.
int launch_sort_shifts(int sm_count, const uint32_t *shifts, uint32_t nshift, uint64_t *d_keys,
                       uint64_t capacity, const uint64_t *d_info, void *d_ws, uint64_t ws_bytes,
                       cudaStream_t stream, bool allow_fused);

uint64_t sort_workspace_bytes(uint64_t capacity);

// Kernels launch_sort starts for these arguments (on the current device).
uint32_t sort_launches(const rk_table *t, uint64_t n, uint64_t capacity);

int check_device(const rk_table *t);

}  // namespace rk

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------
#ifdef __CUDACC__
namespace rk {

// 61-bit rotation: x * 2^s mod p for x < p, 0 < s < 61 (2^61 = 1 mod p).
__device__ __forceinline__ uint64_t rotl61(uint64_t x, uint32_t s) {
    return ((x << s) | (x >> (61 - s))) & kP61;
}

// x mod p for any 64-bit x (one fold leaves at most p + 7).
__device__ __forceinline__ uint64_t fold61(uint64_t x) {
    uint64_t r = (x & kP61) + (x >> 61);
    return r >= kP61 ? r - kP61 : r;
}

__device__ __forceinline__ uint64_t addmod61(uint64_t a, uint64_t b) {  // a, b < p
    uint64_t s = a + b;
    return s >= kP61 ? s - kP61 : s;
}

__device__ __forceinline__ uint64_t submod61(uint64_t a, uint64_t b) {  // a, b < p
    return a >= b ? a - b : a + kP61 - b;
}

__device__ __forceinline__ uint64_t bswap64(uint64_t v) {
    uint32_t lo = (uint32_t)v, hi = (uint32_t)(v >> 32);
    return ((uint64_t)__byte_perm(lo, 0, 0x0123) << 32) | (uint64_t)__byte_perm(hi, 0, 0x0123);
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ---- mbarrier / bulk-copy wrappers (PTX ISA, sm_90+) ----
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

// Make initialised barriers visible to the bulk-copy (async) proxy.
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase with the given parity to complete, for at most
// timeout_ns of wall-clock time.  Returns false if it gave up.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity,
                                                  uint64_t timeout_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    uint64_t t0 = globaltimer_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (globaltimer_ns() - t0 > timeout_ns) return false;
    }
    return true;
}

// 1-D bulk copy global -> shared (no tensor map, no multicast); completion
// is signalled on `bar` as transaction bytes.  dst, src 16-byte aligned,
// bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                         uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

}  // namespace rk
#endif  // __CUDACC__
