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
//             prefilter: it can only drop windows that start no pattern);
//             or, with a role filter, only every 2nd or 4th position's
//             4-byte gram is looked up, and its roles (with those of the gram
//             4 bytes on) decide which of the windows it stands for survive.
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

#include "rk_scan_kernel.cuh"

namespace rk {

using scan::ScanParams;

namespace {

constexpr uint64_t kWaitTimeoutNs = 4000000000ull;  // 4 s per wait (default)

}  // namespace

int launch_scan(const rk_table *t, const uint8_t *d_text, uint64_t n, uint64_t x_begin,
                uint64_t x_end, uint64_t *d_keys, uint64_t capacity, uint64_t *d_info,
                cudaStream_t stream, const CandList *cand) {
    return launch_scan_opts(t, d_text, n, x_begin, x_end, d_keys, capacity, d_info, stream,
                            kWaitTimeoutNs, false, cand);
}

bool can_defer(const rk_table *t) {
    return t->dev.filter_mode != kFilterNone &&
           t->dev.gram_bits <= kCandClassShift - kCandSlotShift;
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
    // (a stage-1 round of a warp: 1 KiB, or 2 KiB with a step-4 role filter
    // without a side set)
    const uint64_t round_bytes =
        (uint64_t)tu.warps * (t->dev.rf_step == 4 && !t->dev.rf_side_off ? 2048u : 1024u);
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
    uint32_t grid = (uint32_t)(p.n_tiles < max_ctas ? p.n_tiles : max_ctas);
    uint32_t threads = (tu.warps + 1) * 32;
    bool q4 = t->dev.q == 4;
    const uint32_t sm = tu.smem_bytes;
    cudaError_t e;
    if (t->dev.rf_step) {
        // every scan of a table with a role filter runs its own kernel, with
        // that bit set staged and survivor warps beside the stage-1 warps
        p.tab.filter = t->dev.rfilter;
        p.tab.filter_bytes = t->dev.rfilter_bytes;
        p.sv_warps = tu.sv_warps;
        threads = (tu.warps + tu.sv_warps + 1) * 32;
        e = scan::launch_role(p, grid, threads, sm, stream, t->dev.rf_step,
                              t->dev.rf_side_off != 0);
        return e == cudaSuccess ? RK_OK : RK_ECUDA;
    }
    // a deferred scan of a sampled table stages the grams' bit set instead
    const bool samp = p.cand.list && t->dev.sample == 4;
    if (samp) {
        p.tab.filter = t->dev.sfilter;
        p.tab.filter_bytes = t->dev.sfilter_bytes;
        p.tab.filter_mode = t->dev.sfilter_mode;
        p.tab.filter_mask = t->dev.sfilter_mask;
    }
    switch (p.tab.filter_mode) {
        case kFilterNone: e = scan::launch_none(p, grid, threads, sm, stream, q4); break;
        case kFilterReplicated:
            e = scan::launch_replicated(p, grid, threads, sm, stream, q4, samp);
            break;
        default: e = scan::launch_flat(p, grid, threads, sm, stream, q4, samp); break;
    }
    return e == cudaSuccess ? RK_OK : RK_ECUDA;
}

}  // namespace rk
