// Batched search: many texts, each with its own pattern table, scanned by one
// persistent kernel captured (with the sort and the per-item offsets) in a
// CUDA graph.
//
// Work is a list of chunks (item, first tile, tile count) that the
// producer thread of each CTA takes from a global counter, so long and short
// texts balance across SMs.  Each pipeline stage carries, beside the text
// tile, the item's stage-1 bit set (and, when chosen, its survivor tables):
// the producer copies them with the tile whenever that stage slot last held
// another table, so consumer warps never wait for each other.  Keys of a
// batch are (item << (id_bits + offset_bits)) | (id << offset_bits) | x, so
// the one sort leaves every item's matches together, in (id, x) order.
#include <algorithm>
#include <new>

#include "rk_scan_body.cuh"
#include "rk_sortws.cuh"

namespace rk {
namespace {

constexpr uint64_t kWaitTimeoutNs = 4000000000ull;
constexpr uint32_t kTilesPerChunk = 4;
constexpr uint32_t kEndItem = 0xFFFFFFFFu;

struct BatchItem {
    const DevTable *tab;
    const uint8_t *text;
    uint64_t n;
};

struct BatchDesc {
    uint32_t n_items, n_chunks;
    uint32_t work_counter;
    uint32_t pad;
};

struct BatchParams {
    const BatchItem *items;
    const uint4 *chunks;  // {item, first tile, tile count, 0}
    BatchDesc *desc;
    uint64_t *keys;
    uint64_t capacity;
    unsigned long long *info;
    uint32_t tile, stages, halo, warps;
    uint32_t fslot;      // bytes reserved per stage for a bit set
    uint32_t s2slot;     // bytes reserved per stage for survivor tables (0: read from L2)
    uint32_t ob, pb;     // offset and id field widths of a key
};

struct BatchLayout {
    uint32_t bar_off, desc_off, queue_off, mcount_off, match_off, stage_off;
    uint32_t stage_stride, filt_in_stage, s2_in_stage, text_in_stage;
    uint32_t total;
};

__host__ __device__ inline BatchLayout batch_layout(uint32_t warps, uint32_t stages,
                                                    uint32_t tile, uint32_t halo, uint32_t fslot,
                                                    uint32_t s2slot) {
    BatchLayout L{};
    uint32_t off = 0;
    L.bar_off = off;
    off = align_up(off + 2 * stages * 8, 16);
    L.desc_off = off;
    off = align_up(off + stages * 8, 16);
    L.queue_off = off;
    off = align_up(off + warps * kQueueCap * 2, 16);
    L.mcount_off = off;
    off = align_up(off + warps * 4, 16);
    L.match_off = off;
    off = align_up(off + warps * kMatchCap * 8, 128);
    L.stage_off = off;
    L.filt_in_stage = 0;
    L.s2_in_stage = align_up(fslot, 128);
    L.text_in_stage = L.s2_in_stage + align_up(s2slot, 128);
    L.stage_stride = align_up(L.text_in_stage + tile + halo + kStagePad, 128);
    off += stages * L.stage_stride;
    L.total = off;
    return L;
}

template <int MODE, bool Q4, int MAXW, bool S2S>
__global__ void __launch_bounds__((MAXW + 1) * 32, 1)
    rk_batch_tiles_kernel(const __grid_constant__ BatchParams P) {
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ volatile uint32_t s_abort;
    const BatchLayout lay = batch_layout(P.warps, P.stages, P.tile, P.halo, P.fslot, P.s2slot);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + lay.bar_off);
    uint64_t *empty = full + P.stages;
    uint2 *sdesc = reinterpret_cast<uint2 *>(smem + lay.desc_off);  // {item, tile}
    uint16_t *queues = reinterpret_cast<uint16_t *>(smem + lay.queue_off);
    uint32_t *mcount = reinterpret_cast<uint32_t *>(smem + lay.mcount_off);
    uint64_t *mbuf = reinterpret_cast<uint64_t *>(smem + lay.match_off);
    uint8_t *stage0 = smem + lay.stage_off;

    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t nw = P.warps;
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

    if (warp == nw) {  // ---------------- producer warp
        if (lane != 0) return;
        const uint32_t n_chunks = P.desc->n_chunks;
        const DevTable *slot_tab[8];
        for (uint32_t s = 0; s < 8; ++s) slot_tab[s] = nullptr;
        uint32_t item = 0, tile = 0, left = 0;
        uint64_t i = 0;
        bool aborted = false;
        for (;; ++i) {
            if (left == 0) {
                const uint32_t c = atomicAdd(&P.desc->work_counter, 1u);
                if (c >= n_chunks) break;
                const uint4 ch = P.chunks[c];
                item = ch.x;
                tile = ch.y;
                left = ch.z;
            }
            const uint32_t s = (uint32_t)(i % P.stages);
            if (i >= P.stages &&
                !mbar_wait_bounded(&empty[s], (uint32_t)((i / P.stages) + 1) & 1u, kWaitTimeoutNs)) {
                aborted = true;
                break;
            }
            if (s_abort) {
                aborted = true;
                break;
            }
            const BatchItem it = P.items[item];
            const DevTable *tab = it.tab;
            uint8_t *sb = stage0 + (size_t)s * lay.stage_stride;
            const uintptr_t addr = reinterpret_cast<uintptr_t>(it.text);
            const uint8_t *base = reinterpret_cast<const uint8_t *>(addr & ~uintptr_t(15));
            const uint64_t n16 = ((addr & 15u) + it.n + 15) & ~uint64_t(15);
            const uint64_t u0 = (uint64_t)tile * P.tile;
            const uint32_t halo = align_up(max(tab->lmax - 1u, 1u), 16u);
            const uint32_t bytes = (uint32_t)(min(n16, u0 + P.tile + halo) - u0);
            uint32_t fb = 0, sb2 = 0;
            if (slot_tab[s] != tab) {
                fb = MODE == kFilterNone ? 0 : tab->filter_bytes;
                sb2 = S2S ? tab->s2_bytes : 0;
                slot_tab[s] = tab;
            }
            sdesc[s] = make_uint2(item, tile);
            mbar_arrive_expect_tx(&full[s], bytes + fb + sb2);
            if (fb) bulk_g2s(sb + lay.filt_in_stage, tab->filter, fb, &full[s]);
            if (sb2) bulk_g2s(sb + lay.s2_in_stage, tab->s2_base, sb2, &full[s]);
            bulk_g2s(sb + lay.text_in_stage, base + u0, bytes, &full[s]);
            ++tile;
            --left;
        }
        if (aborted) {
            s_abort = 1;
            P.info[1] = RK_ETIMEOUT;
        } else {
            // end marker: consumers stop at the first stage that carries it
            const uint32_t s = (uint32_t)(i % P.stages);
            if (i < P.stages ||
                mbar_wait_bounded(&empty[s], (uint32_t)((i / P.stages) + 1) & 1u, kWaitTimeoutNs)) {
                sdesc[s] = make_uint2(kEndItem, 0);
                mbar_arrive(&full[s]);
            } else {
                s_abort = 1;
                P.info[1] = RK_ETIMEOUT;
            }
        }
        // On the normal path the consumers wait for every issued copy before
        // they reach the end marker.  After an abort they may not: then every
        // copy issued must land (bounded wait) before the CTA may exit.
        if (s_abort)
            for (uint64_t j = i > P.stages ? i - P.stages : 0; j < i; ++j)
                mbar_wait_bounded(&full[j % P.stages], (uint32_t)(j / P.stages) & 1u,
                                  kWaitTimeoutNs);
        return;
    }

    // -------------------------------------- consumer warps
    uint16_t *q = queues + warp * kQueueCap;
    WarpCtx w{mcount + warp, mbuf + (size_t)warp * kMatchCap, P.keys, P.capacity, P.info};
    const uint32_t lane4 = lane << 2;
    const uint32_t last = P.tile / 16u - 1u;
    uint32_t cur = kEndItem;
    WinCtx C{};
    uint32_t fmask = 0, qmask = 0xFFFFFFFFu;
    const DevTable *tab = nullptr;
    for (uint64_t i = 0;; ++i) {
        const uint32_t s = (uint32_t)(i % P.stages);
        if (!mbar_wait_bounded(&full[s], (uint32_t)(i / P.stages) & 1u, kWaitTimeoutNs)) {
            s_abort = 1;
            P.info[1] = RK_ETIMEOUT;
            break;
        }
        const uint2 d = sdesc[s];
        if (d.x == kEndItem) break;
        const uint8_t *sb = stage0 + (size_t)s * lay.stage_stride;
        if (d.x != cur) {
            cur = d.x;
            const BatchItem it = P.items[cur];
            tab = it.tab;
            const uint64_t mis = reinterpret_cast<uintptr_t>(it.text) & 15u;
            C.lo = mis;
            C.hi = mis + it.n;
            C.mis = mis;
            C.n = it.n;
            C.key_prefix = (uint64_t)cur << (P.ob + P.pb);
            C.pid_shift = P.ob;
            C.q = tab->q;
            C.gram_bits = tab->gram_bits;
            C.base_log2 = tab->base_log2;
            C.n_lengths = tab->n_lengths;
            fmask = tab->filter_mask;
            qmask = C.q == 4 ? 0xFFFFFFFFu : (1u << (8u * C.q)) - 1u;
            if (!S2S) C.s2 = make_s2(*tab, tab->s2_base);
        }
        if (S2S) {
            // the survivor tables sit in this stage's slot (placed there by
            // the producer for this or an earlier tile of the same table)
            DevTable tt;
            tt.s2_base = tab->s2_base;
            tt.grams = tab->grams;
            tt.gram_lens = tab->gram_lens;
            tt.group_hdr = tab->group_hdr;
            tt.slots = tab->slots;
            tt.group_pids = tab->group_pids;
            tt.pbytes = tab->pbytes;
            tt.poff = tab->poff;
            tt.lengths = tab->lengths;
            C.s2 = make_s2(tt, sb + lay.s2_in_stage);
        }
        const uint8_t *buf = sb + lay.text_in_stage;
        const uint64_t u0 = (uint64_t)d.y * P.tile;
        const uint64_t wend = min(u0 + P.tile, C.hi);
        const uint32_t nchunks = (uint32_t)((wend - u0 + 15) / 16);
        consume_tile<MODE, Q4>(C, w, q, buf, u0, nchunks, last, sb + lay.filt_in_stage, fmask,
                               lane4, qmask, warp, nw, lane);
        if (lane == 0) mbar_arrive(&empty[s]);
    }
    flush(w, lane);
}

// offsets[i] = index of the first key of item i (keys sorted), i = 0..n_items.
__global__ void rk_batch_offsets_kernel(const uint64_t *keys, const unsigned long long *info,
                                        uint64_t cap, const BatchDesc *desc, uint32_t shift,
                                        uint64_t *offsets) {
    const uint64_t M = info[0];
    const uint32_t n_items = desc->n_items;
    const bool ok = M <= cap && info[1] == RK_OK;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i <= n_items;
         i += gridDim.x * blockDim.x) {
        if (!ok) {
            offsets[i] = 0;
            continue;
        }
        const uint64_t target = (uint64_t)i << shift;
        uint64_t lo = 0, hi = M;
        while (lo < hi) {
            const uint64_t mid = (lo + hi) / 2;
            if (keys[mid] < target) lo = mid + 1;
            else hi = mid;
        }
        offsets[i] = i == n_items ? M : lo;
    }
}

uint32_t bits_for(uint64_t max_value) {
    uint32_t b = 0;
    while (b < 64 && (max_value >> b)) ++b;
    return b;
}

template <int MODE, bool Q4, int MAXW, bool S2S>
cudaError_t set_attr(uint32_t smem) {
    return cudaFuncSetAttribute(rk_batch_tiles_kernel<MODE, Q4, MAXW, S2S>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <int MODE, bool Q4, int MAXW, bool S2S>
cudaError_t launch_b(const BatchParams &p, uint32_t grid, uint32_t smem, cudaStream_t st) {
    rk_batch_tiles_kernel<MODE, Q4, MAXW, S2S><<<grid, (p.warps + 1) * 32, smem, st>>>(p);
    return cudaGetLastError();
}

template <int MODE, bool Q4>
cudaError_t dispatch_w(bool attr, const BatchParams &p, uint32_t grid, uint32_t smem,
                       cudaStream_t st) {
#define RK_B(MW, S)                                                    \
    return attr ? set_attr<MODE, Q4, MW, S>(smem) : launch_b<MODE, Q4, MW, S>(p, grid, smem, st)
    if (p.warps <= 8) {
        if (p.s2slot) { RK_B(8, true); } else { RK_B(8, false); }
    }
    if (p.warps <= 16) {
        if (p.s2slot) { RK_B(16, true); } else { RK_B(16, false); }
    }
    if (p.s2slot) { RK_B(31, true); } else { RK_B(31, false); }
#undef RK_B
}

cudaError_t dispatch(uint32_t mode, bool q4, bool attr, const BatchParams &p, uint32_t grid,
                     uint32_t smem, cudaStream_t st) {
    if (mode == kFilterNone)
        return q4 ? dispatch_w<kFilterNone, true>(attr, p, grid, smem, st)
                  : dispatch_w<kFilterNone, false>(attr, p, grid, smem, st);
    return q4 ? dispatch_w<kFilterFlat, true>(attr, p, grid, smem, st)
              : dispatch_w<kFilterFlat, false>(attr, p, grid, smem, st);
}

}  // namespace
}  // namespace rk

using namespace rk;

// ---------------------------------------------------------------- table sets

extern "C" int rk_tableset_build(uint32_t n_tables, const uint8_t *patterns, const uint32_t *lens,
                                 const uint32_t *patterns_per_table, const rk_build_opts *opts,
                                 rk_tableset **out) {
    if (!out) return RK_EINVAL;
    *out = nullptr;
    if (n_tables == 0 || !patterns_per_table) return RK_EINVAL;
    rk_build_opts o{};
    if (opts) o = *opts;
    const uint32_t base_log2 = o.base_log2 ? o.base_log2 : 8;
    if (base_log2 < 1 || base_log2 > 60) return RK_EINVAL;
    if (o.filter != RK_FILTER_AUTO && o.filter != RK_FILTER_FLAT && o.filter != RK_FILTER_NONE)
        return RK_EINVAL;
    const uint32_t filt = o.filter == RK_FILTER_NONE ? RK_FILTER_NONE : RK_FILTER_FLAT;
    uint64_t total_pats = 0;
    for (uint32_t i = 0; i < n_tables; ++i) total_pats += patterns_per_table[i];
    if (total_pats && (!patterns || !lens)) return RK_EINVAL;

    std::vector<TableBlob> blobs(n_tables);
    std::vector<size_t> at(n_tables);
    size_t size = 0;
    uint64_t pat_off = 0, byte_off = 0;
    rk_tableset *ts = new (std::nothrow) rk_tableset();
    if (!ts) return RK_ENOMEM;
    ts->n_tables = n_tables;
    ts->npat.assign(patterns_per_table, patterns_per_table + n_tables);
    ts->filter_mode = filt == RK_FILTER_NONE ? kFilterNone : kFilterFlat;
    ts->base_log2 = base_log2;
    ts->pat_first.resize(n_tables);
    ts->byte_first.resize(n_tables);
    for (uint32_t i = 0; i < n_tables; ++i) {
        const uint32_t k = patterns_per_table[i];
        if (k > RK_MAX_PATTERNS) { delete ts; return RK_EINVAL; }
        ts->pat_first[i] = pat_off;
        ts->byte_first[i] = byte_off;
        // table sets are scanned unsampled, with the prefix filter
        int rc = build_blob(patterns + byte_off, lens + pat_off, k, base_log2, filt,
                            o.filter_log2_bits, 1, 1, &blobs[i]);
        if (rc) { delete ts; return rc; }
        for (uint32_t j = 0; j < k; ++j) byte_off += lens[pat_off + j];
        pat_off += k;
        at[i] = size;
        size += blobs[i].bytes.size();  // each blob is a multiple of 256 bytes
        const DevTable &m = blobs[i].meta;
        ts->max_filter_bytes = std::max(ts->max_filter_bytes, m.filter_bytes);
        ts->max_s2_bytes = std::max(ts->max_s2_bytes, m.s2_bytes);
        ts->max_lmax = std::max(ts->max_lmax, m.lmax);
        ts->max_patterns = std::max(ts->max_patterns, k);
        if (m.q != 4) ts->all_q4 = false;
    }
    if (byte_off) ts->bytes.assign(patterns, patterns + byte_off);
    if (pat_off) ts->lens.assign(lens, lens + pat_off);
    const size_t tab_off = size;
    size += ws_align(sizeof(DevTable) * n_tables);
    if (cudaGetDevice(&ts->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&ts->sm_count, cudaDevAttrMultiProcessorCount, ts->device) !=
            cudaSuccess) {
        delete ts;
        return RK_ECUDA;
    }
    std::vector<uint8_t> host(size, 0);
    for (uint32_t i = 0; i < n_tables; ++i)
        std::copy(blobs[i].bytes.begin(), blobs[i].bytes.end(), host.begin() + at[i]);
    if (cudaMalloc(&ts->d_mem, size) != cudaSuccess) {
        cudaGetLastError();
        delete ts;
        return RK_ENOMEM;
    }
    ts->d_bytes = size;
    uint8_t *dm = (uint8_t *)ts->d_mem;
    DevTable *views = reinterpret_cast<DevTable *>(host.data() + tab_off);
    for (uint32_t i = 0; i < n_tables; ++i) bind_blob(&views[i], blobs[i], dm + at[i]);
    if (cudaMemcpy(dm, host.data(), size, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(ts->d_mem);
        delete ts;
        return RK_ECUDA;
    }
    ts->d_tables = reinterpret_cast<const DevTable *>(dm + tab_off);
    *out = ts;
    return RK_OK;
}

extern "C" void rk_tableset_destroy(rk_tableset *ts) {
    if (!ts) return;
    cudaFree(ts->d_mem);
    delete ts;
}

// ---------------------------------------------------------------- batches

struct rk_batch {
    const rk_tableset *ts = nullptr;
    int device = 0, sm_count = 0;
    rk_batch_opts opts{};
    uint32_t ob = 0, pb = 0, tb = 0;
    uint32_t max_chunks = 0;
    uint32_t smem = 0, halo = 0;
    void *d_mem = nullptr;
    BatchItem *d_items = nullptr;
    uint4 *d_chunks = nullptr;
    BatchDesc *d_desc = nullptr;
    uint64_t *d_keys = nullptr, *d_info = nullptr, *d_offsets = nullptr;
    void *d_ws = nullptr;
    uint64_t ws_bytes = 0;
    // host copies of the current batch (rebuilt into chunks when the tile changes)
    std::vector<BatchItem> h_items;
    std::vector<uint32_t> h_tab;  // table index of each item
    std::vector<uint4> h_chunks;
    BatchDesc h_desc{};
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap_stream = nullptr;
};

namespace {

BatchParams params_of(const rk_batch *b) {
    BatchParams p{};
    p.items = b->d_items;
    p.chunks = b->d_chunks;
    p.desc = b->d_desc;
    p.keys = b->d_keys;
    p.capacity = b->opts.capacity;
    p.info = reinterpret_cast<unsigned long long *>(b->d_info);
    p.tile = b->opts.tile_bytes;
    p.stages = b->opts.stages;
    p.halo = b->halo;
    p.warps = b->opts.warps;
    p.fslot = b->ts->filter_mode == kFilterNone ? 0 : b->ts->max_filter_bytes;
    p.s2slot = b->opts.s2_in_smem ? b->ts->max_s2_bytes : 0;
    p.ob = b->ob;
    p.pb = b->pb;
    return p;
}

uint32_t layout_bytes(const rk_batch *b, const rk_batch_opts &o) {
    const uint32_t fslot = b->ts->filter_mode == kFilterNone ? 0 : b->ts->max_filter_bytes;
    const uint32_t s2slot = o.s2_in_smem ? b->ts->max_s2_bytes : 0;
    return batch_layout(o.warps, o.stages, o.tile_bytes, b->halo, fslot, s2slot).total;
}

int smem_limit(const rk_batch *b, const rk_batch_opts &o, uint32_t *limit) {
    int optin = 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, b->device) !=
        cudaSuccess)
        return RK_ECUDA;
    *limit = (uint32_t)optin / o.ctas_per_sm - 1024;
    return RK_OK;
}

// Chunk list of the current items for the configured tile size.
void make_chunks(rk_batch *b) {
    b->h_chunks.clear();
    const uint32_t tile = b->opts.tile_bytes;
    for (uint32_t i = 0; i < b->h_items.size(); ++i) {
        const BatchItem &it = b->h_items[i];
        if (it.n == 0 || b->ts->npat[b->h_tab[i]] == 0) continue;
        const uint64_t mis = reinterpret_cast<uintptr_t>(it.text) & 15u;
        const uint32_t tiles = (uint32_t)((mis + it.n + tile - 1) / tile);
        for (uint32_t t0 = 0; t0 < tiles; t0 += kTilesPerChunk)
            b->h_chunks.push_back(make_uint4(i, t0, std::min(kTilesPerChunk, tiles - t0), 0));
    }
}

int upload(rk_batch *b, cudaStream_t st) {
    b->h_desc.n_items = (uint32_t)b->h_items.size();
    b->h_desc.n_chunks = (uint32_t)b->h_chunks.size();
    b->h_desc.work_counter = 0;
    if (b->h_chunks.size() > b->max_chunks) return RK_EINVAL;
    bool ok = true;
    if (!b->h_items.empty())
        ok = ok && cudaMemcpyAsync(b->d_items, b->h_items.data(),
                                   b->h_items.size() * sizeof(BatchItem), cudaMemcpyHostToDevice,
                                   st) == cudaSuccess;
    if (!b->h_chunks.empty())
        ok = ok && cudaMemcpyAsync(b->d_chunks, b->h_chunks.data(),
                                   b->h_chunks.size() * sizeof(uint4), cudaMemcpyHostToDevice,
                                   st) == cudaSuccess;
    ok = ok && cudaMemcpyAsync(b->d_desc, &b->h_desc, sizeof(BatchDesc), cudaMemcpyHostToDevice,
                               st) == cudaSuccess;
    ok = ok && cudaStreamSynchronize(st) == cudaSuccess;
    return ok ? RK_OK : RK_ECUDA;
}

// Enqueue one full batch run (scan, sort, offsets) on st.
int enqueue(rk_batch *b, cudaStream_t st, bool scan_only) {
    const BatchParams p = params_of(b);
    const uint32_t grid = (uint32_t)b->sm_count * b->opts.ctas_per_sm;
    if (cudaMemsetAsync(b->d_info, 0, 16, st) != cudaSuccess) return RK_ECUDA;
    if (cudaMemsetAsync(&b->d_desc->work_counter, 0, 4, st) != cudaSuccess) return RK_ECUDA;
    if (dispatch(b->ts->filter_mode, b->ts->all_q4, false, p, grid, b->smem, st) != cudaSuccess)
        return RK_ECUDA;
    if (scan_only) return RK_OK;
    uint32_t shifts[kMaxSortPasses], ns = 0;
    for (uint32_t s = 0; s < b->ob + b->pb + b->tb; s += 8) shifts[ns++] = s;
    int rc = launch_sort_shifts(b->sm_count, shifts, ns, b->d_keys, b->opts.capacity, b->d_info,
                                b->d_ws, b->ws_bytes, st, false);
    if (rc) return rc;
    const uint32_t blocks = std::max<uint32_t>(1, (b->opts.max_items + 1 + 255) / 256);
    rk_batch_offsets_kernel<<<std::min<uint32_t>(blocks, 1024), 256, 0, st>>>(
        b->d_keys, reinterpret_cast<const unsigned long long *>(b->d_info), b->opts.capacity,
        b->d_desc, b->ob + b->pb, b->d_offsets);
    return cudaGetLastError() == cudaSuccess ? RK_OK : RK_ECUDA;
}

int capture(rk_batch *b) {
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    const BatchParams p = params_of(b);
    if (dispatch(b->ts->filter_mode, b->ts->all_q4, true, p, 0, b->smem, nullptr) != cudaSuccess)
        return RK_ECUDA;
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return RK_ECUDA;
    int rc = enqueue(b, b->cap_stream, false);
    cudaError_t e = cudaStreamEndCapture(b->cap_stream, &g);
    if (rc || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return rc ? rc : RK_ECUDA;
    }
    e = cudaGraphInstantiate(&b->exec, g, 0);
    cudaGraphDestroy(g);
    return e == cudaSuccess ? RK_OK : RK_ECUDA;
}

int resolve(rk_batch *b, rk_batch_opts *o) {
    if (!o->warps) o->warps = 16;
    if (!o->tile_bytes) o->tile_bytes = 32768;
    if (!o->stages) o->stages = 2;
    if (!o->ctas_per_sm) o->ctas_per_sm = 1;
    if (o->warps < 1 || o->warps > 31 || o->tile_bytes < 1024 || o->tile_bytes % 16 ||
        o->tile_bytes > kMaxTileBytes || o->stages < 2 || o->stages > 8 || o->ctas_per_sm < 1 ||
        o->ctas_per_sm > 8)
        return RK_EINVAL;
    if (o->s2_in_smem && b->ts->max_s2_bytes > (1u << 17)) return RK_EINVAL;
    uint32_t limit = 0;
    int rc = smem_limit(b, *o, &limit);
    if (rc) return rc;
    return layout_bytes(b, *o) <= limit ? RK_OK : RK_EINVAL;
}

}  // namespace

extern "C" int rk_batch_create(const rk_tableset *ts, const rk_batch_opts *opts, rk_batch **out) {
    if (!out) return RK_EINVAL;
    *out = nullptr;
    if (!ts || !opts) return RK_EINVAL;
    rk_batch_opts o = *opts;
    if (o.max_items == 0 || o.max_text_len == 0 || o.max_text_len > RK_MAX_TEXT_LEN ||
        o.capacity >= (1ull << 32))
        return RK_EINVAL;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return RK_ECUDA;
    if (dev != ts->device) return RK_EINVAL;
    rk_batch *b = new (std::nothrow) rk_batch();
    if (!b) return RK_ENOMEM;
    b->ts = ts;
    b->device = dev;
    b->sm_count = ts->sm_count;
    b->halo = align_up(std::max<uint32_t>(ts->max_lmax - 1, 1), 16);
    b->ob = std::max<uint32_t>(1, bits_for(o.max_text_len - 1));
    b->pb = bits_for(ts->max_patterns ? ts->max_patterns - 1 : 0);
    b->tb = bits_for(o.max_items - 1);
    int rc = resolve(b, &o);
    if (rc || b->ob + b->pb + b->tb > 64) {
        delete b;
        return rc ? rc : RK_EINVAL;
    }
    b->opts = o;
    b->smem = layout_bytes(b, o);
    // enough chunks for the smallest tile allowed (1024 bytes): an item of n
    // bytes has at most (n + 15) / 1024 + 1 tiles, grouped kTilesPerChunk per chunk
    b->max_chunks = (uint32_t)std::min<uint64_t>(
        0xFFFFFFFFull,
        2ull * o.max_items + (o.max_total_bytes + 16ull * o.max_items) / (1024ull * kTilesPerChunk) +
            16);
    const uint64_t cap = std::max<uint64_t>(o.capacity, 2);
    b->ws_bytes = sort_ws_bytes(cap);
    const uint64_t o_items = 0;
    const uint64_t o_chunks = ws_align(o_items + sizeof(BatchItem) * o.max_items);
    const uint64_t o_desc = ws_align(o_chunks + sizeof(uint4) * b->max_chunks);
    const uint64_t o_info = ws_align(o_desc + sizeof(BatchDesc));
    const uint64_t o_off = ws_align(o_info + 16);
    const uint64_t o_keys = ws_align(o_off + 8ull * (o.max_items + 1));
    const uint64_t o_ws = ws_align(o_keys + 8ull * cap);
    const uint64_t total = o_ws + b->ws_bytes;
    if (cudaMalloc(&b->d_mem, total) != cudaSuccess) {
        cudaGetLastError();
        delete b;
        return RK_ENOMEM;
    }
    uint8_t *m = (uint8_t *)b->d_mem;
    b->d_items = reinterpret_cast<BatchItem *>(m + o_items);
    b->d_chunks = reinterpret_cast<uint4 *>(m + o_chunks);
    b->d_desc = reinterpret_cast<BatchDesc *>(m + o_desc);
    b->d_info = reinterpret_cast<uint64_t *>(m + o_info);
    b->d_offsets = reinterpret_cast<uint64_t *>(m + o_off);
    b->d_keys = reinterpret_cast<uint64_t *>(m + o_keys);
    b->d_ws = m + o_ws;
    if (cudaMemset(b->d_mem, 0, o_keys) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaFree(b->d_mem);
        delete b;
        return RK_ECUDA;
    }
    if ((rc = capture(b))) {
        rk_batch_destroy(b);
        return rc;
    }
    *out = b;
    return RK_OK;
}

extern "C" void rk_batch_destroy(rk_batch *b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->cap_stream) {
        cudaStreamSynchronize(b->cap_stream);
        cudaStreamDestroy(b->cap_stream);
    }
    cudaFree(b->d_mem);
    delete b;
}

extern "C" int rk_batch_set(rk_batch *b, uint32_t n_items, const uint32_t *table_of_item,
                            const uint8_t *const *d_texts, const uint64_t *text_lens,
                            void *stream) {
    if (!b || n_items > b->opts.max_items) return RK_EINVAL;
    if (n_items && (!table_of_item || !d_texts || !text_lens)) return RK_EINVAL;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != b->device) return RK_EINVAL;
    uint64_t total = 0;
    for (uint32_t i = 0; i < n_items; ++i) {
        if (table_of_item[i] >= b->ts->n_tables || text_lens[i] > b->opts.max_text_len ||
            (text_lens[i] && !d_texts[i]))
            return RK_EINVAL;
        total += text_lens[i];
    }
    if (total > b->opts.max_total_bytes) return RK_EINVAL;
    b->h_items.resize(n_items);
    b->h_tab.assign(table_of_item, table_of_item + n_items);
    for (uint32_t i = 0; i < n_items; ++i)
        b->h_items[i] = BatchItem{b->ts->d_tables + table_of_item[i], d_texts[i], text_lens[i]};
    make_chunks(b);  // empty texts and tables without patterns get no work
    return upload(b, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" int rk_batch_run(rk_batch *b, void *stream) {
    if (!b || !b->exec) return RK_EINVAL;
    return cudaGraphLaunch(b->exec, reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess
               ? RK_OK
               : RK_ECUDA;
}

extern "C" int rk_batch_results(const rk_batch *b, const uint64_t **d_keys,
                                const uint64_t **d_item_offsets, const uint64_t **d_info) {
    if (!b) return RK_EINVAL;
    if (d_keys) *d_keys = b->d_keys;
    if (d_item_offsets) *d_item_offsets = b->d_offsets;
    if (d_info) *d_info = b->d_info;
    return RK_OK;
}

extern "C" int rk_batch_info_get(const rk_batch *b, rk_batch_info *info) {
    if (!b || !info) return RK_EINVAL;
    rk_batch_info r{};
    r.offset_bits = b->ob;
    r.id_bits = b->pb;
    r.item_bits = b->tb;
    r.warps = b->opts.warps;
    r.tile_bytes = b->opts.tile_bytes;
    r.stages = b->opts.stages;
    r.ctas_per_sm = b->opts.ctas_per_sm;
    r.s2_in_smem = b->opts.s2_in_smem;
    r.smem_bytes = b->smem;
    r.n_chunks = (uint32_t)b->h_chunks.size();
    r.max_chunks = b->max_chunks;
    r.n_items = (uint32_t)b->h_items.size();
    *info = r;
    return RK_OK;
}

extern "C" int rk_batch_autotune(rk_batch *b, uint32_t max_candidates, uint32_t reps,
                                 double *best_ms, void *stream) {
    if (!b) return RK_EINVAL;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (!reps) reps = 3;
    const rk_batch_opts keep = b->opts;
    std::vector<rk_batch_opts> cand;
    for (uint32_t s2 : {0u, 1u})
        for (uint32_t tile : {16384u, 32768u, 49152u, 65536u})
            for (uint32_t warps : {8u, 16u, 24u})
                for (uint32_t stages : {2u, 3u, 4u})
                    for (uint32_t cps : {1u, 2u}) {
                        rk_batch_opts o = keep;
                        o.s2_in_smem = s2;
                        o.tile_bytes = tile;
                        o.warps = warps;
                        o.stages = stages;
                        o.ctas_per_sm = cps;
                        if (resolve(b, &o) == RK_OK) cand.push_back(o);
                    }
    if (max_candidates && cand.size() > max_candidates) {
        // keep an even spread of the candidate list
        std::vector<rk_batch_opts> pick;
        for (uint32_t i = 0; i < max_candidates; ++i)
            pick.push_back(cand[(size_t)i * cand.size() / max_candidates]);
        cand.swap(pick);
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return RK_ECUDA;
    }
    float best = -1.f;
    rk_batch_opts best_o = keep;
    for (const rk_batch_opts &o : cand) {
        b->opts = o;
        b->smem = layout_bytes(b, o);
        make_chunks(b);
        if (upload(b, st)) continue;
        const BatchParams p = params_of(b);
        if (dispatch(b->ts->filter_mode, b->ts->all_q4, true, p, 0, b->smem, nullptr) !=
            cudaSuccess)
            continue;
        enqueue(b, st, true);  // warm-up
        cudaEventRecord(e0, st);
        for (uint32_t r = 0; r < reps; ++r) enqueue(b, st, true);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= reps;
        if (best < 0 || ms < best) {
            best = ms;
            best_o = o;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->opts = best_o;
    b->smem = layout_bytes(b, best_o);
    make_chunks(b);
    int rc = upload(b, st);
    if (rc) return rc;
    if (best_ms) *best_ms = best;
    return capture(b);
}

extern "C" int rk_batch_read(const rk_batch *b, uint64_t *h_keys, uint64_t key_cap,
                             uint64_t *h_item_offsets, uint64_t *h_info, void *stream) {
    if (!b || !h_info) return RK_EINVAL;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    uint64_t info[2];
    if (cudaMemcpyAsync(info, b->d_info, 16, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return RK_ECUDA;
    h_info[0] = info[0];
    h_info[1] = info[1];
    if (info[1] != RK_OK || info[0] > b->opts.capacity) return RK_OK;
    const uint64_t nk = std::min<uint64_t>(info[0], key_cap);
    bool ok = true;
    if (h_item_offsets)
        ok = cudaMemcpyAsync(h_item_offsets, b->d_offsets, 8ull * (b->h_items.size() + 1),
                             cudaMemcpyDeviceToHost, st) == cudaSuccess;
    if (ok && h_keys && nk)
        ok = cudaMemcpyAsync(h_keys, b->d_keys, 8 * nk, cudaMemcpyDeviceToHost, st) == cudaSuccess;
    ok = ok && cudaStreamSynchronize(st) == cudaSuccess;
    return ok ? RK_OK : RK_ECUDA;
}
