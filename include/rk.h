/*
 * rk.h - C ABI of a multi-pattern Rabin-Karp matcher for one GB300 GPU.
 *
 * Problem (Shah & Oza, "Improved Parallel Rabin-Karp Algorithm Using CUDA",
 * Section 1): find every occurrence of every pattern of a set in a byte text.
 * The result is the set of matches
 *
 *     { (id, x) : 0 <= id < k, 0 <= x <= n - len_id, T[x .. x+len_id) == P_id }
 *
 * with one window per text offset x (Section 3.1; the GPU listing's bound
 * x <= n - m, so the last window counts), bytes compared as unsigned values,
 * every pattern index reported on its own (duplicate patterns included), and
 * the list returned in ascending (id, x) order.
 *
 * Each match is one 64-bit key  key = (id << 40) | x  (RK_KEY below), so the
 * ascending key order is the ascending (id, x) order.
 *
 * Conventions for every entry point:
 *   - the return value is an RK_* status code; nothing aborts, throws or traps;
 *   - "d_" pointers are device pointers on the table's device, "h_" pointers
 *     host pointers; the caller owns every buffer it passes in;
 *   - the library owns rk_table objects (rk_build / rk_destroy);
 *   - a table is read-only after rk_build and may serve concurrent searches on
 *     different streams, except rk_search (host buffers), which serialises
 *     calls on one table;
 *   - "stream" is a cudaStream_t passed as void* (NULL = legacy default
 *     stream); *_device calls are asynchronous with respect to the host;
 *   - the current CUDA device must be the table's device (else RK_EINVAL).
 */
#ifndef RK_H
#define RK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define RK_OK 0
#define RK_EINVAL 1      /* bad argument (null pointer, size or limit out of range) */
#define RK_ENOMEM 2      /* a host or device allocation failed */
#define RK_ECAPACITY 3   /* more matches than the output can hold; count reported */
#define RK_ECUDA 4       /* a CUDA runtime call or kernel launch failed */
#define RK_ETIMEOUT 5    /* a bounded device-side wait gave up (pipeline stalled) */

/* ---- limits ------------------------------------------------------------ */
#define RK_MAX_PATTERN_LEN 4096u            /* bytes per pattern */
#define RK_MAX_PATTERNS ((1u << 24) - 1u)   /* patterns per table */
#define RK_MAX_TEXT_LEN ((1ull << 40) - 1u) /* bytes per text */

/* ---- match keys -------------------------------------------------------- */
#define RK_KEY_OFFSET_BITS 40
#define RK_KEY(id, x) ((((uint64_t)(id)) << RK_KEY_OFFSET_BITS) | (uint64_t)(x))
#define RK_KEY_ID(key) ((uint32_t)((key) >> RK_KEY_OFFSET_BITS))
#define RK_KEY_OFFSET(key) ((uint64_t)(key) & ((1ull << RK_KEY_OFFSET_BITS) - 1u))

/* ---- device result header ---------------------------------------------- */
/* d_info points to two uint64_t in device memory:
 *   d_info[0]  number of matches found (may exceed the capacity passed in);
 *   d_info[1]  RK_OK, or RK_ETIMEOUT if a bounded device wait gave up.       */
#define RK_INFO_COUNT 0
#define RK_INFO_STATUS 1

/* ---- stage-1 prefilter choice (see rk_build_opts.filter) ---------------- */
#define RK_FILTER_AUTO 0        /* pick by pattern count (default) */
#define RK_FILTER_REPLICATED 1  /* bit set copied into all 32 shared-memory banks */
#define RK_FILTER_FLAT 2        /* one larger bit set */
#define RK_FILTER_NONE 3        /* no prefilter: every window hashed at every length */

typedef struct rk_table rk_table;

/* Build options; a zero field means "default".  Pass NULL for all defaults. */
typedef struct rk_build_opts {
    uint32_t base_log2;        /* Rabin base B = 2^base_log2, 1..60 (default 8, B = 256);
                                  1 is the paper's shift-add base 2 */
    uint32_t filter;           /* RK_FILTER_* */
    uint32_t filter_log2_bits; /* prefilter size in bits, log2 (default: by pattern count) */
    uint32_t warps;            /* consumer warps per CTA, 1..31 (default 24; with a role
                                  filter: stage-1 warps, default 16, plus up to 6 survivor
                                  warps within 31) */
    uint32_t tile_bytes;       /* text bytes per pipeline tile, multiple of 16, <= 65536
                                  (default 49152) */
    uint32_t stages;           /* tiles in flight per CTA, 2..8 (default 2) */
    uint32_t ctas_per_sm;      /* resident CTAs per SM (default 1) */
    uint32_t sample;           /* 0: when every pattern has >= 7 bytes and no role filter is
                                  built, scans with a candidate list (rk_scan_device_ws) test
                                  every 4th window position against the patterns' 4-byte
                                  grams at offsets 0..3; 1: every position against the
                                  prefixes */
    uint32_t role_step;        /* role filter (see below): 0 = the builder's choice (with
                                  filter RK_FILTER_AUTO; none with a forced filter), 1 = none,
                                  2 or 4 = that sampling step when the patterns allow it.
                                  A role filter tests every 2nd or 4th text position p with
                                  the 4 bytes at p: those bytes stand for the pattern bytes
                                  j..j+3 of a window starting at p - j, either on their own
                                  (shorter patterns) or together with the 4 bytes at p + 4
                                  (the pattern bytes j+4..j+7).  Step 4 covers patterns
                                  shorter than 7 bytes with a side set tested at the other
                                  even positions; both steps take patterns of 4 bytes or more
                                  (at most 64 of exactly 4).  The builder takes step 4 when
                                  every pattern has 7 bytes or more (a side set only when
                                  asked for), else step 2, and declines a set with more than
                                  one gram per 16 bits of the
                                  filter's largest size (2^19 bits), or more than 1024
                                  side-set grams, where the other filters pass fewer windows.
                                  Every scan of the table uses it. */
} rk_build_opts;

/* Read-back of a table's shape and launch configuration. */
typedef struct rk_table_info {
    uint32_t n_patterns, min_len, max_len, n_lengths;
    uint32_t gram_len;         /* q: bytes of the stage-1 key (min(4, min_len)) */
    uint32_t base_log2;
    uint32_t filter, filter_log2_bits, filter_smem_bytes;
    uint32_t n_grams;          /* distinct q-byte pattern prefixes */
    uint32_t warps, tile_bytes, stages, ctas_per_sm, halo_bytes, smem_bytes;
    uint32_t sm_count;
    uint32_t device;
    uint32_t s2_smem_bytes;    /* survivor-stage tables staged in shared memory (0: read from L2) */
    uint64_t device_bytes;     /* device memory held by the table */
    uint32_t sample_step;      /* 4: sampled stage 1 available (see rk_build_opts.sample), else 1 */
    uint32_t sample_filter_log2_bits;  /* its bit set's size (0 without) */
    uint32_t role_step;        /* 2 or 4: the scans use a role filter (rk_build_opts.role_step);
                                  0: none */
    uint32_t role_filter_log2_bits;    /* its bit set's size (0 without) */
    uint32_t survivor_warps;   /* role filter: warps per CTA that handle the windows stage 1
                                  passes (warps counts the stage-1 warps); 0 without */
    uint32_t role_side_log2_bits;  /* step-4 role filter over patterns shorter than 7 bytes:
                                  size of the side set that covers them at the positions
                                  2 mod 4 (14; 0 without) */
} rk_table_info;

/* Human-readable text of a status code (static storage). */
const char *rk_strerror(int status);

/* Build the pattern table (Section 3.1: the pattern hash is computed once on
 * the host and handed to the kernel; here one table serves a whole set).
 *   patterns   all pattern bytes concatenated (pattern i follows pattern i-1);
 *   lens       n_patterns lengths, each 1..RK_MAX_PATTERN_LEN;
 *   n_patterns 0..RK_MAX_PATTERNS (0 gives a table that never matches);
 *   opts       NULL or options; *out receives the table.
 * Pattern ids are the indices 0..n_patterns-1.  The bytes are copied; the
 * table lives in device memory of the current device until rk_destroy.
 * Errors: RK_EINVAL (null pointer, empty or overlong pattern, bad option),
 * RK_ENOMEM, RK_ECUDA.  On error *out is set to NULL.                        */
int rk_build(const uint8_t *patterns, const uint32_t *lens, uint32_t n_patterns,
             const rk_build_opts *opts, rk_table **out);

/* The shape and launch configuration rk_build would give these patterns and
 * options on a device whose opt-in shared memory per block is smem_optin
 * bytes (cudaDevAttrMaxSharedMemoryPerBlockOptin; 232448 on GB300), worked
 * out on the host: no CUDA call and no device memory, so a caller can size a
 * table before building it.  Arguments as rk_build; info receives what
 * rk_table_info_get would report for the built table, except sm_count (0)
 * and device (UINT32_MAX); device_bytes is the size of the table's device
 * allocation.  Errors: RK_EINVAL (as rk_build; null info; smem_optin too
 * small for the requested CTAs per SM or for the longest pattern's halo).  */
int rk_plan(const uint8_t *patterns, const uint32_t *lens, uint32_t n_patterns,
            const rk_build_opts *opts, uint32_t smem_optin, rk_table_info *info);

/* Free a table (NULL is ignored).  No search may be in flight on it. */
void rk_destroy(rk_table *t);

/* Read back a table's shape and launch configuration (host only, no CUDA
 * call).  Errors: RK_EINVAL (t or info NULL).                               */
int rk_table_info_get(const rk_table *t, rk_table_info *info);

/* Bytes of device workspace rk_sort_device / rk_search_device need for an
 * output of `capacity` keys (0 on bad arguments). */
uint64_t rk_workspace_bytes(const rk_table *t, uint64_t capacity);

/* Scan (Section 3.1 GPU listing, rebuilt: staged tiles, per-window Rabin
 * hashes mod 2^61-1, probes of tables grouped by pattern length, byte-exact
 * verification, warp-aggregated emission).  Appends the unsorted keys of all
 * matches in d_text[0..n) to d_keys[0..capacity) and sets d_info.
 *   d_text     n bytes of device memory, any alignment; n <= RK_MAX_TEXT_LEN;
 *   d_keys     capacity uint64_t of device memory, 8-byte aligned;
 *   d_info     2 uint64_t of device memory (zeroed by this call).
 * If d_info[0] > capacity, only `capacity` keys were stored (which ones is
 * unspecified): retry with a larger buffer.  Errors: RK_EINVAL, RK_ECUDA.    */
int rk_scan_device(const rk_table *t, const uint8_t *d_text, uint64_t n, uint64_t *d_keys,
                   uint64_t capacity, uint64_t *d_info, void *stream);

/* Sort the keys left by rk_scan_device ascending (= ascending (id, x)), in
 * place, reading the count from d_info on the device.  Does nothing when
 * d_info[0] > capacity.  n must be the text length given to the scan.
 * Outputs of up to 32 tiles of 2048 keys per resident CTA are sorted by one
 * cooperative launch (all digit passes, grid barriers between phases);
 * larger ones by one decoupled look-back kernel per pass.
 *   d_workspace  at least rk_workspace_bytes(t, capacity) bytes, 16-byte aligned.
 * Errors: RK_EINVAL, RK_ECUDA.                                               */
int rk_sort_device(const rk_table *t, uint64_t n, uint64_t *d_keys, uint64_t capacity,
                   const uint64_t *d_info, void *d_workspace, uint64_t workspace_bytes,
                   void *stream);

/* Kernels rk_sort_device launches on the current device for a text of n
 * bytes and an output of `capacity` keys (the memory clear of its control
 * words is not counted).  Errors: RK_EINVAL (t or launches NULL).           */
int rk_sort_launches(const rk_table *t, uint64_t n, uint64_t capacity, uint32_t *launches);

/* Bytes of device workspace rk_scan_device_ws needs for a text of n bytes:
 * a candidate count and a list of up to n / 64 + 4096 candidates, 16 bytes
 * each (0 on bad arguments). */
uint64_t rk_scan_workspace_bytes(const rk_table *t, uint64_t n);

/* rk_scan_device with the survivors' Rabin hash, table probe and byte
 * comparison (Section 3.1's hx == hy test and compare(P, T + x, m)) moved to
 * a second kernel: the tiled scan only lists each window whose exact q-byte
 * prefix starts some pattern and whose next four bytes pass that prefix's
 * fingerprint set; the second kernel takes the list 32 windows per warp and
 * reads them from d_text.  Same match set as rk_scan_device (the order of
 * the unsorted keys differs).  Windows offered beyond the list's room are
 * verified inside the scan as rk_scan_device does.
 *   d_workspace  at least rk_scan_workspace_bytes(t, n) bytes, 16-byte
 *                aligned, not shared with a call in flight; a smaller,
 *                unaligned or null workspace, a table built with
 *                RK_FILTER_NONE, or one with more than 2^21 distinct q-byte
 *                prefixes (a candidate holds its prefix-map slot in 22 bits)
 *                runs rk_scan_device instead.
 * Other arguments, results and errors as rk_scan_device.                    */
int rk_scan_device_ws(const rk_table *t, const uint8_t *d_text, uint64_t n, uint64_t *d_keys,
                      uint64_t capacity, uint64_t *d_info, void *d_workspace,
                      uint64_t workspace_bytes, void *stream);

/* rk_scan_device_ws that also records the CUDA event mid_event (a
 * cudaEvent_t created by the caller on the current device; NULL: none) on
 * the stream after the tile scan is launched and before the verification
 * kernel is, so that events recorded around the call time the two kernels
 * apart.  When the scan runs as one kernel the event is recorded after it.
 * On return from a deferring call the workspace's first 8 bytes hold, once
 * the stream reaches them, the number of candidate windows the tile scan
 * listed (a uint64_t; it may exceed the list's room).
 * Errors: as rk_scan_device_ws; RK_ECUDA if the event cannot be recorded.   */
int rk_scan_device_ws_split(const rk_table *t, const uint8_t *d_text, uint64_t n,
                            uint64_t *d_keys, uint64_t capacity, uint64_t *d_info,
                            void *d_workspace, uint64_t workspace_bytes, void *stream,
                            void *mid_event);

/* Kernels rk_scan_device_ws launches for a text of n bytes and a workspace
 * of workspace_bytes: 2 (tile scan + verification) when it defers, 1 when it
 * runs rk_scan_device, 0 for an empty text or table (memory clears are not
 * counted).  Errors: RK_EINVAL (t or launches NULL).                        */
int rk_scan_launches(const rk_table *t, uint64_t n, uint64_t workspace_bytes,
                     uint32_t *launches);

/* rk_scan_device followed by rk_sort_device on one stream: the sorted match
 * list of d_text[0..n) in d_keys, its length in d_info[0].
 *   d_workspace  16-byte aligned; at least rk_workspace_bytes(t, capacity)
 *                bytes when capacity >= 2 (the sort's).  With
 *                rk_workspace_bytes(t, capacity) + rk_scan_workspace_bytes(t, n)
 *                bytes the scan part runs as rk_scan_device_ws, its list
 *                placed after the sort's workspace.
 * Errors: as rk_scan_device and rk_sort_device.                              */
int rk_search_device(const rk_table *t, const uint8_t *d_text, uint64_t n, uint64_t *d_keys,
                     uint64_t capacity, uint64_t *d_info, void *d_workspace,
                     uint64_t workspace_bytes, void *stream);

/* Host-buffer search (Section 1's problem on a host text; the whole of
 * Section 3.1's GPU path: the text copied to the device, the kernel, the
 * result copied back): copies h_text to the device in chunks (overlapping the
 * copies with the scan), sorts, and copies the sorted keys back.  Blocks until
 * done.  *n_matches receives the match count; if it exceeds capacity the call
 * returns RK_ECAPACITY and h_keys is left untouched.  Device buffers are cached
 * on the table between calls and freed by rk_destroy.
 * Errors: RK_EINVAL, RK_ENOMEM, RK_ECAPACITY, RK_ECUDA, RK_ETIMEOUT.         */
int rk_search(const rk_table *t, const uint8_t *h_text, uint64_t n, uint64_t *h_keys,
              uint64_t capacity, uint64_t *n_matches);

/* ---- match records ---------------------------------------------------------
 * The result of Section 1's problem as records instead of packed keys, and a
 * table built from one pointer per pattern: thin calls over rk_build,
 * rk_search and rk_search_device.  The record list is in ascending
 * (pattern_id, offset) order, like the keys.                                */
typedef struct rk_match {
    uint64_t offset;      /* the match starts at text byte `offset` */
    uint32_t pattern_id;  /* index of the pattern in the set */
    uint32_t reserved;    /* 0 */
} rk_match;

/* rk_build with the patterns given as n_patterns pointers (patterns[i] points
 * to lens[i] bytes; the bytes are copied).  Errors as rk_build (a null
 * pattern pointer: RK_EINVAL).                                              */
int rk_build_ptrs(const uint8_t *const *patterns, const uint32_t *lens, uint32_t n_patterns,
                  const rk_build_opts *opts, rk_table **out);

/* Host-buffer search returning a record list the library allocates: on
 * RK_OK, *out holds *n_out records (free it with rk_free_matches; it is a
 * valid pointer even when *n_out is 0).  Blocks until done.  Runs
 * rk_search, twice when its first guess at the count was short.  On error
 * *out is NULL and *n_out 0.  Errors: as rk_search (RK_ECAPACITY only for
 * 2^32 or more matches).                                                    */
int rk_search_matches(const rk_table *t, const uint8_t *h_text, uint64_t n, rk_match **out,
                      uint64_t *n_out);

/* Device-buffer search into records: rk_search_device on `stream` with the
 * table's cached workspace, the sorted keys turned into records in
 * d_out[0..capacity) (device memory, 8-byte aligned), then the count copied
 * back: the call waits for `stream`.  *n_out (host memory) receives the
 * match count; if it exceeds capacity the call returns RK_ECAPACITY and
 * d_out holds no valid list (call again with *n_out records of room).  Calls
 * on one table are serialised (the cached workspace).
 * Errors: RK_EINVAL, RK_ENOMEM, RK_ECAPACITY, RK_ECUDA, RK_ETIMEOUT.         */
int rk_search_device_matches(const rk_table *t, const uint8_t *d_text, uint64_t n, void *stream,
                             rk_match *d_out, uint64_t capacity, uint64_t *n_out);

/* Free a record list from rk_search_matches (NULL is ignored).              */
void rk_free_matches(rk_match *m);

/* Rabin hash of every length-L window (Section 3.1's hash h = h*B + c,
 * reduced mod 2^61-1, B = 2^base_log2), by a tiled rolling update:
 *   d_hashes[x] = sum_{i<L} d_text[x+i] * B^(L-1-i)  mod (2^61 - 1),
 *   x = 0 .. n-L  (nothing is written when L > n).
 * L in 1..RK_MAX_PATTERN_LEN, base_log2 in 1..60.  Errors: RK_EINVAL, RK_ECUDA. */
int rk_window_hashes_device(const uint8_t *d_text, uint64_t n, uint32_t L, uint32_t base_log2,
                            uint64_t *d_hashes, void *stream);

/* The paper's own GPU matcher (Section 3.1, GPU listing), kept as a measured
 * comparison point: one pattern h_pattern[0..m) (host memory); one thread per
 * text offset x = 0 .. n-m; the shift-add hash hy = (hy << 1) + T[x+i]
 * recomputed over each window from global memory (64-bit, wrapping); a byte
 * comparison when hy equals the pattern's hash, computed on the host; then
 * d_result[x] = 1.  d_result: n bytes of device memory, zeroed by the call
 * (1 = a match starts at x).  threads_per_block: multiple of 32, <= 1024
 * (0: 1024), the paper's Table 1 parameter.  Asynchronous on `stream`.
 * Errors: RK_EINVAL, RK_ECUDA.                                               */
int rk_paper_search_device(const uint8_t *d_text, uint64_t n, const uint8_t *h_pattern, uint32_t m,
                           uint8_t *d_result, uint32_t threads_per_block, void *stream);

/* The GPU architecture the library's kernels were built for, as
 * cudaFuncGetAttributes reports it on the current device (major * 10 +
 * minor: 103 for sm_103a).  Errors: RK_EINVAL (null), RK_ECUDA.             */
int rk_debug_binary_version(int *version);

/* Diagnostics for failure detection: rk_scan_device with the producer
 * issuing no copy, so every pipeline wait runs out after timeout_ms
 * (1..10000).  The kernel then writes RK_ETIMEOUT to d_info[1] and returns;
 * nothing faults and the context stays usable.  Errors: RK_EINVAL, RK_ECUDA. */
int rk_debug_scan_withheld(const rk_table *t, const uint8_t *d_text, uint64_t n, uint64_t *d_keys,
                           uint64_t capacity, uint64_t *d_info, uint32_t timeout_ms, void *stream);

/* ---- batched search --------------------------------------------------------
 * Many texts, each searched with its own pattern table, in one launch: the
 * persistent batched kernel with its sort captured in a CUDA graph.
 *
 * A match of a batch is one key
 *     key = (item << (id_bits + offset_bits)) | (id << offset_bits) | x
 * (field widths in rk_batch_info), so ascending keys list every item's matches
 * together, in ascending (pattern id, offset) order; the item offsets give
 * where each item's run starts.                                              */
typedef struct rk_tableset rk_tableset;
typedef struct rk_batch rk_batch;

/* n_tables pattern tables in one device allocation.  patterns holds all
 * tables' patterns concatenated (table 0 first), lens their lengths,
 * patterns_per_table[i] the count of table i (ids restart at 0 per table; 0
 * patterns allowed).  opts: NULL or base_log2, filter (RK_FILTER_AUTO or
 * RK_FILTER_FLAT: a flat bit set; RK_FILTER_NONE: no prefilter) and
 * filter_log2_bits; the launch fields are ignored.
 * Errors: RK_EINVAL, RK_ENOMEM, RK_ECUDA.                                    */
int rk_tableset_build(uint32_t n_tables, const uint8_t *patterns, const uint32_t *lens,
                      const uint32_t *patterns_per_table, const rk_build_opts *opts,
                      rk_tableset **out);
/* Free a table set (NULL is ignored).  No batch or server may still use it. */
void rk_tableset_destroy(rk_tableset *ts);

typedef struct rk_batch_opts {
    uint32_t max_items;        /* texts per batch, >= 1 */
    uint64_t max_text_len;     /* longest text, >= 1 (sets offset_bits) */
    uint64_t max_total_bytes;  /* most text bytes in one batch */
    uint64_t capacity;         /* match keys per batch, < 2^32 */
    uint32_t warps;            /* consumer warps per CTA (default 16) */
    uint32_t tile_bytes;       /* bytes per tile, multiple of 16, <= 65536 (default 32768) */
    uint32_t stages;           /* tiles in flight per CTA (default 2) */
    uint32_t ctas_per_sm;      /* resident CTAs per SM (default 1) */
    uint32_t s2_in_smem;       /* 1: the survivor tables travel with each tile into shared
                                  memory; 0: they are read from L2 (default) */
} rk_batch_opts;

typedef struct rk_batch_info {
    uint32_t offset_bits, id_bits, item_bits;  /* key fields */
    uint32_t warps, tile_bytes, stages, ctas_per_sm, s2_in_smem, smem_bytes;
    uint32_t n_chunks, max_chunks;             /* work chunks of the current batch */
    uint32_t n_items;                          /* items of the current batch */
} rk_batch_info;

/* A batch engine over a table set: device buffers for opts' limits and the
 * captured graph.  The table set must outlive the batch.
 * Errors: RK_EINVAL (limits, fields wider than 64 bits), RK_ENOMEM, RK_ECUDA. */
int rk_batch_create(const rk_tableset *ts, const rk_batch_opts *opts, rk_batch **out);
/* Free a batch engine (NULL is ignored) after its capture stream drains; a
 * run on a caller stream must have completed.                               */
void rk_batch_destroy(rk_batch *b);
/* Key field widths, the launch shape in use (after rk_batch_autotune, the
 * one it kept) and the work chunks of the current batch (host only).
 * Errors: RK_EINVAL (b or info NULL).                                       */
int rk_batch_info_get(const rk_batch *b, rk_batch_info *info);

/* Describe the next batch: item i searches d_texts[i][0 .. text_lens[i]) (device
 * memory, any alignment, kept valid until the run completes) with table
 * table_of_item[i].  Host arrays; the descriptors are copied on `stream` and
 * the call returns once they are on the device, so a run of this batch on
 * another stream must have completed.  Errors: RK_EINVAL (limits of
 * rk_batch_opts exceeded, a table index out of range, another current
 * device), RK_ECUDA.                                                        */
int rk_batch_set(rk_batch *b, uint32_t n_items, const uint32_t *table_of_item,
                 const uint8_t *const *d_texts, const uint64_t *text_lens, void *stream);

/* Run the batch: one graph launch (persistent scan of all items, sort,
 * item offsets) on `stream`, asynchronous.  Errors: RK_EINVAL, RK_ECUDA.    */
int rk_batch_run(rk_batch *b, void *stream);

/* Device pointers owned by the batch (valid until rk_batch_destroy): the
 * sorted keys, n_items + 1 item offsets into them (item i's matches are keys
 * [offsets[i], offsets[i+1])), and the header {count, status}.  When count >
 * capacity the keys and offsets are not valid.  Any output pointer may be
 * NULL.  Errors: RK_EINVAL (b NULL).                                        */
int rk_batch_results(const rk_batch *b, const uint64_t **d_keys, const uint64_t **d_item_offsets,
                     const uint64_t **d_info);

/* Copy the results of the last run to host memory and wait: h_info[0..2)
 * (count, status); if the run succeeded and fit, h_item_offsets[0 .. n_items]
 * (n_items of the last rk_batch_set, also in rk_batch_info; NULL allowed) and
 * the first min(count, key_cap) keys (h_keys may be NULL).
 * Errors: RK_EINVAL, RK_ECUDA.                                               */
int rk_batch_read(const rk_batch *b, uint64_t *h_keys, uint64_t key_cap, uint64_t *h_item_offsets,
                  uint64_t *h_info, void *stream);

/* Autotuner (the paper's threads-per-block sweep of Table 1, automated):
 * time up to max_candidates launch shapes (tile size, warps, stages, CTAs
 * per SM, survivor-table placement; 0 = all that fit, else an even spread of
 * them), each `reps` times (0: 3) on the current batch, keep the fastest and
 * re-capture the graph.  Only the scan is timed (the sort's work does not
 * depend on the shape).  *best_ms (may be NULL) gets the best scan time, or
 * -1 when no shape could run (the previous shape is kept).
 * Synchronous; the batch's results are overwritten.
 * Errors: RK_EINVAL (b NULL), RK_ENOMEM, RK_ECUDA.                          */
int rk_batch_autotune(rk_batch *b, uint32_t max_candidates, uint32_t reps, double *best_ms,
                      void *stream);

/* ---- serving ---------------------------------------------------------------
 * A request loop over a resident table set.  Requests (a host text and a
 * table id) are admitted while their texts fit in a device-memory arena of
 * mem_cap bytes, copied to the device, and packed into batched launches on
 * `engines` batch engines; requests arriving while batches run are admitted
 * and copied meanwhile and go into the next free engine.  A lone request on
 * an idle GPU runs as a plain search (rk_search_device with a plain build of
 * its table, made at rk_server_create) and counts as a batch of one.  Each
 * request gets its own sorted match list in the single-text key format
 * RK_KEY(id, x).  The worker thread polls while work is in flight and for
 * 2 ms after, so it keeps one host core busy then.                         */
typedef struct rk_server rk_server;

typedef struct rk_server_opts {
    uint64_t mem_cap;          /* device bytes for admitted texts (the admission cap) */
    uint64_t max_text_len;     /* longest request text, <= mem_cap */
    uint64_t max_batch_bytes;  /* most text bytes per batch (default mem_cap) */
    uint64_t batch_capacity;   /* match keys per batch (default 2^22) */
    uint32_t engines;          /* batches in flight, 1..8 (default 2) */
    uint32_t max_batch_items;  /* requests per batch (default 1024) */
    uint32_t tile_bytes, warps;  /* launch shape of the batch kernel (0 = default) */
} rk_server_opts;

typedef struct rk_request_times {
    double arrive_us, admit_us, launch_us, done_us;  /* since the server started */
} rk_request_times;

typedef struct rk_server_stats {
    uint64_t requests_done, bytes_done, batches, items_batched;
    uint64_t waiting, in_flight, arena_used;
    double now_us;
} rk_server_stats;

/* Start a server (and its worker thread) on the current device.  The table
 * set must outlive it.  Besides the arena it allocates, per engine, a batch
 * engine and a plain search's keys (batch_capacity) and workspace (for
 * max_text_len bytes).  Errors: RK_EINVAL, RK_ENOMEM, RK_ECUDA.             */
int rk_server_create(const rk_tableset *ts, const rk_server_opts *opts, rk_server **out);

/* Finish every submitted request, stop the worker and free everything.     */
void rk_server_destroy(rk_server *s);

/* Submit a request: search h_text[0..n) (host memory, valid and unchanged
 * until the request is taken) with table `table`.  *request_id identifies it.
 * Errors: RK_EINVAL (table, length beyond max_text_len), RK_ENOMEM.         */
int rk_server_submit(rk_server *s, uint32_t table, const uint8_t *h_text, uint64_t n,
                     uint64_t *request_id);

/* Wait up to timeout_ms (< 0: forever) for a request and take its result:
 * *n_keys gets the match count, h_keys[0..n_keys) the sorted keys, *times
 * (may be NULL) its timestamps.  RK_ECAPACITY: key_cap < *n_keys, the result
 * is kept (call again); RK_ETIMEOUT: not finished yet; RK_EINVAL: no such
 * request (never submitted, or already taken).  Other errors (RK_ECUDA: its
 * copy or batch failed): the request failed and is released.                */
int rk_server_take(rk_server *s, uint64_t request_id, int timeout_ms, uint64_t *h_keys,
                   uint64_t key_cap, uint64_t *n_keys, rk_request_times *times);

/* Counters of the server (a consistent snapshot): requests and bytes done,
 * batches launched and requests they held, requests waiting for admission,
 * requests admitted and not finished (in_flight: copying, queued for an
 * engine or running), arena bytes in use, and the server's clock.
 * Errors: RK_EINVAL (s or stats NULL).                                      */
int rk_server_stats_get(rk_server *s, rk_server_stats *stats);

/* ---- search without allocation ------------------------------------------
 * No counterpart in the paper: a convenience for callers that cannot allocate.
 *
 * Some callers cannot call cudaMalloc or pass a workspace: applications whose
 * own allocator has reserved all device memory (a foreign cudaMalloc fails),
 * or latency-bound loops that cannot afford cudaMalloc/cudaFree, which may
 * synchronise the device.  rk_search_device_noalloc does what
 * rk_search_device does, but the sort's scratch space is a fixed array inside
 * the library (RK_NOALLOC_MAX_KEYS keys: RK_NOALLOC_SCRATCH_BYTES bytes, about
 * 16.8 MB), reserved on every GPU where the library's device code is loaded
 * and held until the process exits.  It allocates nothing.
 *   - capacity > RK_NOALLOC_MAX_KEYS is rejected with RK_EINVAL;
 *   - the first call on each device looks up the array's device address
 *     (once per device, with that device current) and keeps it: make that
 *     first call before any stream capture; a device reset (cudaDeviceReset,
 *     or anything else that destroys the device's primary context) unloads
 *     the array, and the kept address must not be used after it, so do not
 *     call this entry point in a process after resetting a device it ran on;
 *   - every call on a device shares the one array, and it keeps the last
 *     call's contents: calls that overlap on the GPU (other streams, other
 *     threads, other tables) race on it and must be serialised by the caller.
 * Other arguments, results and errors as rk_search_device.                  */
#define RK_NOALLOC_MAX_KEYS (1u << 20)
#define RK_NOALLOC_SCRATCH_BYTES 16785920u
int rk_search_device_noalloc(const rk_table *t, const uint8_t *d_text, uint64_t n,
                             uint64_t *d_keys, uint64_t capacity, uint64_t *d_info,
                             void *stream);

#ifdef __cplusplus
}
#endif

#endif /* RK_H */
