// Public entry points of rk.h: device-buffer scan / sort / search, the
// host-buffer search with copy/scan overlap, and the per-window hash kernel.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "rk_internal.cuh"
#include "rk_sortws.cuh"

using namespace rk;

namespace {

bool aligned(const void *p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

int scan_args_ok(const rk_table *t, const uint8_t *d_text, uint64_t n, const uint64_t *d_keys,
                 uint64_t capacity, const uint64_t *d_info) {
    if (!t || !d_info || !aligned(d_info, 8)) return RK_EINVAL;
    if (n > RK_MAX_TEXT_LEN || (n && !d_text)) return RK_EINVAL;
    if (capacity && (!d_keys || !aligned(d_keys, 8))) return RK_EINVAL;
    if (capacity >= (1ull << 32)) return RK_EINVAL;
    return check_device(t);
}

// ---- A2 on its own: Rabin hash of every window by a tiled rolling update --
constexpr uint32_t kRollRun = 64;  // windows per thread

__global__ void rk_window_hash_kernel(const uint8_t *text, uint64_t n, uint32_t L, uint32_t k,
                                   uint64_t *out) {
    const uint64_t nw = n - L + 1;
    const uint32_t s_out = (uint32_t)((uint64_t)k * (L - 1) % 61);  // B^(L-1) = 2^s_out
    for (uint64_t run = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; run * kRollRun < nw;
         run += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t x0 = run * kRollRun;
        const uint64_t x1 = min(nw, x0 + kRollRun);
        uint64_t h = 0;
        for (uint32_t i = 0; i < L; ++i) {
            h = rotl61(h, k) + text[x0 + i];
            if (h >= kP61) h -= kP61;
        }
        out[x0] = h;
        for (uint64_t x = x0; x + 1 < x1; ++x) {
            // h(x+1) = (h(x) - T[x] * B^(L-1)) * B + T[x+L]
            uint64_t outgoing = s_out ? rotl61((uint64_t)text[x], s_out) : (uint64_t)text[x];
            h = submod61(h, outgoing);
            h = rotl61(h, k) + text[x + L];
            if (h >= kP61) h -= kP61;
            out[x + 1] = h;
        }
    }
}

int ensure(void **p, uint64_t *cap, uint64_t need) {
    if (*cap >= need && *p) return RK_OK;
    if (*p) cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    if (cudaMalloc(p, need) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return RK_ENOMEM;
    }
    *cap = need;
    return RK_OK;
}

}  // namespace

extern "C" uint64_t rk_workspace_bytes(const rk_table *t, uint64_t capacity) {
    if (!t) return 0;
    return sort_workspace_bytes(capacity);
}

extern "C" uint64_t rk_scan_workspace_bytes(const rk_table *t, uint64_t n) {
    if (!t || n > RK_MAX_TEXT_LEN) return 0;
    return scan_ws_layout(n).total;
}

namespace {

// The candidate list inside a deferred scan's workspace (null: too small, or
// a table that cannot defer).
bool cand_list(const rk_table *t, uint64_t n, void *ws, uint64_t ws_bytes, CandList *cl) {
    const ScanWsLayout L = scan_ws_layout(n);
    if (!can_defer(t) || !ws || !aligned(ws, 16) || ws_bytes < L.total) return false;
    uint8_t *b = reinterpret_cast<uint8_t *>(ws);
    *cl = CandList{reinterpret_cast<ulonglong2 *>(b + L.list_off), L.cap,
                   reinterpret_cast<unsigned long long *>(b + L.count_off)};
    return true;
}

// Scan with the survivors' hash/probe/verify in a second kernel.
// `mid` (optional) is recorded between the two launches.
int deferred_scan(const rk_table *t, const uint8_t *d_text, uint64_t n, uint64_t *d_keys,
                  uint64_t capacity, uint64_t *d_info, const CandList &cl, cudaStream_t st,
                  cudaEvent_t mid = nullptr) {
    if (cudaMemsetAsync(d_info, 0, 2 * sizeof(uint64_t), st) != cudaSuccess ||
        cudaMemsetAsync(cl.count, 0, sizeof(unsigned long long), st) != cudaSuccess)
        return RK_ECUDA;
    int rc = launch_scan(t, d_text, n, 0, n, d_keys, capacity, d_info, st, &cl);
    if (rc) return rc;
    if (mid && cudaEventRecord(mid, st) != cudaSuccess) return RK_ECUDA;
    return launch_verify(t, d_text, n, cl, d_keys, capacity, d_info, st);
}

}  // namespace

extern "C" int rk_scan_launches(const rk_table *t, uint64_t n, uint64_t workspace_bytes,
                                uint32_t *launches) {
    if (!t || !launches) return RK_EINVAL;
    if (n == 0 || t->dev.n_patterns == 0) {
        *launches = 0;
        return RK_OK;
    }
    *launches = can_defer(t) && n <= RK_MAX_TEXT_LEN && workspace_bytes >= scan_ws_layout(n).total
                    ? 2u
                    : 1u;
    return RK_OK;
}

extern "C" int rk_scan_device_ws(const rk_table *t, const uint8_t *d_text, uint64_t n,
                                 uint64_t *d_keys, uint64_t capacity, uint64_t *d_info,
                                 void *d_workspace, uint64_t workspace_bytes, void *stream) {
    int rc = scan_args_ok(t, d_text, n, d_keys, capacity, d_info);
    if (rc) return rc;
    CandList cl;
    if (!cand_list(t, n, d_workspace, workspace_bytes, &cl))
        return rk_scan_device(t, d_text, n, d_keys, capacity, d_info, stream);
    return deferred_scan(t, d_text, n, d_keys, capacity, d_info, cl,
                         reinterpret_cast<cudaStream_t>(stream));
}

extern "C" int rk_scan_device_ws_split(const rk_table *t, const uint8_t *d_text, uint64_t n,
                                       uint64_t *d_keys, uint64_t capacity, uint64_t *d_info,
                                       void *d_workspace, uint64_t workspace_bytes, void *stream,
                                       void *mid_event) {
    int rc = scan_args_ok(t, d_text, n, d_keys, capacity, d_info);
    if (rc) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaEvent_t mid = reinterpret_cast<cudaEvent_t>(mid_event);
    CandList cl;
    if (cand_list(t, n, d_workspace, workspace_bytes, &cl))
        return deferred_scan(t, d_text, n, d_keys, capacity, d_info, cl, st, mid);
    rc = rk_scan_device(t, d_text, n, d_keys, capacity, d_info, stream);
    if (rc == RK_OK && mid && cudaEventRecord(mid, st) != cudaSuccess) return RK_ECUDA;
    return rc;
}

extern "C" int rk_scan_device(const rk_table *t, const uint8_t *d_text, uint64_t n,
                              uint64_t *d_keys, uint64_t capacity, uint64_t *d_info,
                              void *stream) {
    int rc = scan_args_ok(t, d_text, n, d_keys, capacity, d_info);
    if (rc) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(d_info, 0, 2 * sizeof(uint64_t), st) != cudaSuccess) return RK_ECUDA;
    return launch_scan(t, d_text, n, 0, n, d_keys, capacity, d_info, st);
}

extern "C" int rk_sort_launches(const rk_table *t, uint64_t n, uint64_t capacity,
                                uint32_t *launches) {
    if (!t || !launches) return RK_EINVAL;
    *launches = sort_launches(t, n, capacity);
    return RK_OK;
}

extern "C" int rk_sort_device(const rk_table *t, uint64_t n, uint64_t *d_keys, uint64_t capacity,
                              const uint64_t *d_info, void *d_workspace, uint64_t workspace_bytes,
                              void *stream) {
    if (!t || !d_info || !aligned(d_info, 8) || n > RK_MAX_TEXT_LEN) return RK_EINVAL;
    if (capacity >= (1ull << 32)) return RK_EINVAL;
    if (capacity && (!d_keys || !aligned(d_keys, 8))) return RK_EINVAL;
    if (capacity >= 2 && (!d_workspace || !aligned(d_workspace, 16) ||
                          workspace_bytes < sort_workspace_bytes(capacity)))
        return RK_EINVAL;
    int rc = check_device(t);
    if (rc) return rc;
    return launch_sort(t, n, d_keys, capacity, d_info, d_workspace, workspace_bytes,
                       reinterpret_cast<cudaStream_t>(stream));
}

extern "C" int rk_search_device(const rk_table *t, const uint8_t *d_text, uint64_t n,
                                uint64_t *d_keys, uint64_t capacity, uint64_t *d_info,
                                void *d_workspace, uint64_t workspace_bytes, void *stream) {
    int rc = scan_args_ok(t, d_text, n, d_keys, capacity, d_info);
    if (rc) return rc;
    if (capacity >= 2 && (!d_workspace || !aligned(d_workspace, 16) ||
                          workspace_bytes < sort_workspace_bytes(capacity)))
        return RK_EINVAL;
    // a workspace that also holds a scan workspace after the sort's defers
    // the survivors' verification to a second kernel
    const uint64_t sort_bytes = capacity >= 2 ? sort_workspace_bytes(capacity) : 0;
    CandList cl;
    if (d_workspace && workspace_bytes > sort_bytes &&
        cand_list(t, n, reinterpret_cast<uint8_t *>(d_workspace) + sort_bytes,
                  workspace_bytes - sort_bytes, &cl))
        rc = deferred_scan(t, d_text, n, d_keys, capacity, d_info, cl,
                           reinterpret_cast<cudaStream_t>(stream));
    else
        rc = rk_scan_device(t, d_text, n, d_keys, capacity, d_info, stream);
    if (rc) return rc;
    return launch_sort(t, n, d_keys, capacity, d_info, d_workspace, workspace_bytes,
                       reinterpret_cast<cudaStream_t>(stream));
}

extern "C" int rk_search(const rk_table *tc, const uint8_t *h_text, uint64_t n, uint64_t *h_keys,
                         uint64_t capacity, uint64_t *n_matches) {
    if (!tc || !n_matches || n > RK_MAX_TEXT_LEN || (n && !h_text) || (capacity && !h_keys))
        return RK_EINVAL;
    if (capacity >= (1ull << 32)) return RK_EINVAL;
    int rc = check_device(tc);
    if (rc) return rc;
    rk_table *t = const_cast<rk_table *>(tc);  // only the host-path cache is mutated
    std::lock_guard<std::mutex> lock(t->host_mu);
    *n_matches = 0;

    if (!t->s_copy && cudaStreamCreateWithFlags(&t->s_copy, cudaStreamNonBlocking) != cudaSuccess)
        return RK_ECUDA;
    if (!t->s_comp && cudaStreamCreateWithFlags(&t->s_comp, cudaStreamNonBlocking) != cudaSuccess)
        return RK_ECUDA;
    if ((rc = ensure(reinterpret_cast<void **>(&t->h_text), &t->h_text_cap, std::max<uint64_t>(n, 16))))
        return rc;
    uint64_t kcap = std::max<uint64_t>(capacity, 2);
    uint64_t cap_bytes = t->h_keys_cap;
    if ((rc = ensure(reinterpret_cast<void **>(&t->h_keys), &cap_bytes, kcap * 8))) return rc;
    t->h_keys_cap = cap_bytes;
    uint64_t info_cap = t->h_info ? 16 : 0;
    if ((rc = ensure(reinterpret_cast<void **>(&t->h_info), &info_cap, 16))) return rc;
    // sort workspace, then the deferred scan's candidate list
    const uint64_t sort_bytes = sort_workspace_bytes(kcap);
    const uint64_t scan_bytes = can_defer(t) ? scan_ws_layout(n).total : 0;
    if ((rc = ensure(&t->h_ws, &t->h_ws_cap, sort_bytes + scan_bytes))) return rc;
    CandList cl;
    const bool defer = scan_bytes && cand_list(t, n, reinterpret_cast<uint8_t *>(t->h_ws) + sort_bytes,
                                               scan_bytes, &cl);

    // Copy the text in chunks on one stream while the other scans the windows
    // whose bytes (window + longest pattern - 1) have arrived.
    const uint64_t chunk = 64ull << 20;
    const uint64_t nchunks = n ? (n + chunk - 1) / chunk : 0;
    while (t->events.size() < nchunks) {
        cudaEvent_t e;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return RK_ECUDA;
        t->events.push_back(e);
    }
    cudaStream_t sc = t->s_comp, sx = t->s_copy;
    bool ok = cudaMemsetAsync(t->h_info, 0, 16, sc) == cudaSuccess &&
              (!defer || cudaMemsetAsync(cl.count, 0, 8, sc) == cudaSuccess);
    for (uint64_t c = 0; ok && c < nchunks; ++c) {
        uint64_t b = c * chunk, e = std::min(n, b + chunk);
        ok = cudaMemcpyAsync(t->h_text + b, h_text + b, e - b, cudaMemcpyHostToDevice, sx) ==
                 cudaSuccess &&
             cudaEventRecord(t->events[c], sx) == cudaSuccess;
    }
    const uint64_t reach = t->dev.lmax ? t->dev.lmax - 1 : 0;
    for (uint64_t c = 0; ok && c < nchunks; ++c) {
        uint64_t b = c * chunk, e = std::min(n, b + chunk);
        uint64_t need = std::min(n, e + reach);                  // last byte a window may read
        uint64_t last = need ? (need - 1) / chunk : 0;          // chunk holding it
        ok = cudaStreamWaitEvent(sc, t->events[last], 0) == cudaSuccess;
        if (ok && launch_scan(t, t->h_text, n, b, e, t->h_keys, capacity, t->h_info, sc,
                              defer ? &cl : nullptr) != RK_OK)
            ok = false;
    }
    if (ok && defer &&
        launch_verify(t, t->h_text, n, cl, t->h_keys, capacity, t->h_info, sc) != RK_OK)
        ok = false;
    if (!ok) {
        cudaStreamSynchronize(sx);
        cudaStreamSynchronize(sc);
        return RK_ECUDA;
    }
    if (capacity >= 2 &&
        launch_sort(t, n, t->h_keys, capacity, t->h_info, t->h_ws, t->h_ws_cap, sc) != RK_OK)
        return RK_ECUDA;
    uint64_t info[2] = {0, 0};
    if (cudaMemcpyAsync(info, t->h_info, 16, cudaMemcpyDeviceToHost, sc) != cudaSuccess ||
        cudaStreamSynchronize(sc) != cudaSuccess)
        return RK_ECUDA;
    *n_matches = info[0];
    if (info[1] != RK_OK) return (int)info[1];
    if (info[0] > capacity) return RK_ECAPACITY;
    if (info[0] && (cudaMemcpyAsync(h_keys, t->h_keys, info[0] * 8, cudaMemcpyDeviceToHost, sc) !=
                        cudaSuccess ||
                    cudaStreamSynchronize(sc) != cudaSuccess))
        return RK_ECUDA;
    return RK_OK;
}

extern "C" int rk_window_hashes_device(const uint8_t *d_text, uint64_t n, uint32_t L,
                                       uint32_t base_log2, uint64_t *d_hashes, void *stream) {
    if (L < 1 || L > RK_MAX_PATTERN_LEN || base_log2 < 1 || base_log2 > 60) return RK_EINVAL;
    if (n > RK_MAX_TEXT_LEN) return RK_EINVAL;
    if (L > n) return RK_OK;
    if (!d_text || !d_hashes || !aligned(d_hashes, 8)) return RK_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return RK_ECUDA;
    uint64_t runs = (n - L + 1 + kRollRun - 1) / kRollRun;
    uint64_t blocks = std::min<uint64_t>((runs + 255) / 256, (uint64_t)sms * 8);
    rk_window_hash_kernel<<<(uint32_t)std::max<uint64_t>(blocks, 1), 256, 0,
                         reinterpret_cast<cudaStream_t>(stream)>>>(d_text, n, L, base_log2,
                                                                     d_hashes);
    return cudaGetLastError() == cudaSuccess ? RK_OK : RK_ECUDA;
}

extern "C" int rk_debug_scan_withheld(const rk_table *t, const uint8_t *d_text, uint64_t n,
                                      uint64_t *d_keys, uint64_t capacity, uint64_t *d_info,
                                      uint32_t timeout_ms, void *stream) {
    int rc = scan_args_ok(t, d_text, n, d_keys, capacity, d_info);
    if (rc) return rc;
    if (timeout_ms == 0 || timeout_ms > 10000) return RK_EINVAL;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(d_info, 0, 2 * sizeof(uint64_t), st) != cudaSuccess) return RK_ECUDA;
    return launch_scan_opts(t, d_text, n, 0, n, d_keys, capacity, d_info, st,
                            (uint64_t)timeout_ms * 1000000ull, true);
}

// ---------------------------------------------------------------- match records

namespace {

// Sorted keys -> match records, for the first min(count, capacity) keys
// (count read on the device).
__global__ void rk_keys_to_matches_kernel(const uint64_t *keys, const uint64_t *info,
                                          uint64_t capacity, rk_match *out) {
    const uint64_t m = min((uint64_t)info[0], capacity);
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t k = keys[i];
        out[i] = rk_match{RK_KEY_OFFSET(k), RK_KEY_ID(k), 0u};
    }
}

}  // namespace

extern "C" int rk_build_ptrs(const uint8_t *const *patterns, const uint32_t *lens,
                             uint32_t n_patterns, const rk_build_opts *opts, rk_table **out) {
    if (!out) return RK_EINVAL;
    *out = nullptr;
    if (n_patterns > RK_MAX_PATTERNS) return RK_EINVAL;
    if (n_patterns && (!patterns || !lens)) return RK_EINVAL;
    uint64_t total = 0;
    for (uint32_t i = 0; i < n_patterns; ++i) {
        if (lens[i] < 1 || lens[i] > RK_MAX_PATTERN_LEN || !patterns[i]) return RK_EINVAL;
        total += lens[i];
    }
    std::vector<uint8_t> cat;
    try {
        cat.resize(total ? total : 1);
    } catch (...) {
        return RK_ENOMEM;
    }
    uint64_t at = 0;
    for (uint32_t i = 0; i < n_patterns; ++i) {
        memcpy(cat.data() + at, patterns[i], lens[i]);
        at += lens[i];
    }
    return rk_build(n_patterns ? cat.data() : nullptr, n_patterns ? lens : nullptr, n_patterns,
                    opts, out);
}

extern "C" void rk_free_matches(rk_match *m) { free(m); }

extern "C" int rk_search_matches(const rk_table *t, const uint8_t *h_text, uint64_t n,
                                 rk_match **out, uint64_t *n_out) {
    if (!out || !n_out) return RK_EINVAL;
    *out = nullptr;
    *n_out = 0;
    if (!t || n > RK_MAX_TEXT_LEN || (n && !h_text)) return RK_EINVAL;
    // a first guess at the count; a second search runs when it was short
    uint64_t cap = std::min<uint64_t>(n / 256 + 4096, 1ull << 22);
    std::vector<uint64_t> keys;
    for (;;) {
        try {
            keys.resize(cap);
        } catch (...) {
            return RK_ENOMEM;
        }
        uint64_t m = 0;
        const int rc = rk_search(t, h_text, n, keys.data(), cap, &m);
        if (rc == RK_ECAPACITY && m > cap) {
            if (m >= (1ull << 32)) return RK_ECAPACITY;  // beyond rk_search's output limit
            cap = m;
            continue;
        }
        if (rc) return rc;
        rk_match *r = static_cast<rk_match *>(malloc(std::max<uint64_t>(m, 1) * sizeof(rk_match)));
        if (!r) return RK_ENOMEM;
        for (uint64_t i = 0; i < m; ++i)
            r[i] = rk_match{RK_KEY_OFFSET(keys[i]), RK_KEY_ID(keys[i]), 0u};
        *out = r;
        *n_out = m;
        return RK_OK;
    }
}

extern "C" int rk_search_device_matches(const rk_table *tc, const uint8_t *d_text, uint64_t n,
                                        void *stream, rk_match *d_out, uint64_t capacity,
                                        uint64_t *n_out) {
    if (!n_out) return RK_EINVAL;
    *n_out = 0;
    if (!tc || n > RK_MAX_TEXT_LEN || (n && !d_text) || (capacity && !d_out) ||
        !aligned(d_out, 8) || capacity >= (1ull << 32))
        return RK_EINVAL;
    int rc = check_device(tc);
    if (rc) return rc;
    rk_table *t = const_cast<rk_table *>(tc);  // only the host-path cache is mutated
    std::lock_guard<std::mutex> lock(t->host_mu);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    // key buffer, header and workspace (the sort's, then the candidate list)
    // cached on the table like rk_search's
    const uint64_t kcap = std::max<uint64_t>(capacity, 2);
    uint64_t cap_bytes = t->h_keys_cap;
    if ((rc = ensure(reinterpret_cast<void **>(&t->h_keys), &cap_bytes, kcap * 8))) return rc;
    t->h_keys_cap = cap_bytes;
    uint64_t info_cap = t->h_info ? 16 : 0;
    if ((rc = ensure(reinterpret_cast<void **>(&t->h_info), &info_cap, 16))) return rc;
    const uint64_t sort_bytes = sort_workspace_bytes(kcap);
    const uint64_t scan_bytes = can_defer(t) ? scan_ws_layout(n).total : 0;
    if ((rc = ensure(&t->h_ws, &t->h_ws_cap, sort_bytes + scan_bytes))) return rc;
    rc = rk_search_device(t, d_text, n, t->h_keys, capacity, t->h_info, t->h_ws,
                          sort_bytes + scan_bytes, stream);
    if (rc) return rc;
    if (capacity) {
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return RK_ECUDA;
        const uint64_t blocks = std::min<uint64_t>((capacity + 255) / 256, (uint64_t)sms * 4);
        rk_keys_to_matches_kernel<<<(uint32_t)blocks, 256, 0, st>>>(t->h_keys, t->h_info,
                                                                  capacity, d_out);
        if (cudaGetLastError() != cudaSuccess) return RK_ECUDA;
    }
    uint64_t info[2] = {0, 0};
    if (cudaMemcpyAsync(info, t->h_info, 16, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return RK_ECUDA;
    *n_out = info[0];
    if (info[1] != RK_OK) return (int)info[1];
    return info[0] > capacity ? RK_ECAPACITY : RK_OK;
}

extern "C" int rk_debug_binary_version(int *version) {
    if (!version) return RK_EINVAL;
    cudaFuncAttributes a{};
    if (cudaFuncGetAttributes(&a, rk_keys_to_matches_kernel) != cudaSuccess) {
        cudaGetLastError();
        return RK_ECUDA;
    }
    *version = a.binaryVersion;
    return RK_OK;
}
