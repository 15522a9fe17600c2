// Serving loop: search requests arrive with host texts and a resident table
// id; a worker thread admits them while their texts fit in a device-memory
// arena (the admission cap), copies the texts on a copy stream, packs
// admitted requests into whichever batch engine is free (each engine: an
// rk_batch with its own stream and captured graph; the engine's stream waits
// on the device for the copies of its requests), and hands each request its
// sorted match list.  New requests are admitted and copied while earlier
// batches run (continuous batching); a finished batch frees its requests'
// memory for the next arrivals.  A lone request on an idle GPU runs as a
// plain search with its table's plain build.  The worker polls while work is
// in flight or recent, else sleeps until a submission or a finished run (a
// host function queued after each run) wakes it.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>

#include <sys/prctl.h>
#include <unordered_map>
#include <unordered_set>

#include "rk_arena.h"
#include "rk_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;
constexpr double kSpinUs = 2000;  // the worker polls for this long after its last activity
using rk::Arena;

struct Request {
    uint64_t id = 0;
    uint32_t table = 0;
    const uint8_t *h_text = nullptr;
    uint64_t n = 0;
    uint64_t arena_off = 0;
    bool on_arena = false;
    cudaEvent_t copied = nullptr;
    double t_arrive = 0, t_admit = 0, t_launch = 0, t_done = 0;
    int status = RK_OK;
    std::vector<uint64_t> keys;  // (id << 40) | x, ascending
};

struct Engine {
    rk_batch *b = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t done = nullptr;
    bool busy = false;
    std::vector<Request *> reqs;
    uint64_t *h_keys = nullptr;     // pinned: the batch's sorted keys
    uint64_t *h_offsets = nullptr;  // pinned: item offsets
    // a lone request run as a plain search (scan + sort) instead of a batch
    bool plain = false;
    uint64_t *d_pkeys = nullptr;    // its sorted keys (batch_capacity of them)
    uint64_t *d_pinfo = nullptr;    // its {count, status}
    uint64_t *h_pinfo = nullptr;    // pinned copy of d_pinfo
    void *d_pws = nullptr;          // its workspace (sort + candidate list)
    uint64_t pws_bytes = 0;
};

}  // namespace

struct rk_server {
    const rk_tableset *ts = nullptr;
    std::vector<rk_table *> plain_tables;  // one per resident table
    rk_server_opts opts{};
    int device = 0;
    uint8_t *arena_mem = nullptr;
    Arena arena;
    std::vector<Engine> engines;
    cudaStream_t copy_stream = nullptr;
    Clock::time_point t0;

    std::mutex mu;
    std::condition_variable cv_done;
    std::deque<Request *> arrived, ready;
    // wake-ups of the worker: submissions, finished batches (from a host
    // function on the engine's stream, which must not take `mu`: the worker
    // holds it across CUDA calls on that stream), shutdown
    std::mutex wake_mu;
    std::condition_variable cv_wake;
    bool wake = false;
    std::unordered_map<uint64_t, Request *> finished;
    std::unordered_set<uint64_t> open_ids;  // submitted and not yet taken
    uint64_t next_id = 1;
    uint32_t batch_limit = 0;  // items per batch after an overflow (0: no limit)
    bool stop = false;
    uint64_t bytes_done = 0, requests_done = 0, batches = 0, items_batched = 0;
    double t_active = 0;  // last time the worker had work in flight or made progress
    std::vector<cudaEvent_t> spare_events;
    std::thread worker;

    double now_us() const {
        return std::chrono::duration<double, std::micro>(Clock::now() - t0).count();
    }

    void kick() {
        {
            std::lock_guard<std::mutex> wl(wake_mu);
            wake = true;
        }
        cv_wake.notify_one();
    }
};

namespace {

cudaEvent_t take_event(rk_server *s) {
    if (!s->spare_events.empty()) {
        cudaEvent_t e = s->spare_events.back();
        s->spare_events.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    return e;
}

void finish(rk_server *s, Request *r, int status) {
    r->status = status;
    r->t_done = s->now_us();
    if (r->on_arena) s->arena.release(r->arena_off);
    r->on_arena = false;
    if (r->copied) s->spare_events.push_back(r->copied);
    r->copied = nullptr;
    s->finished[r->id] = r;
    s->bytes_done += r->n;
    s->requests_done += 1;
}

// Collect a finished engine's results into its requests (mutex held).  A
// batch whose matches overflowed the key capacity goes back to the head of the
// ready queue and later batches take half as many requests; a single request
// that overflows alone fails with RK_ECAPACITY.
void harvest(rk_server *s, Engine &e) {
    uint64_t info[2] = {0, 0};
    const uint32_t n_items = (uint32_t)e.reqs.size();
    rk_batch_info bi{};
    rk_batch_info_get(e.b, &bi);
    const uint64_t *keys = e.h_keys, *offs = e.h_offsets;
    int rc = rk_batch_read(e.b, e.h_keys, s->opts.batch_capacity, e.h_offsets, info, e.st);
    if (rc == RK_OK && info[1] == RK_OK && info[0] > s->opts.batch_capacity && n_items > 1) {
        for (uint32_t i = n_items; i-- > 0;) s->ready.push_front(e.reqs[i]);
        s->batch_limit = std::max<uint32_t>(1, n_items / 2);
        e.reqs.clear();
        e.busy = false;
        return;
    }
    const double t = s->now_us();
    for (uint32_t i = 0; i < n_items; ++i) {
        Request *r = e.reqs[i];
        if (rc != RK_OK || info[1] != RK_OK) {
            finish(s, r, rc != RK_OK ? rc : (int)info[1]);
            continue;
        }
        if (info[0] > s->opts.batch_capacity) {
            finish(s, r, RK_ECAPACITY);
            continue;
        }
        const uint64_t lo = offs[i], hi = offs[i + 1];
        const uint64_t omask = (1ull << bi.offset_bits) - 1;
        const uint64_t imask = (1ull << bi.id_bits) - 1;
        r->keys.resize(hi - lo);
        for (uint64_t j = lo; j < hi; ++j) {
            const uint64_t k = keys[j];
            r->keys[j - lo] =
                (((k >> bi.offset_bits) & imask) << RK_KEY_OFFSET_BITS) | (k & omask);
        }
        finish(s, r, RK_OK);
        r->t_done = t;
    }
    s->batches += 1;
    s->items_batched += n_items;
    e.reqs.clear();
    e.busy = false;
}

void CUDART_CB batch_finished(void *p) { static_cast<rk_server *>(p)->kick(); }

// A lone request as a plain search on the engine's stream: wait for its
// copy, scan + sort with its table's plain build, then the header to the
// host; the keys are read when the run is done (harvest_plain).
int launch_plain(rk_server *s, Engine &e, Request *r) {
    r->t_launch = s->now_us();
    e.reqs.assign(1, r);
    e.plain = true;
    int rc = cudaStreamWaitEvent(e.st, r->copied, 0) == cudaSuccess ? RK_OK : RK_ECUDA;
    if (rc == RK_OK)
        rc = rk_search_device(s->plain_tables[r->table], s->arena_mem + r->arena_off, r->n,
                              e.d_pkeys, s->opts.batch_capacity, e.d_pinfo, e.d_pws,
                              e.pws_bytes, e.st);
    if (rc == RK_OK && cudaMemcpyAsync(e.h_pinfo, e.d_pinfo, 16, cudaMemcpyDeviceToHost, e.st) !=
                           cudaSuccess)
        rc = RK_ECUDA;
    if (rc == RK_OK && cudaEventRecord(e.done, e.st) != cudaSuccess) rc = RK_ECUDA;
    if (rc == RK_OK && cudaLaunchHostFunc(e.st, batch_finished, s) != cudaSuccess) rc = RK_ECUDA;
    if (rc != RK_OK) {
        e.reqs.clear();
        e.plain = false;
    }
    return rc;
}

// Collect a finished plain search (mutex held).
void harvest_plain(rk_server *s, Engine &e) {
    Request *r = e.reqs[0];
    const uint64_t count = e.h_pinfo[0], status = e.h_pinfo[1];
    int rc = (int)status;
    if (rc == RK_OK && count > s->opts.batch_capacity) rc = RK_ECAPACITY;
    if (rc == RK_OK) {
        r->keys.resize(count);
        if (count &&
            (cudaMemcpyAsync(r->keys.data(), e.d_pkeys, 8 * count, cudaMemcpyDeviceToHost, e.st) !=
                 cudaSuccess ||
             cudaStreamSynchronize(e.st) != cudaSuccess)) {
            cudaGetLastError();
            r->keys.clear();
            rc = RK_ECUDA;
        }
    }
    finish(s, r, rc);
    s->batches += 1;
    s->items_batched += 1;
    e.reqs.clear();
    e.plain = false;
    e.busy = false;
}

void loop(rk_server *s) {
    cudaSetDevice(s->device);
    prctl(PR_SET_TIMERSLACK, 1UL, 0UL, 0UL, 0UL);  // timed waits end on time
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        bool progress = false;
        // 1. admit arrivals while their texts fit in the arena
        while (!s->arrived.empty()) {
            Request *r = s->arrived.front();
            uint64_t off = 0;
            if (!s->arena.alloc(r->n, &off)) break;  // wait for memory to free up
            s->arrived.pop_front();
            r->arena_off = off;
            r->on_arena = true;
            r->t_admit = s->now_us();
            r->copied = take_event(s);
            progress = true;
            bool ok = r->copied != nullptr;
            if (ok && r->n)
                ok = cudaMemcpyAsync(s->arena_mem + off, r->h_text, r->n, cudaMemcpyHostToDevice,
                                     s->copy_stream) == cudaSuccess;
            if (ok) ok = cudaEventRecord(r->copied, s->copy_stream) == cudaSuccess;
            if (!ok) {
                // no copy may still write into the arena block being released
                cudaStreamSynchronize(s->copy_stream);
                cudaGetLastError();
                finish(s, r, RK_ECUDA);
                continue;
            }
            // ready at once: the engine that takes it waits for the copy on
            // the device
            s->ready.push_back(r);
        }
        // 2. finished batches hand back results and memory
        for (Engine &e : s->engines) {
            if (!e.busy) continue;
            const cudaError_t q = cudaEventQuery(e.done);
            if (q == cudaErrorNotReady) continue;
            progress = true;
            if (q == cudaSuccess) {
                if (e.plain) harvest_plain(s, e);
                else harvest(s, e);
            } else {
                cudaGetLastError();
                for (Request *r : e.reqs) finish(s, r, RK_ECUDA);
                e.reqs.clear();
                e.plain = false;
                e.busy = false;
            }
        }
        if (progress) s->cv_done.notify_all();
        // 3. pack ready requests into free engines; a lone request on an
        // idle GPU (nothing else admitted or waiting) runs as a plain search
        bool all_idle = true;
        for (const Engine &e : s->engines) all_idle = all_idle && !e.busy;
        for (Engine &e : s->engines) {
            if (e.busy || s->ready.empty()) continue;
            if (all_idle && s->ready.size() == 1 && s->arrived.empty() &&
                s->ready.front()->n > 0) {
                Request *r = s->ready.front();
                s->ready.pop_front();
                const int rc = launch_plain(s, e, r);
                if (rc != RK_OK) {
                    finish(s, r, rc);
                    s->cv_done.notify_all();
                    continue;
                }
                e.busy = true;
                all_idle = false;
                progress = true;
                continue;
            }
            std::vector<uint32_t> tabs;
            std::vector<const uint8_t *> texts;
            std::vector<uint64_t> lens;
            uint64_t bytes = 0;
            const uint32_t limit = s->batch_limit ? s->batch_limit : s->opts.max_batch_items;
            while (!s->ready.empty() && e.reqs.size() < limit &&
                   bytes + s->ready.front()->n <= s->opts.max_batch_bytes) {
                Request *r = s->ready.front();
                s->ready.pop_front();
                bytes += r->n;
                e.reqs.push_back(r);
                tabs.push_back(r->table);
                texts.push_back(s->arena_mem + r->arena_off);
                lens.push_back(r->n);
            }
            if (e.reqs.empty()) continue;
            const double t = s->now_us();
            // the item descriptors first (rk_batch_set waits for its upload),
            // then the stream waits for the texts' copies and runs the batch
            int rc = rk_batch_set(e.b, (uint32_t)e.reqs.size(), tabs.data(), texts.data(),
                                  lens.data(), e.st);
            for (Request *r : e.reqs) {
                r->t_launch = t;
                if (rc == RK_OK && cudaStreamWaitEvent(e.st, r->copied, 0) != cudaSuccess)
                    rc = RK_ECUDA;
            }
            if (rc == RK_OK) rc = rk_batch_run(e.b, e.st);
            if (rc == RK_OK && cudaEventRecord(e.done, e.st) != cudaSuccess) rc = RK_ECUDA;
            if (rc == RK_OK && cudaLaunchHostFunc(e.st, batch_finished, s) != cudaSuccess)
                rc = RK_ECUDA;
            if (rc != RK_OK) {
                for (Request *r : e.reqs) finish(s, r, rc);
                e.reqs.clear();
                s->cv_done.notify_all();
                continue;
            }
            e.busy = true;
            all_idle = false;
            progress = true;
        }
        bool idle = true;
        for (Engine &e : s->engines) idle = idle && !e.busy;
        if (s->stop && s->arrived.empty() && s->ready.empty() && idle) break;
        const double now = s->now_us();
        if (progress || !idle) s->t_active = now;
        if (!progress && now - s->t_active < kSpinUs) {
            // work in flight, or recent: look again at once, letting
            // submissions and takes have the lock in between (a sleeping
            // worker would add two thread wake-ups to every request)
            lk.unlock();
            std::this_thread::yield();
            lk.lock();
        } else if (!progress) {
            // idle: sleep until a submission, a finished batch or shutdown
            // wakes the worker (and look again after 1 ms regardless)
            lk.unlock();
            {
                std::unique_lock<std::mutex> wl(s->wake_mu);
                s->cv_wake.wait_for(wl, std::chrono::milliseconds(1), [s] { return s->wake; });
                s->wake = false;
            }
            lk.lock();
        }
    }
}

}  // namespace

extern "C" int rk_server_create(const rk_tableset *ts, const rk_server_opts *opts,
                                rk_server **out) {
    if (!out) return RK_EINVAL;
    *out = nullptr;
    if (!ts || !opts) return RK_EINVAL;
    rk_server_opts o = *opts;
    if (!o.engines) o.engines = 2;
    if (!o.max_batch_items) o.max_batch_items = 1024;
    if (!o.max_text_len || !o.mem_cap) return RK_EINVAL;
    if (!o.max_batch_bytes) o.max_batch_bytes = o.mem_cap;
    if (!o.batch_capacity) o.batch_capacity = 1 << 22;
    if (o.engines > 8 || o.max_text_len > o.mem_cap) return RK_EINVAL;
    rk_server *s = new (std::nothrow) rk_server();
    if (!s) return RK_ENOMEM;
    s->ts = ts;
    s->opts = o;
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        delete s;
        return RK_ECUDA;
    }
    // whole granules, so that every text up to max_text_len (<= mem_cap)
    // fits in the empty arena
    const uint64_t arena_bytes = Arena::round_up(o.mem_cap);
    if (cudaMalloc(&s->arena_mem, arena_bytes) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return RK_ENOMEM;
    }
    s->arena.reset(arena_bytes);
    int rc = RK_OK;
    if (cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking) != cudaSuccess)
        rc = RK_ECUDA;
    // plain builds of the resident tables, for lone requests; their
    // workspace: the sort's for batch_capacity keys and the candidate list
    // for max_text_len bytes
    const rk_tableset *T = ts;
    s->plain_tables.assign(T->n_tables, nullptr);
    uint64_t pws = 0;
    for (uint32_t i = 0; i < T->n_tables && !rc; ++i) {
        rk_build_opts bo{};
        bo.base_log2 = T->base_log2;
        const uint32_t k = T->npat[i];
        rc = rk_build(k ? T->bytes.data() + T->byte_first[i] : nullptr,
                      k ? T->lens.data() + T->pat_first[i] : nullptr, k, &bo,
                      &s->plain_tables[i]);
        if (!rc)
            pws = std::max(pws, rk_workspace_bytes(s->plain_tables[i], o.batch_capacity) +
                                    rk_scan_workspace_bytes(s->plain_tables[i], o.max_text_len));
    }
    s->engines.resize(o.engines);
    for (Engine &e : s->engines) {
        if (rc) break;
        e.pws_bytes = pws;
        if (cudaMalloc(&e.d_pkeys, 8 * o.batch_capacity) != cudaSuccess ||
            cudaMalloc(&e.d_pinfo, 16) != cudaSuccess ||
            (pws && cudaMalloc(&e.d_pws, pws) != cudaSuccess) ||
            cudaMallocHost(&e.h_pinfo, 16) != cudaSuccess) {
            cudaGetLastError();
            rc = RK_ENOMEM;
            break;
        }
        rk_batch_opts bo{};
        bo.max_items = o.max_batch_items;
        bo.max_text_len = o.max_text_len;
        bo.max_total_bytes = o.max_batch_bytes;
        bo.capacity = o.batch_capacity;
        bo.tile_bytes = o.tile_bytes;
        bo.warps = o.warps;
        rc = rk_batch_create(ts, &bo, &e.b);
        if (!rc && (cudaStreamCreateWithFlags(&e.st, cudaStreamNonBlocking) != cudaSuccess ||
                    cudaEventCreateWithFlags(&e.done, cudaEventDisableTiming) != cudaSuccess))
            rc = RK_ECUDA;
        if (!rc && (cudaMallocHost(&e.h_keys, 8 * o.batch_capacity) != cudaSuccess ||
                    cudaMallocHost(&e.h_offsets, 8ull * (o.max_batch_items + 1)) != cudaSuccess)) {
            cudaGetLastError();
            rc = RK_ENOMEM;
        }
    }
    if (rc) {
        rk_server_destroy(s);
        return rc;
    }
    s->t0 = Clock::now();
    s->worker = std::thread(loop, s);
    *out = s;
    return RK_OK;
}

extern "C" void rk_server_destroy(rk_server *s) {
    if (!s) return;
    if (s->worker.joinable()) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->stop = true;
        }
        s->kick();
        s->worker.join();
    }
    for (Engine &e : s->engines) {
        if (e.st) cudaStreamSynchronize(e.st);
        rk_batch_destroy(e.b);
        if (e.st) cudaStreamDestroy(e.st);
        if (e.done) cudaEventDestroy(e.done);
        if (e.h_keys) cudaFreeHost(e.h_keys);
        if (e.h_offsets) cudaFreeHost(e.h_offsets);
        if (e.h_pinfo) cudaFreeHost(e.h_pinfo);
        cudaFree(e.d_pkeys);
        cudaFree(e.d_pinfo);
        cudaFree(e.d_pws);
    }
    for (rk_table *t : s->plain_tables) rk_destroy(t);
    if (s->copy_stream) {
        cudaStreamSynchronize(s->copy_stream);
        cudaStreamDestroy(s->copy_stream);
    }
    for (auto &kv : s->finished) {
        if (kv.second->copied) cudaEventDestroy(kv.second->copied);
        delete kv.second;
    }
    for (cudaEvent_t e : s->spare_events) cudaEventDestroy(e);
    cudaFree(s->arena_mem);
    delete s;
}

extern "C" int rk_server_submit(rk_server *s, uint32_t table, const uint8_t *h_text, uint64_t n,
                                uint64_t *request_id) {
    if (!s || !request_id || (n && !h_text)) return RK_EINVAL;
    if (table >= s->ts->n_tables || n > s->opts.max_text_len || n > s->opts.max_batch_bytes)
        return RK_EINVAL;
    Request *r = new (std::nothrow) Request();
    if (!r) return RK_ENOMEM;
    r->table = table;
    r->h_text = h_text;
    r->n = n;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) {
            delete r;
            return RK_EINVAL;
        }
        r->id = s->next_id++;
        r->t_arrive = s->now_us();
        s->arrived.push_back(r);
        s->open_ids.insert(r->id);
        *request_id = r->id;
    }
    s->kick();
    return RK_OK;
}

extern "C" int rk_server_take(rk_server *s, uint64_t request_id, int timeout_ms, uint64_t *h_keys,
                              uint64_t key_cap, uint64_t *n_keys, rk_request_times *times) {
    if (!s || !n_keys) return RK_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    if (!s->open_ids.count(request_id)) return RK_EINVAL;  // never submitted, or taken
    auto pred = [&] { return s->finished.count(request_id) != 0; };
    if (timeout_ms < 0) s->cv_done.wait(lk, pred);
    else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred))
        return RK_ETIMEOUT;
    Request *r = s->finished[request_id];
    *n_keys = r->keys.size();
    if (times) {
        times->arrive_us = r->t_arrive;
        times->admit_us = r->t_admit;
        times->launch_us = r->t_launch;
        times->done_us = r->t_done;
    }
    if (r->status != RK_OK) {
        const int st = r->status;
        s->finished.erase(request_id);
        s->open_ids.erase(request_id);
        delete r;
        return st;
    }
    if (r->keys.size() > key_cap) return RK_ECAPACITY;  // kept: call again with a larger buffer
    if (h_keys && !r->keys.empty()) std::copy(r->keys.begin(), r->keys.end(), h_keys);
    s->finished.erase(request_id);
    s->open_ids.erase(request_id);
    delete r;
    return RK_OK;
}

extern "C" int rk_server_stats_get(rk_server *s, rk_server_stats *st) {
    if (!s || !st) return RK_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    rk_server_stats r{};
    r.requests_done = s->requests_done;
    r.bytes_done = s->bytes_done;
    r.batches = s->batches;
    r.items_batched = s->items_batched;
    r.waiting = s->arrived.size();
    r.in_flight = s->ready.size();
    for (const Engine &e : s->engines) r.in_flight += e.reqs.size();
    r.arena_used = s->arena.used();
    r.now_us = s->now_us();
    *st = r;
    return RK_OK;
}
