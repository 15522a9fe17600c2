#!/usr/bin/env python3
"""Benchmark of the plain single-text multi-pattern search.

Workload: 1 GiB text of English-like Zipf letters with spaces, 100 patterns of
lengths 4..32 from the same process, each planted at density 1e-6 per byte
(seeded, synthetic; the paper's DNA files are not available).  One step is one
pass of the whole hot path over the resident text: the scan (staging, hashing,
probing, verification, emission) and the sort into (pattern id, offset) order.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  `value` is text GB/s (1e9 bytes/s) with the
text resident in HBM; `e2e` repeats the measurement through the host-buffer
call (host->device copy of the text and device->host copy of the sorted list
inside the timed region).  Under torchrun each rank searches its own copy of
the workload (independent problems, weak scaling).
"""

from __future__ import annotations

import argparse
import hashlib
import json
import multiprocessing as mp
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "text GB/s scanned (plain single-text multi-pattern search, sorted match list)"
UNIT = "GB/s"
WORKLOAD = "zipf_text_1GiB_100_patterns_len4-32_density1e-6"
# the sources the scan kernel is compiled from (the profile records their hash)
SCAN_SRCS = [os.path.join(ROOT, "paper_1810_01051_gb300", "csrc", f)
             for f in ("rk_scan.cu", "rk_scan_kernel.cuh", "rk_scan_rf.cuh", "rk_scan_k_role.cu",
                       "rk_scan_body.cuh", "rk_layout.cuh", "rk_internal.cuh", "rk_verify.cu",
                       "rk_sortws.cuh", "rk_table.cu")]
PROFILE = os.path.join(ROOT, "profiles", "rk_scan_zipf_1GiB.md")
PROFILE_SIG = os.path.join(ROOT, "profiles", "rk_scan_signature_4GiB.md")
CPU_SAMPLE_PER_CORE = 8 << 20   # bytes per core for the oracle baseline
SIG_CPU_SAMPLE_PER_CORE = 2 << 20  # the same on the signature set
SLICE_HALO_NOTE = "each slice carries (longest pattern - 1) extra bytes"


# ---------------------------------------------------------------- helpers

def env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def config_dict(n, k):
    return {"workload": WORKLOAD, "text_bytes": n, "patterns": k, "pattern_len": "4..32",
            "alphabet": "a-z Zipf(s=1) + space p=1/6", "plant_density": 1e-6,
            "l2": "text (1 GiB) larger than the 129 MB L2; no flush needed"}


def _oracle_slice(args):
    text_bytes, patterns = args
    import oracle  # noqa: WPS433  (worker process)
    t0 = time.perf_counter()
    ids, _ = oracle.rabin_karp(np.frombuffer(text_bytes, dtype=np.uint8), patterns)
    return time.perf_counter() - t0, int(ids.size)


def cpu_slices(text, lmax, per_core, cores, seed=11):
    rng = np.random.default_rng(seed)
    n = text.size
    starts = rng.integers(0, n - per_core - lmax, cores)
    return [text[s:s + per_core + lmax - 1].tobytes() for s in starts]


def time_oracle(pool, slices, patterns):
    t0 = time.perf_counter()
    pool.map(_oracle_slice, [(s, patterns) for s in slices])
    return time.perf_counter() - t0


def hbm_peak():
    """(GB/s, source): the measured copy bandwidth of the GB300s, else
    the fallback figure of one earlier measurement."""
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(peaks["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def scan_sources_sha256():
    """SHA-256 of the scan kernel's sources, concatenated in SCAN_SRCS order."""
    h = hashlib.sha256()
    for f in SCAN_SRCS:
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def read_profile(path=None):
    """Figures of a committed ncu summary (default: the Zipf scan's), if it
    was taken on the current scan kernel sources (else None): DRAM bytes per
    full launch and the tile scan's integer-pipe fractions."""
    try:
        txt = open(path or PROFILE).read()
    except OSError:
        return None
    m_src = re.search(r"scan_sources_sha256:\s*([0-9a-f]{64})", txt)
    if not m_src or m_src.group(1) != scan_sources_sha256():
        return None
    out = {}
    for key in ("dram_bytes_per_full_launch", "tile_scan_alu_pipe_frac",
                "tile_scan_fmaheavy_pipe_frac", "tile_scan_issue_active_frac",
                "tile_scan_warp_inst_per_byte"):
        m = re.search(key + r":\s*([0-9.eE+]+)", txt)
        out[key] = float(m.group(1)) if m else None
    return out


class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", gpu_id, f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sms, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            p = [x.strip() for x in line.split(",")]
            if len(p) < 8:
                continue
            try:
                sms.append(float(p[0]))
                mx = float(p[1])
            except ValueError:
                continue
            for nm, v in zip(names, p[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sms:
            return None
        return {"sm_mhz": statistics.median(sms), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sms)}


# ---------------------------------------------------------------- scan step

class StepBuffers:
    """Output and workspace for one table and text, sized from one probe
    search: the sort's scratch first, the deferred scan's candidate list
    after it."""

    def __init__(self, torch, rk, table, d_text, n, dev, st, cap=1 << 22):
        self.scan_b = rk.rk_scan_workspace_bytes(table, n)
        self.info = torch.zeros(2, dtype=torch.int64, device=dev)
        while True:
            self.keys = torch.empty(cap, dtype=torch.int64, device=dev)
            self.wsb = rk.rk_workspace_bytes(table, cap)
            self.ws = torch.empty(self.wsb + self.scan_b, dtype=torch.uint8, device=dev)
            rk.rk_search_device(table, d_text, n, self.keys, cap, self.info, self.ws,
                                self.wsb + self.scan_b, st)
            st.synchronize()
            m, status = (int(v) for v in self.info.cpu().tolist())
            if status != rk.RK_OK:
                raise RuntimeError(f"search failed: {rk.strerror(status)}")
            if m <= cap:
                break
            cap = m + 1024
        self.cap, self.m = cap, m
        self.sws = self.ws[self.wsb:]
        self.scan_kernels = rk.rk_scan_launches(table, n, self.scan_b)
        self.sort_kernels = rk.rk_sort_launches(table, n, cap)

    def candidates(self, torch):
        """Candidate windows the last deferred tile scan listed."""
        return int(self.sws[:8].view(torch.int64)[0].item()) if self.scan_kernels == 2 else 0


def scan_sort(rk, table, d_text, n, b, st, ev=None):
    """One step: tile scan (+ verification) and sort; `ev` = four events
    recorded before the tile scan, between it and the verification kernel,
    before the sort and after it."""
    if ev:
        ev[0].record(st)
        rk.rk_scan_device_ws_split(table, d_text, n, b.keys, b.cap, b.info, b.sws, b.scan_b, st,
                                   ev[1])
        ev[2].record(st)
    else:
        rk.rk_scan_device_ws(table, d_text, n, b.keys, b.cap, b.info, b.sws, b.scan_b, st)
    rk.rk_sort_device(table, n, b.keys, b.cap, b.info, b.ws, b.wsb, st)
    if ev:
        ev[3].record(st)


def new_events(torch, k):
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(k)]
    return evs


def create_events(evs, st):
    """Record every event once so that each exists before its handle is passed
    to the library."""
    for e in evs:
        e[1].record(st)


def kernel_times(evs):
    """Mean milliseconds of (tile scan, verification, sort) over the steps."""
    tile = statistics.mean(e[0].elapsed_time(e[1]) for e in evs)
    ver = statistics.mean(e[1].elapsed_time(e[2]) for e in evs)
    srt = statistics.mean(e[2].elapsed_time(e[3]) for e in evs)
    return tile, ver, srt


def per_kernel_roofline(n, m, cands, scan_kernels, sort_kernels, tile_kernel, tile_ms, verify_ms,
                        sort_ms, peak):
    """Each kernel of the step against the HBM peak with its own algorithmic
    bytes: the tile scan reads the text once and writes 16 bytes per listed
    candidate (8 per match when it verifies itself); the verification kernel
    reads the list and writes 8 bytes per match; the sort reads and writes
    each 8-byte key once."""
    def row(kind, ms, nbytes, rule):
        gbps = nbytes / ms / 1e6 if ms > 0 else None
        return {"kernel": kind, "ms": ms, "algorithmic_bytes": nbytes, "achieved_gbps": gbps,
                "frac": gbps / peak if gbps else None, "bytes_rule": rule}
    out = {}
    if scan_kernels == 2:
        out["tile_scan"] = row(tile_kernel, tile_ms, n + 16 * cands,
                               "text once + 16 B per listed candidate")
        out["verify"] = row("rk_verify_kernel", verify_ms, 16 * cands + 8 * m,
                            "16 B per candidate read + 8 B per match written")
    else:
        out["tile_scan"] = row(tile_kernel, tile_ms + verify_ms, n + 8 * m,
                               "text once + 8 B per match")
    sort_name = "rk_sort_fused_kernel" if sort_kernels == 1 else "rk_sort_hist/pass kernels"
    out["sort"] = row(sort_name, sort_ms, 16 * m, "8 B per key read + 8 B written")
    out["sort"]["launches"] = sort_kernels
    return out


def tile_kernel_name(info_t):
    return "rk_scan_rf_kernel" if info_t.get("role_step", 0) in (2, 4) else "rk_scan_tiles_kernel"


# ---------------------------------------------------------------- replicas

def max_over_ranks(values, device="cpu"):
    """Each value's maximum over all ranks (every rank passes its own
    measurements); unchanged in a single process."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(v) for v in values]
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def job_gbps(world, bytes_per_rank, steps, total_ms):
    """Whole-job GB/s of `world` replicas: every rank's bytes over the
    slowest rank's time."""
    return world * bytes_per_rank * steps / (total_ms / 1e3) / 1e9


# ---------------------------------------------------------------- reference arm

def run_reference(args, rank, world):
    if rank != 0:
        return 0
    from oracle import build as oracle_build
    from workloads import make_config
    oracle_build.build()
    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        w = make_config(1)
        lmax = max(len(p) for p in w.patterns)
        # calibrate one core, then size each step to keep the run within minutes
        cal = cpu_slices(w.text, lmax, 256 << 10, 1, seed=3)
        t_cal = time_oracle(pool, cal, w.patterns)
        rate = (256 << 10) / max(t_cal, 1e-6)
        budget = min(10.0, 150.0 / max(1, args.steps + args.warmup))
        per_core = int(min(16 << 20, max(64 << 10, rate * budget)))
        for i in range(args.warmup):
            time_oracle(pool, cpu_slices(w.text, lmax, per_core, cores, seed=100 + i), w.patterns)
        times = []
        for i in range(args.steps):
            times.append(time_oracle(pool, cpu_slices(w.text, lmax, per_core, cores, seed=200 + i),
                                     w.patterns))
    total = sum(times)
    value = cores * per_core * args.steps / total / 1e9
    sample = (f"{cores} slices of {per_core} bytes per step (one per core) at random offsets of "
              f"the 1 GiB text; {SLICE_HALO_NOTE}")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic", "config": config_dict(w.n, len(w.patterns)),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "build": "gcc " + " ".join(oracle_build.CFLAGS), "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- batched and served

def measure_batched(torch, rk, dev, max_len, reps=5, tune_candidates=12):
    """Batched workload (4096 texts, log-uniform lengths up to max_len, 20
    letters, 1..256 patterns of 4..48 bytes per text): one autotuned graph
    replay for all texts against one plain launch (scan + sort) per text."""
    from workloads import batched
    bt = batched(n_items=4096, max_len=max_len)
    n_items, total = len(bt.texts), bt.total_bytes
    offs, at = [], 0
    for t in bt.texts:
        offs.append(at)
        at += (t.size + 255) // 256 * 256
    host = torch.empty(at + 256, dtype=torch.uint8, pin_memory=True)
    hv = host.numpy()
    for t, o in zip(bt.texts, offs):
        hv[o:o + t.size] = t
    d_all = host.to(dev)
    ptrs = [d_all.data_ptr() + o for o in offs]
    lens = [t.size for t in bt.texts]
    st = torch.cuda.Stream(dev)
    ts = rk.rk_tableset_build(bt.tables)
    cap = 1 << 24
    b = rk.rk_batch_create(ts, n_items, max(lens), total, cap)
    try:
        rk.rk_batch_set(b, bt.table_of, ptrs, lens, st)
        tuned_ms = rk.rk_batch_autotune(b, max_candidates=tune_candidates, reps=2, stream=st)
        info = rk.rk_batch_info(b)
        rk.rk_batch_run(b, st)
        st.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(reps):
            rk.rk_batch_run(b, st)
        e1.record(st)
        st.synchronize()
        batch_ms = e0.elapsed_time(e1) / reps
        count, status, _, _ = rk.rk_batch_read(b, n_items, 0, st)
    finally:
        rk.rk_batch_destroy(b)
        rk.rk_tableset_destroy(ts)
    # plain per-request launches: one table and one search (scan + sort) per text
    tabs = [rk.rk_build(p) for p in bt.tables]
    try:
        pcap = 1 << 20
        keys = torch.empty(pcap, dtype=torch.int64, device=dev)
        infos = torch.zeros(n_items, 2, dtype=torch.int64, device=dev)
        wsb = rk.rk_workspace_bytes(tabs[0], pcap)
        ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
        for i in range(min(8, n_items)):  # warm-up
            rk.rk_search_device(tabs[i], ptrs[i], lens[i], keys, pcap, infos[i], ws, wsb, st)
        st.synchronize()
        marks = [torch.cuda.Event(enable_timing=True) for _ in range(n_items + 1)]
        e0.record(st)
        marks[0].record(st)
        for i in range(n_items):
            rk.rk_search_device(tabs[i], ptrs[i], lens[i], keys, pcap, infos[i], ws, wsb, st)
            marks[i + 1].record(st)
        e1.record(st)
        st.synchronize()
        plain_ms = e0.elapsed_time(e1)
        item_ms = [marks[i].elapsed_time(marks[i + 1]) for i in range(n_items)]
        # completion time of each item when all arrive at once and the plain
        # launches run one after another in submission order
        done_ms = [marks[0].elapsed_time(marks[i + 1]) for i in range(n_items)]
        plain_count = int(infos[:, 0].sum().item())
    finally:
        for t in tabs:
            rk.rk_destroy(t)
    del d_all
    return {
        "workload": f"4096 texts, log-uniform 1 KiB..{max_len >> 20} MiB, 20 letters, "
                    "1..256 patterns of 4..48 bytes each, density 1e-5",
        "text_bytes": total, "matches": count, "status": status,
        "matches_equal_per_request": count == plain_count,
        "batched_gbps": total / (batch_ms / 1e3) / 1e9, "batched_ms": batch_ms,
        "per_request_gbps": total / (plain_ms / 1e3) / 1e9, "per_request_ms": plain_ms,
        "speedup": plain_ms / batch_ms, "autotuned_scan_ms": tuned_ms,
        "latency_ms": {
            "batched_every_item": batch_ms,
            "per_request_launch_p50": float(np.percentile(item_ms, 50)),
            "per_request_launch_p99": float(np.percentile(item_ms, 99)),
            "per_request_completion_p50": float(np.percentile(done_ms, 50)),
            "per_request_completion_p99": float(np.percentile(done_ms, 99)),
            "note": "all texts submitted at once: a batched item completes with the batch; "
                    "a plain launch's completion includes the launches queued before it"},
        "tuned": {k: info[k] for k in ("warps", "tile_bytes", "stages", "ctas_per_sm",
                                       "s2_in_smem")},
    }


def measure_serving(torch, rk, dev, n_req=200, loads=(0.5, 1.0, 2.0, 4.0, 8.0), pool_size=48):
    """Serving workload (64 resident tables of 1..1024 patterns of 4..64 bytes;
    requests of log-uniform 4 KiB..64 MiB uniform bytes, Poisson arrivals):
    p50/p99 latency and GB/s at offered loads relative to the plain
    per-request call's throughput, for the server and for plain calls."""
    import random
    from workloads import serving_tables, serving_texts
    tables = serving_tables()
    pool = serving_texts(0x5EED0005, pool_size, tables)
    pinned = []
    for tid, text in pool:
        h = torch.empty(text.size, dtype=torch.uint8, pin_memory=True)
        h.numpy()[:] = text
        pinned.append((tid, h))
    mean_bytes = sum(h.numel() for _, h in pinned) / len(pinned)
    tabs = [rk.rk_build(t) for t in tables]
    hkeys = torch.empty(1 << 20, dtype=torch.int64, pin_memory=True)

    def plain(tid, h):
        rc, cnt = rk.rk_search(tabs[tid], h, h.numel(), hkeys, hkeys.numel())
        return rc

    try:
        for tid, h in pinned[:4]:
            plain(tid, h)
        t0 = time.perf_counter()
        for tid, h in pinned:
            plain(tid, h)
        plain_gbps = sum(h.numel() for _, h in pinned) / (time.perf_counter() - t0) / 1e9
        ts = rk.rk_tableset_build(tables)
        free, _ = torch.cuda.mem_get_info(dev)
        cap = int(min(64 << 30, free // 4))
        srv = rk.rk_server_create(ts, mem_cap=cap, max_text_len=64 << 20,
                                  batch_capacity=1 << 23, engines=2, max_batch_items=256)
        rng = random.Random(7)
        levels = []
        try:
            for tid, h in pinned[:16]:  # warm-up: engines, events, arena
                rk.rk_server_take(srv, rk.rk_server_submit(srv, tid, h, h.numel()),
                                  timeout_ms=120000, key_cap=1 << 22)
            for load in loads:
                rate = load * plain_gbps * 1e9 / mean_bytes  # requests per second
                arrivals, t = [], 0.0
                for _ in range(n_req):
                    t += rng.expovariate(rate)
                    arrivals.append(t)
                picks = [rng.randrange(len(pinned)) for _ in range(n_req)]
                # served: submit at the arrival times, then collect
                start = time.perf_counter()
                ids = []
                for at, i in zip(arrivals, picks):
                    while time.perf_counter() - start < at:
                        pass
                    tid, h = pinned[i]
                    ids.append(rk.rk_server_submit(srv, tid, h, h.numel()))
                lat, first, last, failed = [], None, 0.0, 0
                for rid in ids:
                    rc, _, tm = rk.rk_server_take(srv, rid, timeout_ms=120000, key_cap=1 << 22)
                    failed += rc != rk.RK_OK
                    lat.append(tm["done_us"] - tm["arrive_us"])
                    first = tm["arrive_us"] if first is None else min(first, tm["arrive_us"])
                    last = max(last, tm["done_us"])
                nbytes = sum(pinned[i][1].numel() for i in picks)
                # plain per-request calls, one at a time in arrival order
                start = time.perf_counter()
                plat, plain_failed = [], 0
                for at, i in zip(arrivals, picks):
                    while time.perf_counter() - start < at:
                        pass
                    tid, h = pinned[i]
                    plain_failed += plain(tid, h) != rk.RK_OK
                    plat.append((time.perf_counter() - start - at) * 1e6)
                plain_span = time.perf_counter() - start - arrivals[0]
                levels.append({
                    "offered_load": load, "offered_gbps": load * plain_gbps,
                    "served_gbps": nbytes / ((last - first) / 1e6) / 1e9,
                    "served_p50_ms": float(np.percentile(lat, 50)) / 1e3,
                    "served_p99_ms": float(np.percentile(lat, 99)) / 1e3,
                    "plain_gbps": nbytes / plain_span / 1e9,
                    "plain_p50_ms": float(np.percentile(plat, 50)) / 1e3,
                    "plain_p99_ms": float(np.percentile(plat, 99)) / 1e3,
                    "failed": failed, "plain_failed": plain_failed,
                })
            stats = rk.rk_server_stats(srv)
        finally:
            rk.rk_server_destroy(srv)
            rk.rk_tableset_destroy(ts)
    finally:
        for t in tabs:
            rk.rk_destroy(t)
    return {
        "workload": "64 resident tables (1..1024 patterns, 4..64 bytes), requests log-uniform "
                    "4 KiB..64 MiB uniform bytes, Poisson arrivals, host texts in pinned memory",
        "requests_per_level": n_req, "mean_request_bytes": mean_bytes,
        "plain_closed_loop_gbps": plain_gbps, "admission_cap_bytes": cap,
        "batches": stats["batches"], "items_batched": stats["items_batched"],
        "levels": levels,
    }


def measure_paper_kernel(torch, rk, dev, reps=5):
    """The paper's workloads on this GPU: its own kernel (one thread per
    offset, O(m) shift-add hash) against the tiled scan, for one pattern on
    DNA-like text: 320 MB with m = 7 over the block sizes of Table 1, and
    Table 3's pattern lengths on 2 MB."""
    from workloads import dna_single
    st = torch.cuda.Stream(dev)

    def timed(fn):
        fn()
        st.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(reps):
            fn()
        e1.record(st)
        st.synchronize()
        return e0.elapsed_time(e1) / reps

    def ours(table, d, n):
        cap = 1 << 16
        keys = torch.empty(cap, dtype=torch.int64, device=dev)
        info = torch.zeros(2, dtype=torch.int64, device=dev)
        wsb = rk.rk_workspace_bytes(table, cap)
        ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
        return lambda: rk.rk_search_device(table, d, n, keys, cap, info, ws, wsb, st)

    out = {"table1_dna_320MB_m7": {}, "table3_dna_2MB": {}}
    w = dna_single(seed=0x5EED0101, n=320_000_000, k=1, m=7, plants=100)
    d = torch.from_numpy(w.text).to(dev)
    res = torch.empty(w.n, dtype=torch.uint8, device=dev)
    for tpb in (32, 64, 128, 256, 512, 1024):
        ms = timed(lambda: rk.rk_paper_search_device(d, w.n, w.patterns[0], res, tpb, st))
        out["table1_dna_320MB_m7"][f"paper_kernel_tpb{tpb}_ms"] = ms
    t = rk.rk_build(w.patterns)
    out["table1_dna_320MB_m7"]["tiled_scan_ms"] = timed(ours(t, d, w.n))
    rk.rk_destroy(t)
    del d, res
    for m in (25, 50, 100, 200, 800):
        w = dna_single(seed=0x5EED0200 + m, n=2_000_000, k=1, m=m, plants=20)
        d = torch.from_numpy(w.text).to(dev)
        res = torch.empty(w.n, dtype=torch.uint8, device=dev)
        pk = timed(lambda: rk.rk_paper_search_device(d, w.n, w.patterns[0], res, 1024, st))
        t = rk.rk_build(w.patterns)
        ok = timed(ours(t, d, w.n))
        rk.rk_destroy(t)
        out["table3_dna_2MB"][f"m{m}"] = {"paper_kernel_ms": pk, "tiled_scan_ms": ok}
    out["note"] = ("times on this GB300; the paper's Table 1 reports 847.1 ms (1024 threads per "
                   "block, GeForce 920) and Table 3 7.5..201.2 ms for m = 25..800")
    return out


def measure_signature_set(torch, rk, dev, peak, peak_src, steps=10, warmup=3, pool=None,
                          cores=1, n=None):
    """The 4 GiB signature set (uniform bytes, 10,000 patterns of 8..64
    bytes, 1,000 plants each): the same step as the headline line (tile
    scan, verification, sort over the resident text), each kernel timed with
    CUDA events, with its own roofline and, given a process pool, the oracle
    timed on slices of the same text."""
    from workloads import make_config
    w = make_config(2, n=n) if n else make_config(2)
    n = w.n
    st = torch.cuda.Stream(dev)
    d = torch.from_numpy(w.text).to(dev)
    table = rk.rk_build(w.patterns)
    try:
        info_t = rk.rk_table_info(table)
        b = StepBuffers(torch, rk, table, d, n, dev, st, cap=1 << 24)
        for _ in range(warmup):
            scan_sort(rk, table, d, n, b, st)
        evs = new_events(torch, steps)
        create_events(evs, st)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for i in range(steps):
            scan_sort(rk, table, d, n, b, st, evs[i])
        e1.record(st)
        st.synchronize()
        step_ms = e0.elapsed_time(e1) / steps
        tile_ms, verify_ms, sort_ms = kernel_times(evs)
        m = int(b.info[0].item())
        cands = b.candidates(torch)
        rows = per_kernel_roofline(n, m, cands, b.scan_kernels, b.sort_kernels,
                                   tile_kernel_name(info_t), tile_ms, verify_ms, sort_ms, peak)
        scan_ms = statistics.mean(e[0].elapsed_time(e[2]) for e in evs)
        launches = b.scan_kernels + b.sort_kernels
        del b
    finally:
        rk.rk_destroy(table)
        del d
    tile = rows["tile_scan"]
    prof = read_profile(PROFILE_SIG) or {}
    out = {
        "workload": "signature_set_4GiB_10000_patterns_len8-64_uniform_bytes",
        "text_bytes": n, "patterns": len(w.patterns), "matches": m, "candidates": cands,
        "value": n / step_ms / 1e6, "unit": UNIT, "ms_per_step": step_ms, "steps": steps,
        "warmup": warmup, "scan_ms": scan_ms, "gpu_launches_per_step": launches,
        "table": {kk: info_t[kk] for kk in ("filter", "filter_log2_bits", "role_step",
                                             "role_filter_log2_bits", "warps", "tile_bytes",
                                             "stages", "sample_step", "sample_filter_log2_bits")},
        "roofline": {"bound": "hbm", "achieved": tile["achieved_gbps"], "peak": peak,
                     "unit": "GB/s", "frac": tile["frac"],
                     "traffic": prof.get("dram_bytes_per_full_launch"),
                     "kernel": tile["kernel"], "peak_source": f"{peak_src} hbm_gbs",
                     "algorithmic_bytes_per_launch": tile["algorithmic_bytes"],
                     "bytes_rule": tile["bytes_rule"],
                     "scan_step_frac": (n + 8 * m) / scan_ms / 1e6 / peak,
                     "per_kernel": rows,
                     "integer_pipes": None if prof.get("tile_scan_alu_pipe_frac") is None else {
                         "alu_pipe_frac": prof["tile_scan_alu_pipe_frac"],
                         "fmaheavy_pipe_frac": prof["tile_scan_fmaheavy_pipe_frac"],
                         "issue_active_frac": prof["tile_scan_issue_active_frac"],
                         "warp_instructions_per_byte": prof.get("tile_scan_warp_inst_per_byte"),
                         "source": os.path.relpath(PROFILE_SIG, ROOT)}},
        "l2": "text (4 GiB) larger than the 129 MB L2; no flush needed",
    }
    if pool is not None:
        per_core = SIG_CPU_SAMPLE_PER_CORE
        lmax = max(len(p) for p in w.patterns)
        slices = cpu_slices(w.text, lmax, per_core, cores, seed=21)
        wall = time_oracle(pool, slices, w.patterns)
        out["cpu_baseline"] = {"value": cores * per_core / wall / 1e9, "unit": UNIT,
                               "cores": cores, "kind": "oracle",
                               "sample": f"{cores} slices of {per_core} bytes (one per core) at "
                                         f"random offsets of the 4 GiB text, all 10,000 "
                                         f"patterns; {SLICE_HALO_NOTE}"}
    del w
    return out


def measure_plain_configs(torch, rk, dev, hbm_gbs, reps=5):
    """The small plain configuration (1 MiB DNA text, 8 patterns of 16
    bytes): the same step, timed with CUDA events; GB/s = text bytes / step
    time (the text fits in L2, so its HBM fraction means little)."""
    from workloads import make_config
    st = torch.cuda.Stream(dev)
    out = {}
    w = make_config(0)
    d = torch.from_numpy(w.text).to(dev)
    table = rk.rk_build(w.patterns)
    try:
        b = StepBuffers(torch, rk, table, d, w.n, dev, st, cap=1 << 16)
        for _ in range(3):
            scan_sort(rk, table, d, w.n, b, st)
        evs = new_events(torch, reps)
        create_events(evs, st)
        for i in range(reps):
            scan_sort(rk, table, d, w.n, b, st, evs[i])
        st.synchronize()
        tile_ms, verify_ms, sort_ms = kernel_times(evs)
        step = statistics.mean(e[0].elapsed_time(e[3]) for e in evs)
        out["dna_1MiB_8x16"] = {"text_bytes": w.n, "patterns": len(w.patterns),
                                "matches": int(b.info[0].item()), "search_ms": step,
                                "gbps": w.n / step / 1e6, "tile_scan_ms": tile_ms,
                                "verify_ms": verify_ms, "sort_ms": sort_ms,
                                "launches": b.scan_kernels + b.sort_kernels}
        del b
    finally:
        rk.rk_destroy(table)
    return out


# ---------------------------------------------------------------- our arm


def run_ours(args, rank, world, local_rank):
    from oracle import build as oracle_build
    from workloads import make_config

    want_cpu = rank == 0 and world == 1 and not args.no_cpu_baseline
    pool = None
    cores = os.cpu_count() or 1
    if want_cpu:
        oracle_build.build()
        pool = mp.get_context("spawn").Pool(cores)  # before the first GPU call

    import torch
    import torch.distributed as dist
    from paper_1810_01051_gb300 import build_lib, rk

    build_lib.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    w = make_config(1, n=args.text_mib << 20) if args.text_mib else make_config(1)
    n, k = w.n, len(w.patterns)
    t0 = time.perf_counter()
    table = rk.rk_build(w.patterns)
    build_ms = (time.perf_counter() - t0) * 1e3
    info_t = rk.rk_table_info(table)

    d_text = torch.from_numpy(w.text).to(dev)
    st = torch.cuda.Stream(dev)
    bufs = StepBuffers(torch, rk, table, d_text, n, dev, st)
    cap = bufs.cap

    for _ in range(args.warmup):
        scan_sort(rk, table, d_text, n, bufs, st)
    torch.cuda.synchronize()

    gpu_id = None
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        gpu_id = str(local_rank)
    sampler = ClockSampler(gpu_id)
    time.sleep(0.3)

    evs = new_events(torch, args.steps)
    create_events(evs, st)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev_start = torch.cuda.Event(enable_timing=True)
    ev_end = torch.cuda.Event(enable_timing=True)
    ev_start.record(st)
    for i in range(args.steps):
        scan_sort(rk, table, d_text, n, bufs, st, evs[i])
    ev_end.record(st)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    total_ms = ev_start.elapsed_time(ev_end)
    tile_ms, verify_ms, sort_ms = kernel_times(evs)
    scan_steps = [e[0].elapsed_time(e[2]) for e in evs]
    m = int(bufs.info[0].item())
    cands = bufs.candidates(torch)
    scan_kernels, sort_kernels = bufs.scan_kernels, bufs.sort_kernels

    # end to end through the host-buffer call: pinned text in, sorted list out
    e2e_s = float("nan")
    if not args.no_e2e:
        h_text = torch.empty(n, dtype=torch.uint8, pin_memory=True)
        h_text.numpy()[:] = w.text
        h_keys = torch.empty(cap, dtype=torch.int64, pin_memory=True)
        e2e_steps = max(1, min(args.steps, args.e2e_steps))
        rk.rk_search(table, h_text, n, h_keys, cap)  # warm the cached device buffers
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            rc, cnt = rk.rk_search(table, h_text, n, h_keys, cap)
            assert rc == rk.RK_OK and cnt == m
        e2e_s = (time.perf_counter() - t0) / e2e_steps
    clocks = sampler.stop()
    del d_text, bufs

    peak, peak_src = hbm_peak()
    extra = {}
    # the extra workloads are single-GPU measurements: at N > 1 the other ranks
    # would wait for them inside the max-over-ranks collective
    if rank == 0 and world == 1 and not args.no_extras:
        for name, fn in (("signature_set", lambda: measure_signature_set(
                              torch, rk, dev, peak, peak_src, pool=pool, cores=cores)),
                         ("batched", lambda: measure_batched(torch, rk, dev, 16 << 20)),
                         ("served", lambda: measure_serving(torch, rk, dev)),
                         ("paper_kernel", lambda: measure_paper_kernel(torch, rk, dev)),
                         ("plain_configs",
                          lambda: measure_plain_configs(torch, rk, dev, peak))):
            try:
                extra[name] = fn()
            except Exception as exc:  # a failed extra must not lose the main line
                extra[name] = {"error": f"{type(exc).__name__}: {exc}"}
            torch.cuda.empty_cache()

    total_ms, e2e_s = max_over_ranks([total_ms, e2e_s], dev)

    rk.rk_destroy(table)
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0

    step_ms = total_ms / args.steps
    value = job_gbps(world, n, args.steps, total_ms)
    rows = per_kernel_roofline(n, m, cands, scan_kernels, sort_kernels, tile_kernel_name(info_t),
                               tile_ms, verify_ms, sort_ms, peak)
    tile = rows["tile_scan"]
    prof = read_profile() or {}
    traffic = prof.get("dram_bytes_per_full_launch")
    pipes = None
    if prof.get("tile_scan_alu_pipe_frac") is not None:
        pipes = {"kernel": tile["kernel"],
                 "alu_pipe_frac": prof["tile_scan_alu_pipe_frac"],
                 "fmaheavy_pipe_frac": prof["tile_scan_fmaheavy_pipe_frac"],
                 "issue_active_frac": prof["tile_scan_issue_active_frac"],
                 "warp_instructions_per_byte": prof.get("tile_scan_warp_inst_per_byte"),
                 "source": f"ncu --set full of the tile scan kernel ({os.path.relpath(PROFILE, ROOT)})"}
    scan_step_ms = statistics.mean(scan_steps)

    cpu = None
    if pool is not None:
        lmax = max(len(p) for p in w.patterns)
        slices = cpu_slices(w.text, lmax, CPU_SAMPLE_PER_CORE, cores)
        wall = time_oracle(pool, slices, w.patterns)
        pool.close()
        one_s, _ = _oracle_slice((slices[0], w.patterns))  # one core, in this process
        cpu = {"value": cores * CPU_SAMPLE_PER_CORE / wall / 1e9, "unit": UNIT, "cores": cores,
               "value_one_core": CPU_SAMPLE_PER_CORE / one_s / 1e9,
               "kind": "oracle", "build": "gcc " + " ".join(oracle_build.CFLAGS),
               "sample": f"{cores} slices of {CPU_SAMPLE_PER_CORE} bytes (one per core) at random "
                         f"offsets of the 1 GiB text, all 100 patterns; {SLICE_HALO_NOTE}"}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": config_dict(n, k), "replicas": world,
        "matches": m, "candidates": cands,
        "scan_ms": scan_step_ms, "tile_scan_ms": tile_ms, "verify_ms": verify_ms,
        "sort_ms": sort_ms,
        "scan_ms_p10_p90": [float(np.percentile(scan_steps, 10)),
                            float(np.percentile(scan_steps, 90))],
        "hbm_frac_whole_step": (n + 8 * m) / (step_ms / 1e3) / 1e9 / peak,
        "build_ms": build_ms,
        "table": {kk: info_t[kk] for kk in ("filter", "filter_log2_bits", "role_step",
                                             "role_filter_log2_bits", "survivor_warps", "warps",
                                             "tile_bytes", "stages", "ctas_per_sm", "smem_bytes",
                                             "s2_smem_bytes", "sm_count")},
        "roofline": {"bound": "hbm", "achieved": tile["achieved_gbps"], "peak": peak,
                     "unit": "GB/s", "frac": tile["frac"], "traffic": traffic,
                     "kernel": tile["kernel"],
                     "peak_source": f"{peak_src} hbm_gbs",
                     "algorithmic_bytes_per_launch": tile["algorithmic_bytes"],
                     "bytes_rule": tile["bytes_rule"],
                     "scan_step_frac": (n + 8 * m) / scan_step_ms / 1e6 / peak,
                     "per_kernel": rows,
                     "integer_pipes": pipes},
        "e2e": None if args.no_e2e else {
            "value": job_gbps(world, n, 1, e2e_s * 1e3), "unit": UNIT, "h2d_bytes_per_step": n,
            "d2h_bytes_per_step": 16 + 8 * m},
        "gpu_launches": args.steps * (scan_kernels + sort_kernels),
        "clocks": clocks,
        "cpu_baseline": cpu,
    }
    line.update(extra)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer measurement")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched and served comparisons")
    ap.add_argument("--text-mib", type=int, default=0,
                    help="profiling: the plain or signature workload on a text of this many "
                         "MiB (same generator and density) instead of the full one; the "
                         "batched workload with texts of at most this many MiB")
    ap.add_argument("--workload", choices=["plain", "batched", "signature", "served"],
                    default="plain",
                    help="batched: the 4096-text batch (up to 16 MiB per text) alone; "
                         "signature: the 4 GiB signature set alone; served: the serving "
                         "loop's load sweep alone")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    world = env_int("WORLD_SIZE", 1)
    rank = env_int("RANK", 0)
    local_rank = env_int("LOCAL_RANK", 0)
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload == "batched":
        return run_batched_full(args)
    if args.workload == "signature":
        return run_signature_full(args)
    if args.workload == "served":
        return run_served_full(args)
    return run_ours(args, rank, world, local_rank)


def run_batched_full(args):
    import torch
    from paper_1810_01051_gb300 import build_lib, rk
    build_lib.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    r = measure_batched(torch, rk, dev, (args.text_mib or 16) << 20,
                        reps=max(3, min(args.steps, 20)))
    line = {"metric": METRIC + " [batched workload]", "value": r["batched_gbps"], "unit": UNIT,
            "n_gpus": 1, "steps": max(3, min(args.steps, 20)), "warmup": args.warmup,
            "ms_per_step": r["batched_ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": r["workload"], "text_bytes": r["text_bytes"]},
            "batched": r}
    print(json.dumps(line), flush=True)
    return 0


def run_served_full(args):
    """The serving workload's load sweep as its own line (one GPU): `value`
    is the served GB/s at the highest offered load."""
    import torch
    from paper_1810_01051_gb300 import build_lib, rk
    build_lib.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    r = measure_serving(torch, rk, dev)
    top = r["levels"][-1]
    line = {"metric": METRIC + " [served workload]", "value": top["served_gbps"], "unit": UNIT,
            "n_gpus": 1, "steps": r["requests_per_level"], "warmup": args.warmup,
            "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": r["workload"]}, "served": r}
    print(json.dumps(line), flush=True)
    return 0


def run_signature_full(args):
    """The 4 GiB signature set as its own line (one GPU)."""
    import torch
    from paper_1810_01051_gb300 import build_lib, rk
    build_lib.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    peak, src = hbm_peak()
    steps = max(1, min(args.steps, 50))
    r = measure_signature_set(torch, rk, dev, peak, src, steps=steps, warmup=args.warmup,
                              n=(args.text_mib << 20) or None)
    line = {"metric": METRIC + " [signature set]", "value": r["value"], "unit": UNIT,
            "n_gpus": 1, "steps": steps, "warmup": args.warmup, "ms_per_step": r["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic",
            "config": {"workload": r["workload"], "text_bytes": r["text_bytes"],
                       "patterns": r["patterns"], "l2": r["l2"]},
            "roofline": r["roofline"], "gpu_launches": steps * r["gpu_launches_per_step"],
            "signature_set": r}
    print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
