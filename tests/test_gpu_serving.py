"""GPU tests of the serving loop: requests admitted by device memory, packed
into batched launches while others run, each result identical to the oracle
and to the same request served alone."""

import numpy as np
import pytest

import oracle
from oracle_pool import oracle_items
from workloads import serving_tables, serving_texts

pytestmark = pytest.mark.gpu

from gpu_util import require_gpu  # noqa: E402
from paper_1810_01051_gb300 import rk  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


@pytest.fixture(scope="module")
def tables():
    return serving_tables(seed=21, n_tables=8, k_max=120, lmin=4, lmax=40)


@pytest.fixture(scope="module")
def tableset(tables):
    ts = rk.rk_tableset_build(tables)
    yield ts
    rk.rk_tableset_destroy(ts)


def serve(ts, reqs, **opts):
    s = rk.rk_server_create(ts, **opts)
    try:
        ids = [rk.rk_server_submit(s, tid, text, text.size) for tid, text in reqs]
        out = []
        for rid in ids:
            rc, keys, times = rk.rk_server_take(s, rid, timeout_ms=60000)
            assert rc == rk.RK_OK, rk.strerror(rc)
            out.append((keys, times))
        stats = rk.rk_server_stats(s)
        return out, stats
    finally:
        rk.rk_server_destroy(s)


def expect(tables, tid, text):
    ids, offs = oracle.rabin_karp(text, tables[tid])
    return (ids.astype(np.uint64) << np.uint64(40)) | offs


def test_mixed_requests_match_oracle_and_alone(tables, tableset):
    reqs = serving_texts(5, 120, tables, min_len=1 << 10, max_len=1 << 20, density=2e-5)
    # a small arena (4 MiB) makes admission wait for memory to be freed
    mixed, stats = serve(tableset, reqs, mem_cap=4 << 20, max_text_len=1 << 20,
                         max_batch_items=32, engines=2)
    assert stats["requests_done"] == len(reqs) and stats["batches"] >= 2
    for (tid, text), (keys, times) in zip(reqs, mixed):
        assert np.array_equal(keys, expect(tables, tid, text))
        assert times["arrive_us"] <= times["admit_us"] <= times["launch_us"] <= times["done_us"]
    # the same requests one at a time give the same lists
    for (tid, text), (keys, _) in list(zip(reqs, mixed))[:12]:
        alone, _ = serve(tableset, [(tid, text)], mem_cap=4 << 20, max_text_len=1 << 20)
        assert np.array_equal(alone[0][0], keys)


def test_overflowing_batches_are_split(tables, tableset):
    reqs = serving_texts(9, 40, tables, min_len=1 << 12, max_len=1 << 16, density=3e-4)
    total = sum(expect(tables, t, x).size for t, x in reqs)
    biggest = max(expect(tables, t, x).size for t, x in reqs)
    cap = max(biggest + 8, total // 6)
    assert cap < total
    out, stats = serve(tableset, reqs, mem_cap=64 << 20, max_text_len=1 << 16,
                       batch_capacity=cap, max_batch_items=64, engines=1)
    for (tid, text), (keys, _) in zip(reqs, out):
        assert np.array_equal(keys, expect(tables, tid, text))


def test_submit_rejects_bad_requests(tableset):
    s = rk.rk_server_create(tableset, mem_cap=1 << 20, max_text_len=1 << 16)
    try:
        big = np.zeros(1 << 17, np.uint8)
        with pytest.raises(rk.RkError):
            rk.rk_server_submit(s, 0, big, big.size)
        with pytest.raises(rk.RkError):
            rk.rk_server_submit(s, 999, big[:10], 10)
        empty = np.zeros(0, np.uint8)
        rid = rk.rk_server_submit(s, 1, empty, 0)
        rc, keys, _ = rk.rk_server_take(s, rid, timeout_ms=10000)
        assert rc == rk.RK_OK and keys.size == 0
        # a request already taken, or an id never issued, is refused at once
        # (a bounded wait, so that a regression fails instead of hanging)
        for bad in (rid, rid + 1000):
            rc, _, _ = rk.rk_server_take(s, bad, timeout_ms=2000)
            assert rc == rk.RK_EINVAL
    finally:
        rk.rk_server_destroy(s)


def test_text_of_mem_cap_bytes_is_admitted(tables, tableset):
    """A cap off the 256-byte granule still admits a text of exactly cap
    bytes, and an empty text (a granule of its own), one after the other."""
    cap = (1 << 16) + 100
    reqs = serving_texts(13, 1, tables, min_len=cap, max_len=cap)
    tid, text = reqs[0]
    text = np.resize(text, cap)
    s = rk.rk_server_create(tableset, mem_cap=cap, max_text_len=cap)
    try:
        rid = rk.rk_server_submit(s, tid, text, cap)
        rid0 = rk.rk_server_submit(s, tid, np.zeros(0, np.uint8), 0)
        rc, keys, _ = rk.rk_server_take(s, rid, timeout_ms=20000)
        assert rc == rk.RK_OK, rk.strerror(rc)
        assert np.array_equal(keys, expect(tables, tid, text))
        rc, keys, _ = rk.rk_server_take(s, rid0, timeout_ms=20000)
        assert rc == rk.RK_OK and keys.size == 0
    finally:
        rk.rk_server_destroy(s)


def test_large_requests_match_oracle():
    """Requests at the serving configuration's upper sizes (16..64 MiB of
    uniform bytes) against its 64 resident tables (1..1024 patterns of 4..64
    bytes), admitted under a 192 MiB cap so that some wait for memory: each
    list equals the oracle's, run on every host core."""
    tables = serving_tables()
    reqs = serving_texts(0x5EED0031, 8, tables, min_len=16 << 20, max_len=64 << 20)
    assert max(t.size for _, t in reqs) > 48 << 20
    expect = oracle_items([(text, tables[tid]) for tid, text in reqs])
    ts = rk.rk_tableset_build(tables)
    try:
        out, stats = serve(ts, reqs, mem_cap=192 << 20, max_text_len=64 << 20, engines=2)
    finally:
        rk.rk_tableset_destroy(ts)
    assert stats["requests_done"] == len(reqs)
    for (tid, text), (keys, _), (ei, eo) in zip(reqs, out, expect):
        want = (ei.astype(np.uint64) << np.uint64(40)) | eo
        assert np.array_equal(keys, want), (tid, text.size, keys.size, want.size)
