"""GPU parity at the full workload sizes with default table options, against
the oracle over the whole text, element by element.

  * 1 GiB Zipf text, 100 patterns: rk_search_device with the sort's
    workspace only (the scan that verifies its survivors itself), the launch
    sequence the bench times (rk_scan_device_ws with the candidate list after
    the sort's workspace, the verification kernel, rk_sort_device) and the
    allocation-free search all give the oracle's list for the whole text
    (the oracle runs in chunks on every host core; tests/oracle_pool.py).
  * 4 GiB signature set, 10,000 patterns: both scan paths over the whole
    text agree key for key, the list is strictly ascending and every match
    real; the last 1 GiB, ragged end included, equals the oracle's list.
"""

import numpy as np
import pytest

from oracle_pool import oracle_matches
from workloads import make_config

pytestmark = pytest.mark.gpu

from gpu_util import (assert_same, keys_to_pairs, require_gpu, search_table,  # noqa: E402
                      to_device, torch)
from paper_1810_01051_gb300 import rk  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def bench_step(table, d_text, n, cap):
    """The bench's step: deferred scan into a workspace placed after the
    sort's, then the sort; returns (keys on the host, count)."""
    keys = torch.empty(cap, dtype=torch.int64, device="cuda")
    info = torch.full((2,), -1, dtype=torch.int64, device="cuda")
    sort_b = rk.rk_workspace_bytes(table, cap)
    scan_b = rk.rk_scan_workspace_bytes(table, n)
    assert rk.rk_scan_launches(table, n, scan_b) == 2  # tile scan + verification
    ws = torch.empty(sort_b + scan_b, dtype=torch.uint8, device="cuda")
    rk.rk_scan_device_ws(table, d_text, n, keys, cap, info, ws[sort_b:], scan_b)
    rk.rk_sort_device(table, n, keys, cap, info, ws, sort_b)
    torch.cuda.synchronize()
    count, status = (int(v) for v in info.cpu().tolist())
    assert status == rk.RK_OK, rk.strerror(status)
    assert count <= cap, (count, cap)
    return keys[:count].cpu(), count


def single_kernel(table, d_text, n):
    cap = 1 << 24
    while True:
        keys, count, status = search_table(table, d_text, n, cap)
        assert status == rk.RK_OK, rk.strerror(status)
        if count <= cap:
            return keys_to_pairs(keys[:count]), count
        cap = count


def noalloc(table, d_text, n, cap):
    keys = torch.empty(cap, dtype=torch.int64, device="cuda")
    info = torch.full((2,), -1, dtype=torch.int64, device="cuda")
    rk.rk_search_device_noalloc(table, d_text, n, keys, cap, info)
    torch.cuda.synchronize()
    count, status = (int(v) for v in info.cpu().tolist())
    assert status == rk.RK_OK, rk.strerror(status)
    assert count <= cap
    return keys_to_pairs(keys[:count])


def assert_real_and_ascending(w, ids, offs):
    packed = (ids.astype(np.uint64) << np.uint64(40)) | offs
    assert np.all(packed[1:] > packed[:-1]), "not strictly ascending"
    bounds = np.searchsorted(ids, np.arange(len(w.patterns) + 1))
    for p, pat in enumerate(w.patterns):
        o = offs[bounds[p]:bounds[p + 1]].astype(np.int64)
        if o.size == 0:
            continue
        L = len(pat)
        assert o.max() + L <= w.n
        win = w.text[o[:, None] + np.arange(L)[None, :]]
        assert np.array_equal(win, np.broadcast_to(np.frombuffer(pat, np.uint8), win.shape)), p


def test_zipf_1gib_whole_text():
    w = make_config(1)
    n = w.n
    expect = oracle_matches(w.text, w.patterns)
    table = rk.rk_build(w.patterns)
    try:
        assert rk.rk_table_info(table)["role_step"] == 2
        d = to_device(w.text)
        got, count = single_kernel(table, d, n)
        assert_same(got, expect, "single-kernel scan")
        bkeys, _ = bench_step(table, d, n, max(count, 2))
        assert_same(keys_to_pairs(bkeys), expect, "the bench's deferred scan")
        assert count <= rk.RK_NOALLOC_MAX_KEYS
        assert_same(noalloc(table, d, n, rk.RK_NOALLOC_MAX_KEYS), expect, "allocation-free search")
        del d
    finally:
        rk.rk_destroy(table)


def test_signature_set_4gib():
    w = make_config(2)
    n = w.n
    start = n - (1 << 30)
    table = rk.rk_build(w.patterns)
    try:
        d = to_device(w.text)
        (ids, offs), count = single_kernel(table, d, n)
        bkeys, bcount = bench_step(table, d, n, max(count, 2))
        del d
    finally:
        rk.rk_destroy(table)
    assert bcount == count, f"deferred path {bcount} matches, single-kernel {count}"
    bids, boffs = keys_to_pairs(bkeys)
    del bkeys
    assert np.array_equal(bids, ids) and np.array_equal(boffs, offs), "paths differ"
    assert count > 0
    assert_real_and_ascending(w, ids, offs)
    # the last 1 GiB against the oracle, the text's ragged end included
    expect = oracle_matches(w.text, w.patterns, start=start)
    keep = offs >= start
    assert_same((ids[keep], offs[keep]), expect, "signature set, last 1 GiB")
