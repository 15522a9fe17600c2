"""GPU parity at the full workload sizes (1 GiB Zipf text, 4 GiB signature
set) with default table options, through both scan paths: rk_search_device
with the sort's workspace only (single-kernel scan), and the launch sequence
the bench times (rk_scan_device_ws with the candidate list after the sort's
workspace, verification kernel, rk_sort_device; sampled stage 1 on the
signature set).

The oracle cannot rescan gigabytes in test time, so this checks:
  * both paths give the same list, key for key;
  * the list is strictly ascending (sorted by (id, offset), no duplicates);
  * every reported match is real (bytes compared with numpy);
  * on sampled 256 KiB slices, plus the first and the last (ragged) slice,
    the matches starting in the slice equal the oracle's on that slice.
"""

import numpy as np
import pytest

import oracle
from workloads import make_config

pytestmark = pytest.mark.gpu

from gpu_util import (assert_same, keys_to_pairs, require_gpu, search_table,  # noqa: E402
                      to_device, torch)
from paper_1810_01051_gb300 import rk  # noqa: E402

SLICE = 256 << 10


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


@pytest.mark.parametrize("cfg,n_slices", [(1, 14), (2, 10)])
def test_full_size_sampled(cfg, n_slices):
    w = make_config(cfg)
    n = w.n
    table = rk.rk_build(w.patterns)
    try:
        d = to_device(w.text)
        cap = 1 << 24
        while True:
            keys, count, status = search_table(table, d, n, cap)
            assert status == rk.RK_OK
            if count <= cap:
                break
            cap = count
        ids, offs = keys_to_pairs(keys[:count])
        del keys
        if cfg == 2:
            assert rk.rk_table_info(table)["sample_step"] == 4  # sampled stage 1 runs
        bkeys, bcount = bench_step(table, d, n, max(count, 2))
        del d
    finally:
        rk.rk_destroy(table)
    assert bcount == count, f"deferred path {bcount} matches, single-kernel {count}"
    bids, boffs = keys_to_pairs(bkeys)
    assert np.array_equal(bids, ids) and np.array_equal(boffs, offs), "paths differ"

    packed = (ids.astype(np.uint64) << np.uint64(40)) | offs
    assert np.all(packed[1:] > packed[:-1]), "not strictly ascending"
    assert count > 0

    # every match is real
    bounds = np.searchsorted(ids, np.arange(len(w.patterns) + 1))
    for p, pat in enumerate(w.patterns):
        o = offs[bounds[p]:bounds[p + 1]].astype(np.int64)
        if o.size == 0:
            continue
        L = len(pat)
        assert o.max() + L <= n
        win = w.text[o[:, None] + np.arange(L)[None, :]]
        assert np.array_equal(win, np.broadcast_to(np.frombuffer(pat, np.uint8), win.shape)), p

    # sampled slices against the oracle
    lmax = max(len(p) for p in w.patterns)
    rng = np.random.default_rng(77 + cfg)
    starts = [0, n - SLICE] + [int(s) for s in rng.integers(0, n - SLICE, n_slices)]
    for s in starts:
        sub = w.text[s:min(n, s + SLICE + lmax - 1)]
        ei, eo = oracle.rabin_karp(sub, w.patterns)
        keep = eo < SLICE
        expect = (ei[keep], eo[keep] + np.uint64(s))
        sel = (offs >= s) & (offs < s + SLICE)
        assert_same((ids[sel], offs[sel]), expect, f"config {cfg} slice at {s}")
