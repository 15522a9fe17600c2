"""GPU parity at the full workload sizes (1 GiB Zipf text, 4 GiB signature
set), in the launch configuration the bench times (default table options).

The oracle cannot rescan gigabytes in test time, so this checks:
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

from gpu_util import assert_same, keys_to_pairs, require_gpu, search_table, to_device  # noqa: E402
from paper_1810_01051_gb300 import rk  # noqa: E402

SLICE = 256 << 10


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


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
        del d, keys
    finally:
        rk.rk_destroy(table)

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
