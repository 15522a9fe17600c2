"""GPU parity of the batched search (one persistent graph-captured launch over
many texts, each with its own table): every item's sorted (id, offset) list
equals the oracle's on that item alone."""

import numpy as np
import pytest

import oracle
from oracle_pool import oracle_items
from workloads import batched, random_small

pytestmark = pytest.mark.gpu

from gpu_util import require_gpu  # noqa: E402
from paper_1810_01051_gb300 import rk  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def run_batch(texts, tables, table_of, misalign=0, autotune=False, **opts):
    import torch
    ts = rk.rk_tableset_build(tables, filter=opts.pop("filter", rk.RK_FILTER_AUTO),
                              base_log2=opts.pop("base_log2", 0))
    try:
        max_len = max([t.size for t in texts] + [1])
        total = sum(t.size for t in texts)
        cap = opts.pop("capacity", 1 << 20)
        b = rk.rk_batch_create(ts, len(texts), max_len, max(total, 1), cap, **opts)
        try:
            bufs = []
            for t in texts:
                buf = torch.zeros(t.size + misalign + 64, dtype=torch.uint8, device="cuda")
                if t.size:
                    buf[misalign:misalign + t.size].copy_(torch.from_numpy(np.ascontiguousarray(t)))
                bufs.append(buf[misalign:])
            rk.rk_batch_set(b, table_of, bufs, [t.size for t in texts])
            if autotune:
                rk.rk_batch_autotune(b, max_candidates=6, reps=1)
            info = rk.rk_batch_info(b)
            results = []
            for _ in range(2):  # the graph replays; both runs must agree
                rk.rk_batch_run(b)
                torch.cuda.synchronize()
                count, status, keys, offs = rk.rk_batch_read(b, len(texts), cap)
                assert status == rk.RK_OK and count <= cap
                results.append((keys.copy(), offs.copy()))
            assert np.array_equal(results[0][0], results[1][0])
            keys, offs = results[0]
            items, ids, xs = rk.unpack_batch_keys(keys, info["offset_bits"], info["id_bits"])
            return items, ids, xs, offs, info
        finally:
            rk.rk_batch_destroy(b)
    finally:
        rk.rk_tableset_destroy(ts)


def check_items(texts, tables, table_of, items, ids, xs, offs, expect=None):
    """Every item's slice of the batch list equals the oracle's list for that
    item (`expect`: the oracle's lists, computed here when not given)."""
    assert np.all(np.diff(offs.astype(np.int64)) >= 0)
    for i, text in enumerate(texts):
        lo, hi = int(offs[i]), int(offs[i + 1])
        assert np.all(items[lo:hi] == i)
        ei, eo = expect[i] if expect is not None else oracle.rabin_karp(text, tables[table_of[i]])
        assert np.array_equal(ids[lo:hi], ei) and np.array_equal(xs[lo:hi], eo), f"item {i}"


@pytest.mark.parametrize("opts", [dict(), dict(s2_in_smem=1), dict(filter=rk.RK_FILTER_NONE),
                                  dict(tile_bytes=1024, warps=2, stages=3),
                                  dict(base_log2=1, warps=24, tile_bytes=4096)],
                         ids=["default", "s2_smem", "no_filter", "small_tiles", "base2"])
def test_batch_small(opts):
    rng = np.random.default_rng(7)
    texts, tables = [], []
    for i in range(40):
        n = int(rng.choice([0, 1, 5, 100, 3000, 70000]))
        w = random_small(100 + i, n, int(rng.integers(0, 12)), 1 + i % 4, 6 + i % 9,
                         alphabet=[b"ab", b"abc", b"ACGT", None][i % 4], plants=2)
        texts.append(w.text)
        tables.append(w.patterns)
    table_of = list(range(len(texts)))
    # several items share one table, one table appears twice in a row
    table_of[5] = table_of[6] = 3
    out = run_batch(texts, tables, table_of, misalign=3, **opts)
    check_items(texts, tables, table_of, *out[:4])


def test_batch_config_shape_reduced():
    """The batched configuration's shape (20-letter alphabet, 1..256 patterns
    of 4..48 bytes per text, density 1e-5) with smaller texts."""
    bt = batched(n_items=300, max_len=1 << 20)
    out = run_batch(bt.texts, bt.tables, bt.table_of, capacity=1 << 18)
    check_items(bt.texts, bt.tables, bt.table_of, *out[:4])
    assert out[0].size > 0


def test_batch_autotune_keeps_results():
    bt = batched(seed=11, n_items=64, max_len=1 << 18)
    out = run_batch(bt.texts, bt.tables, bt.table_of, autotune=True)
    check_items(bt.texts, bt.tables, bt.table_of, *out[:4])


def test_batch_config_full_max_len():
    """A batch drawn from the batched configuration's recipe at its full text
    sizes (log-uniform 1 KiB..16 MiB; 512 texts, about 0.9 GB, the largest
    above 8 MiB), with the default launch shape and autotuned: every item
    against the oracle, run on every host core."""
    bt = batched(seed=0x5EED0013, n_items=512, max_len=16 << 20)
    assert max(t.size for t in bt.texts) > 8 << 20
    expect = oracle_items([(t, bt.tables[bt.table_of[i]]) for i, t in enumerate(bt.texts)])
    for autotune in (False, True):
        out = run_batch(bt.texts, bt.tables, bt.table_of, capacity=1 << 23, autotune=autotune)
        check_items(bt.texts, bt.tables, bt.table_of, *out[:4], expect=expect)
        assert out[0].size > 0
