"""The search entry point that allocates nothing (rk_search_device_noalloc).

It exists for callers that cannot allocate device memory, for instance when
their own allocator has reserved the whole GPU or when cudaMalloc's possible
device synchronisation is unaffordable; its sort scratch is a fixed array in
the library, shared by every call on a device and keeping the last call's
contents.  Its output must equal the oracle's list and rk_search_device's,
bit for bit, on calls in a row that leave each other different leftovers: a
large output, a small one with a smaller capacity, the large one again, and
one with a tiny capacity.  This file sorts last so a run that stops at the
first failure has run every other test already.
"""

import numpy as np
import pytest

import oracle
from workloads import make_config, random_small

pytestmark = pytest.mark.gpu

from gpu_util import assert_same, keys_to_pairs, require_gpu, search_table, to_device  # noqa: E402
from paper_1810_01051_gb300 import rk  # noqa: E402


def _noalloc(table, d_text, n, capacity):
    import torch
    keys = torch.empty(max(capacity, 1), dtype=torch.int64, device="cuda")
    info = torch.full((2,), -1, dtype=torch.int64, device="cuda")
    rk.rk_search_device_noalloc(table, d_text, n, keys, capacity, info)
    torch.cuda.synchronize()
    count, status = (int(v) for v in info.cpu().tolist())
    return keys, count, status


def test_noalloc_equals_oracle_and_workspace_search_in_a_row():
    require_gpu()
    large = random_small(9, 300000, 30, 1, 12, alphabet=b"abc")      # ~10^5 matches
    small = make_config(1, n=(4 << 20) + 333)                        # Zipf: a few thousand
    tiny = random_small(3, 5000, 3, 3, 5, alphabet=b"ab", plants=2)
    runs = [(large, rk.RK_NOALLOC_MAX_KEYS), (small, 1 << 15), (large, rk.RK_NOALLOC_MAX_KEYS),
            (tiny, 0), (small, rk.RK_NOALLOC_MAX_KEYS)]
    expect = {}
    for w, cap in runs:
        key = id(w)
        if key not in expect:
            expect[key] = oracle.rabin_karp(w.text, w.patterns)
        ei, eo = expect[key]
        table = rk.rk_build(w.patterns)
        try:
            d = to_device(w.text, 3)
            want = max(cap, ei.size) if cap else ei.size  # tiny: exactly the matches
            ref_keys, ref_count, ref_status = search_table(table, d, w.n, max(want, 1))
            assert ref_status == rk.RK_OK and ref_count == ei.size
            assert_same(keys_to_pairs(ref_keys[:ref_count]), (ei, eo), "rk_search_device")
            keys, count, status = _noalloc(table, d, w.n, want)
            assert status == rk.RK_OK and count == ei.size, (count, ei.size)
            assert_same(keys_to_pairs(keys[:count]), (ei, eo), f"noalloc, capacity {want}")
        finally:
            rk.rk_destroy(table)


def test_noalloc_capacity_short_reports_the_count():
    """A capacity below the match count: the count is reported and the call
    succeeds (the list is not sorted then, as with rk_search_device)."""
    require_gpu()
    w = random_small(11, 100000, 10, 2, 4, alphabet=b"ab")
    ei, _ = oracle.rabin_karp(w.text, w.patterns)
    table = rk.rk_build(w.patterns)
    try:
        d = to_device(w.text)
        _, count, status = _noalloc(table, d, w.n, 100)
        assert status == rk.RK_OK and count == ei.size > 100
    finally:
        rk.rk_destroy(table)


def test_noalloc_rejects_capacity_beyond_its_scratch():
    require_gpu()
    import torch
    table = rk.rk_build([b"abc"])
    try:
        d = to_device(np.frombuffer(b"xxabcxx", np.uint8))
        keys = torch.empty(4, dtype=torch.int64, device="cuda")
        info = torch.zeros(2, dtype=torch.int64, device="cuda")
        with pytest.raises(rk.RkError) as e:
            rk.rk_search_device_noalloc(table, d, 7, keys, rk.RK_NOALLOC_MAX_KEYS + 1, info)
        assert e.value.code == rk.RK_EINVAL
    finally:
        rk.rk_destroy(table)
