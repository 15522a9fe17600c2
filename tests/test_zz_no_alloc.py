"""The search entry point that allocates nothing (rk_search_device_noalloc).

It exists for callers that cannot allocate device memory, for instance when
their own allocator has reserved the whole GPU or when cudaMalloc's possible
device synchronisation is unaffordable; its sort scratch is a fixed array in
the library.  Its output must equal rk_search_device's (bit for bit, as every
parity test here), on two calls in a row so the second call starts from the
first call's leftovers in that shared array.  This file sorts last so a run
that stops at the first failure has run every other test already.
"""

import numpy as np
import pytest

from workloads import make_config, random_small

pytestmark = pytest.mark.gpu

from gpu_util import keys_to_pairs, require_gpu, search_table, to_device  # noqa: E402
from paper_1810_01051_gb300 import rk  # noqa: E402


def _noalloc(table, d_text, n, capacity):
    import torch
    keys = torch.empty(max(capacity, 1), dtype=torch.int64, device="cuda")
    info = torch.full((2,), -1, dtype=torch.int64, device="cuda")
    rk.rk_search_device_noalloc(table, d_text, n, keys, capacity, info)
    torch.cuda.synchronize()
    count, status = (int(v) for v in info.cpu().tolist())
    return keys, count, status


def test_noalloc_equals_workspace_search_twice():
    require_gpu()
    cases = [make_config(1, n=(4 << 20) + 333), random_small(9, 200000, 30, 1, 12, alphabet=b"abc")]
    for w in cases:
        table = rk.rk_build(w.patterns)
        try:
            d = to_device(w.text, 3)
            cap = rk.RK_NOALLOC_MAX_KEYS
            ref_keys, ref_count, ref_status = search_table(table, d, w.n, cap)
            assert ref_status == rk.RK_OK and 0 < ref_count <= cap
            ref = keys_to_pairs(ref_keys[:ref_count])
            for _ in range(2):
                keys, count, status = _noalloc(table, d, w.n, cap)
                assert status == rk.RK_OK and count == ref_count
                got = keys_to_pairs(keys[:count])
                assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
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
