"""The record-list calls of the C ABI against the oracle: a table built from
one pointer per pattern (rk_build_ptrs) equals one built from the
concatenated bytes; rk_search_matches (host text, library-allocated list)
and rk_search_device_matches (device text, caller's record buffer, host
count) give the oracle's (pattern id, offset) list, with RK_ECAPACITY and
the count when the buffer is short; the kernels report sm_103a."""

import numpy as np
import pytest

import oracle
from workloads import make_config, random_small

pytestmark = pytest.mark.gpu

from gpu_util import assert_same, gpu_search, require_gpu, to_device, torch  # noqa: E402
from paper_1810_01051_gb300 import rk  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def test_binary_version_is_sm103():
    assert rk.rk_debug_binary_version() == 103


@pytest.mark.parametrize("case", ["zipf", "tiny-alphabet", "empty-text"])
def test_record_lists_equal_oracle(case):
    if case == "zipf":
        w = make_config(1, n=(8 << 20) + 5)
    elif case == "tiny-alphabet":
        w = random_small(21, 70000, 25, 1, 9, alphabet=b"abc")
    else:
        w = random_small(22, 0, 5, 2, 4)
    expect = oracle.rabin_karp(w.text, w.patterns)
    table = rk.rk_build_ptrs(w.patterns)
    try:
        # the pointer-array table gives the concatenated table's list
        assert_same(gpu_search(w.patterns, w.text), expect, "concatenated build")
        recs = rk.rk_search_matches(table, w.text, w.n)
        assert (recs["reserved"] == 0).all()
        assert_same((recs["pattern_id"], recs["offset"]), expect, "rk_search_matches")

        d = to_device(w.text, 5)
        m = int(expect[0].size)
        # a short buffer: RK_ECAPACITY and the count
        if m > 1:
            short = torch.empty((m // 2) * 2, dtype=torch.int64, device="cuda")
            rc, cnt = rk.rk_search_device_matches(table, d, w.n, short, m // 2)
            assert rc == rk.RK_ECAPACITY and cnt == m
        out = torch.empty(max(m, 1) * 2, dtype=torch.int64, device="cuda")
        rc, cnt = rk.rk_search_device_matches(table, d, w.n, out, m)
        assert rc == rk.RK_OK and cnt == m
        got = out.cpu().numpy().view(np.uint8)[: m * 16].view(rk.MATCH_DTYPE)
        assert_same((got["pattern_id"], got["offset"]), expect, "rk_search_device_matches")
    finally:
        rk.rk_destroy(table)
