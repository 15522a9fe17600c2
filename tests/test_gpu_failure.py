"""Failure detection without faulting the GPU: a scan whose pipeline copies
never arrive (a flag nothing sets) must give up after its wait limit, record
RK_ETIMEOUT in the device header, and leave the context usable."""

import time

import pytest

import oracle
from workloads import make_config

pytestmark = pytest.mark.gpu

from gpu_util import assert_same, gpu_search, require_gpu, to_device  # noqa: E402
from paper_1810_01051_gb300 import rk  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def test_withheld_copies_time_out_and_context_survives():
    import torch
    w = make_config(1, n=1 << 20)
    table = rk.rk_build(w.patterns)
    try:
        d = to_device(w.text)
        keys = torch.empty(1 << 16, dtype=torch.int64, device="cuda")
        info = torch.zeros(2, dtype=torch.int64, device="cuda")
        t0 = time.perf_counter()
        rk.rk_debug_scan_withheld(table, d, w.n, keys, keys.numel(), info, 200)
        torch.cuda.synchronize()
        elapsed = time.perf_counter() - t0
        assert int(info[1]) == rk.RK_ETIMEOUT
        assert int(info[0]) == 0
        assert elapsed < 5.0
        # the sort skips a result whose status is not RK_OK
        wsb = rk.rk_workspace_bytes(table, keys.numel())
        ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
        rk.rk_sort_device(table, w.n, keys, keys.numel(), info, ws, wsb)
        torch.cuda.synchronize()
    finally:
        rk.rk_destroy(table)
    # the same context still searches correctly
    assert_same(gpu_search(w.patterns, w.text), oracle.rabin_karp(w.text, w.patterns), "after")
