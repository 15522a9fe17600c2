"""Helpers for the GPU tests: run the library on numpy inputs."""

from __future__ import annotations

from typing import Sequence, Tuple

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1810_01051_gb300 import build_lib, rk  # noqa: E402


def require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build_lib.build()
    rk.load()


def to_device(text: np.ndarray, misalign: int = 0) -> "torch.Tensor":
    """Copy text to the GPU starting `misalign` bytes past a 256-byte boundary."""
    n = int(text.size)
    buf = torch.zeros(n + misalign + 64, dtype=torch.uint8, device="cuda")
    view = buf[misalign:misalign + n]
    if n:
        view.copy_(torch.from_numpy(np.array(text, dtype=np.uint8, copy=True)))
    return view


def keys_to_pairs(keys: "torch.Tensor") -> Tuple[np.ndarray, np.ndarray]:
    k = keys.cpu().numpy().view(np.uint64)
    return rk.unpack_keys(k)


def search_table(table: int, d_text: "torch.Tensor", n: int, capacity: int,
                 stream=None) -> Tuple["torch.Tensor", int, int]:
    keys = torch.empty(max(capacity, 1), dtype=torch.int64, device="cuda")
    info = torch.full((2,), -1, dtype=torch.int64, device="cuda")
    wsb = rk.rk_workspace_bytes(table, capacity)
    ws = torch.empty(max(wsb, 16), dtype=torch.uint8, device="cuda")
    rk.rk_search_device(table, d_text if n else 0, n, keys, capacity, info, ws, wsb, stream)
    torch.cuda.synchronize()
    count, status = (int(v) for v in info.cpu().tolist())
    return keys, count, status


def gpu_search(patterns: Sequence[bytes], text: np.ndarray, misalign: int = 0,
               capacity: int = 0, **opts) -> Tuple[np.ndarray, np.ndarray]:
    """Sorted (ids, offsets) from rk_search_device; grows the output until it fits."""
    table = rk.rk_build(list(patterns), **opts)
    try:
        d = to_device(text, misalign)
        cap = capacity or max(1024, int(text.size) // 8)
        while True:
            keys, count, status = search_table(table, d, int(text.size), cap)
            assert status == rk.RK_OK, rk.strerror(status)
            if count <= cap:
                return keys_to_pairs(keys[:count])
            cap = count
    finally:
        rk.rk_destroy(table)


def assert_same(got, expect, what=""):
    gi, go = got
    ei, eo = expect
    assert gi.size == ei.size, f"{what}: {gi.size} matches, oracle {ei.size}"
    assert np.array_equal(gi.astype(np.uint64), ei.astype(np.uint64)), what
    assert np.array_equal(go.astype(np.uint64), eo.astype(np.uint64)), what


def deferred_search(patterns: Sequence[bytes], text: np.ndarray, misalign: int = 0,
                    via_search: bool = True, **opts) -> Tuple[np.ndarray, np.ndarray]:
    """Sorted (ids, offsets) through the deferred scan (rk_search_device given
    room for the candidate list, or rk_scan_device_ws + rk_sort_device);
    grows the output until it fits."""
    table = rk.rk_build(list(patterns), **opts)
    try:
        n = int(text.size)
        d = to_device(text, misalign)
        cap = max(1024, n // 8)
        while True:
            keys = torch.empty(cap, dtype=torch.int64, device="cuda")
            info = torch.full((2,), -1, dtype=torch.int64, device="cuda")
            sort_b = rk.rk_workspace_bytes(table, cap)
            scan_b = rk.rk_scan_workspace_bytes(table, n)
            ws = torch.empty(sort_b + scan_b, dtype=torch.uint8, device="cuda")
            if via_search:
                rk.rk_search_device(table, d if n else 0, n, keys, cap, info, ws, sort_b + scan_b)
            else:
                sws = torch.empty(scan_b, dtype=torch.uint8, device="cuda")
                rk.rk_scan_device_ws(table, d if n else 0, n, keys, cap, info, sws, scan_b)
                rk.rk_sort_device(table, n, keys, cap, info, ws, sort_b)
            torch.cuda.synchronize()
            count, status = (int(v) for v in info.cpu().tolist())
            assert status == rk.RK_OK, rk.strerror(status)
            if count <= cap:
                return keys_to_pairs(keys[:count])
            cap = count
    finally:
        rk.rk_destroy(table)
