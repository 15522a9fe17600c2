"""ctypes binding of ``librk.so`` (declared in ``include/rk.h``).

Argument marshalling only: every step of the search runs in the library's
CUDA kernels.  Device buffers may be given as raw integer addresses or as
torch CUDA tensors (PyTorch supplies device memory and streams, nothing
else).  If the library has not been built the import fails loudly; there is
no fallback implementation.
"""

from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence, Tuple

import numpy as np

from . import build_lib

RK_OK, RK_EINVAL, RK_ENOMEM, RK_ECAPACITY, RK_ECUDA, RK_ETIMEOUT = range(6)
RK_MAX_PATTERN_LEN = 4096
RK_MAX_PATTERNS = (1 << 24) - 1
RK_MAX_TEXT_LEN = (1 << 40) - 1
RK_KEY_OFFSET_BITS = 40
RK_FILTER_AUTO, RK_FILTER_REPLICATED, RK_FILTER_FLAT, RK_FILTER_NONE = range(4)
RK_NOALLOC_MAX_KEYS = 1 << 20

#: names of every function include/rk.h declares
EXPORTS = [
    "rk_strerror", "rk_build", "rk_destroy", "rk_table_info_get", "rk_workspace_bytes",
    "rk_scan_device", "rk_sort_device", "rk_search_device", "rk_search",
    "rk_window_hashes_device", "rk_search_device_noalloc",
]


class RkError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {strerror(code)} ({code})")


class BuildOpts(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint32) for n in (
        "base_log2", "filter", "filter_log2_bits", "warps", "tile_bytes", "stages", "ctas_per_sm")]


class TableInfo(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint32) for n in (
        "n_patterns", "min_len", "max_len", "n_lengths", "gram_len", "base_log2", "filter",
        "filter_log2_bits", "filter_smem_bytes", "n_grams", "warps", "tile_bytes", "stages",
        "ctas_per_sm", "halo_bytes", "smem_bytes", "sm_count", "device", "s2_smem_bytes")] + [
        ("device_bytes", ctypes.c_uint64)]


_lib: Optional[ctypes.CDLL] = None


def library_path() -> str:
    return build_lib.LIB


def load() -> ctypes.CDLL:
    """Load librk.so (raises OSError if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = build_lib.LIB
    if not os.path.exists(path):
        raise OSError(f"{path} is missing: build it with __graft_entry__.build() "
                      "(python -m paper_1810_01051_gb300.build_lib)")
    L = ctypes.CDLL(path)
    vp, u64, u32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32
    L.rk_strerror.restype = ctypes.c_char_p
    L.rk_strerror.argtypes = [ctypes.c_int]
    L.rk_build.restype = ctypes.c_int
    L.rk_build.argtypes = [vp, vp, u32, ctypes.POINTER(BuildOpts), ctypes.POINTER(vp)]
    L.rk_destroy.restype = None
    L.rk_destroy.argtypes = [vp]
    L.rk_table_info_get.restype = ctypes.c_int
    L.rk_table_info_get.argtypes = [vp, ctypes.POINTER(TableInfo)]
    L.rk_workspace_bytes.restype = u64
    L.rk_workspace_bytes.argtypes = [vp, u64]
    L.rk_scan_device.restype = ctypes.c_int
    L.rk_scan_device.argtypes = [vp, vp, u64, vp, u64, vp, vp]
    L.rk_sort_device.restype = ctypes.c_int
    L.rk_sort_device.argtypes = [vp, u64, vp, u64, vp, vp, u64, vp]
    L.rk_search_device.restype = ctypes.c_int
    L.rk_search_device.argtypes = [vp, vp, u64, vp, u64, vp, vp, u64, vp]
    L.rk_search.restype = ctypes.c_int
    L.rk_search.argtypes = [vp, vp, u64, vp, u64, ctypes.POINTER(u64)]
    L.rk_window_hashes_device.restype = ctypes.c_int
    L.rk_window_hashes_device.argtypes = [vp, u64, u32, u32, vp, vp]
    L.rk_search_device_noalloc.restype = ctypes.c_int
    L.rk_search_device_noalloc.argtypes = [vp, vp, u64, vp, u64, vp, vp]
    _lib = L
    return L


def strerror(code: int) -> str:
    return load().rk_strerror(code).decode()


def _check(code: int, where: str) -> None:
    if code != RK_OK:
        raise RkError(code, where)


def _ptr(x) -> int:
    """Address of a torch tensor, numpy array or integer address."""
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return int(x.data_ptr())
    if isinstance(x, np.ndarray):
        return int(x.ctypes.data)
    raise TypeError(f"cannot take the address of {type(x)!r}")


def _stream(stream) -> int:
    if stream is None:
        return 0
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


# ------------------------------------------------------------------ entry points

def rk_build(patterns: Sequence[bytes], base_log2: int = 0, filter: int = RK_FILTER_AUTO,
             filter_log2_bits: int = 0, warps: int = 0, tile_bytes: int = 0, stages: int = 0,
             ctas_per_sm: int = 0) -> int:
    """Build a table from a sequence of byte strings; returns the handle."""
    L = load()
    lens = np.array([len(p) for p in patterns], dtype=np.uint32)
    cat = np.frombuffer(b"".join(bytes(p) for p in patterns) or b"\0", dtype=np.uint8).copy()
    opts = BuildOpts(base_log2, filter, filter_log2_bits, warps, tile_bytes, stages, ctas_per_sm)
    out = ctypes.c_void_p()
    _check(L.rk_build(cat.ctypes.data if len(patterns) else None,
                      lens.ctypes.data if len(patterns) else None,
                      len(patterns), ctypes.byref(opts), ctypes.byref(out)), "rk_build")
    return int(out.value)


def rk_destroy(table: int) -> None:
    load().rk_destroy(table)


def rk_table_info(table: int) -> dict:
    info = TableInfo()
    _check(load().rk_table_info_get(table, ctypes.byref(info)), "rk_table_info_get")
    return {name: getattr(info, name) for name, _ in TableInfo._fields_}


def rk_workspace_bytes(table: int, capacity: int) -> int:
    return int(load().rk_workspace_bytes(table, capacity))


def rk_scan_device(table: int, d_text, n: int, d_keys, capacity: int, d_info,
                   stream=None) -> None:
    _check(load().rk_scan_device(table, _ptr(d_text), n, _ptr(d_keys), capacity, _ptr(d_info),
                                 _stream(stream)), "rk_scan_device")


def rk_sort_device(table: int, n: int, d_keys, capacity: int, d_info, d_workspace,
                   workspace_bytes: int, stream=None) -> None:
    _check(load().rk_sort_device(table, n, _ptr(d_keys), capacity, _ptr(d_info),
                                 _ptr(d_workspace), workspace_bytes, _stream(stream)),
           "rk_sort_device")


def rk_search_device(table: int, d_text, n: int, d_keys, capacity: int, d_info, d_workspace,
                     workspace_bytes: int, stream=None) -> None:
    _check(load().rk_search_device(table, _ptr(d_text), n, _ptr(d_keys), capacity, _ptr(d_info),
                                   _ptr(d_workspace), workspace_bytes, _stream(stream)),
           "rk_search_device")


def rk_search(table: int, h_text, n: int, h_keys, capacity: int) -> Tuple[int, int]:
    """Host-buffer search.  Returns (status, n_matches); RK_ECAPACITY is
    returned, not raised, so the caller can retry with the reported count."""
    cnt = ctypes.c_uint64(0)
    rc = load().rk_search(table, _ptr(h_text), n, _ptr(h_keys), capacity, ctypes.byref(cnt))
    if rc not in (RK_OK, RK_ECAPACITY):
        raise RkError(rc, "rk_search")
    return rc, int(cnt.value)


def rk_window_hashes_device(d_text, n: int, L: int, base_log2: int, d_hashes,
                            stream=None) -> None:
    _check(load().rk_window_hashes_device(_ptr(d_text), n, L, base_log2, _ptr(d_hashes),
                                          _stream(stream)), "rk_window_hashes_device")


def rk_search_device_noalloc(table: int, d_text, n: int, d_keys, capacity: int, d_info,
                             stream=None) -> None:
    """rk_search_device for callers that cannot allocate: the sort's scratch is
    a fixed array inside the library (capacity <= RK_NOALLOC_MAX_KEYS); calls
    that overlap on the GPU race on it."""
    _check(load().rk_search_device_noalloc(table, _ptr(d_text), n, _ptr(d_keys), capacity,
                                           _ptr(d_info), _stream(stream)),
           "rk_search_device_noalloc")


# ------------------------------------------------------------------ key packing

def unpack_keys(keys: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """Split keys (id << 40 | x) into (ids uint32, offsets uint64)."""
    keys = np.asarray(keys, dtype=np.uint64)
    ids = (keys >> np.uint64(RK_KEY_OFFSET_BITS)).astype(np.uint32)
    offs = keys & np.uint64((1 << RK_KEY_OFFSET_BITS) - 1)
    return ids, offs
