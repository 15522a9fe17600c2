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
RK_NOALLOC_SCRATCH_BYTES = 16785920

#: names of every function include/rk.h declares
EXPORTS = [
    "rk_strerror", "rk_build", "rk_plan", "rk_destroy", "rk_table_info_get", "rk_workspace_bytes",
    "rk_sort_launches", "rk_scan_workspace_bytes", "rk_scan_device_ws", "rk_scan_launches",
    "rk_scan_device", "rk_sort_device", "rk_search_device", "rk_search",
    "rk_window_hashes_device", "rk_search_device_noalloc",
    "rk_tableset_build", "rk_tableset_destroy", "rk_batch_create", "rk_batch_destroy",
    "rk_batch_info_get", "rk_batch_set", "rk_batch_run", "rk_batch_results", "rk_batch_read",
    "rk_batch_autotune", "rk_server_create", "rk_server_destroy", "rk_server_submit",
    "rk_server_take", "rk_server_stats_get", "rk_paper_search_device",
    "rk_debug_scan_withheld", "rk_build_ptrs", "rk_search_matches", "rk_search_device_matches",
    "rk_free_matches", "rk_debug_binary_version", "rk_scan_device_ws_split",
]


class RkError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {strerror(code)} ({code})")


class BuildOpts(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint32) for n in (
        "base_log2", "filter", "filter_log2_bits", "warps", "tile_bytes", "stages", "ctas_per_sm",
        "sample", "role_step")]


class Match(ctypes.Structure):
    """rk_match: one (pattern id, offset) record."""
    _fields_ = [("offset", ctypes.c_uint64), ("pattern_id", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32)]


#: numpy view of an rk_match array
MATCH_DTYPE = np.dtype([("offset", np.uint64), ("pattern_id", np.uint32), ("reserved", np.uint32)])


class TableInfo(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint32) for n in (
        "n_patterns", "min_len", "max_len", "n_lengths", "gram_len", "base_log2", "filter",
        "filter_log2_bits", "filter_smem_bytes", "n_grams", "warps", "tile_bytes", "stages",
        "ctas_per_sm", "halo_bytes", "smem_bytes", "sm_count", "device", "s2_smem_bytes")] + [
        ("device_bytes", ctypes.c_uint64)] + [
        (n, ctypes.c_uint32) for n in ("sample_step", "sample_filter_log2_bits", "role_step",
                                       "role_filter_log2_bits", "survivor_warps",
                                       "role_side_log2_bits")]


class BatchOpts(ctypes.Structure):
    _fields_ = [("max_items", ctypes.c_uint32), ("max_text_len", ctypes.c_uint64),
                ("max_total_bytes", ctypes.c_uint64), ("capacity", ctypes.c_uint64)] + [
        (n, ctypes.c_uint32) for n in ("warps", "tile_bytes", "stages", "ctas_per_sm",
                                       "s2_in_smem")]


class BatchInfo(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint32) for n in (
        "offset_bits", "id_bits", "item_bits", "warps", "tile_bytes", "stages", "ctas_per_sm",
        "s2_in_smem", "smem_bytes", "n_chunks", "max_chunks", "n_items")]


class ServerOpts(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in (
        "mem_cap", "max_text_len", "max_batch_bytes", "batch_capacity")] + [
        (n, ctypes.c_uint32) for n in ("engines", "max_batch_items", "tile_bytes", "warps")]


class RequestTimes(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("arrive_us", "admit_us", "launch_us", "done_us")]


class ServerStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in (
        "requests_done", "bytes_done", "batches", "items_batched", "waiting", "in_flight",
        "arena_used")] + [("now_us", ctypes.c_double)]


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
    L.rk_plan.restype = ctypes.c_int
    L.rk_plan.argtypes = [vp, vp, u32, ctypes.POINTER(BuildOpts), u32, ctypes.POINTER(TableInfo)]
    L.rk_destroy.restype = None
    L.rk_destroy.argtypes = [vp]
    L.rk_table_info_get.restype = ctypes.c_int
    L.rk_table_info_get.argtypes = [vp, ctypes.POINTER(TableInfo)]
    L.rk_workspace_bytes.restype = u64
    L.rk_workspace_bytes.argtypes = [vp, u64]
    L.rk_sort_launches.restype = ctypes.c_int
    L.rk_sort_launches.argtypes = [vp, u64, u64, ctypes.POINTER(u32)]
    L.rk_scan_device.restype = ctypes.c_int
    L.rk_scan_device.argtypes = [vp, vp, u64, vp, u64, vp, vp]
    L.rk_scan_workspace_bytes.restype = u64
    L.rk_scan_workspace_bytes.argtypes = [vp, u64]
    L.rk_scan_launches.restype = ctypes.c_int
    L.rk_scan_launches.argtypes = [vp, u64, u64, ctypes.POINTER(u32)]
    L.rk_scan_device_ws.restype = ctypes.c_int
    L.rk_scan_device_ws.argtypes = [vp, vp, u64, vp, u64, vp, vp, u64, vp]
    L.rk_scan_device_ws_split.restype = ctypes.c_int
    L.rk_scan_device_ws_split.argtypes = [vp, vp, u64, vp, u64, vp, vp, u64, vp, vp]
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
    L.rk_tableset_build.restype = ctypes.c_int
    L.rk_tableset_build.argtypes = [u32, vp, vp, vp, ctypes.POINTER(BuildOpts), ctypes.POINTER(vp)]
    L.rk_tableset_destroy.restype = None
    L.rk_tableset_destroy.argtypes = [vp]
    L.rk_batch_create.restype = ctypes.c_int
    L.rk_batch_create.argtypes = [vp, ctypes.POINTER(BatchOpts), ctypes.POINTER(vp)]
    L.rk_batch_destroy.restype = None
    L.rk_batch_destroy.argtypes = [vp]
    L.rk_batch_info_get.restype = ctypes.c_int
    L.rk_batch_info_get.argtypes = [vp, ctypes.POINTER(BatchInfo)]
    L.rk_batch_set.restype = ctypes.c_int
    L.rk_batch_set.argtypes = [vp, u32, vp, vp, vp, vp]
    L.rk_batch_run.restype = ctypes.c_int
    L.rk_batch_run.argtypes = [vp, vp]
    L.rk_batch_results.restype = ctypes.c_int
    L.rk_batch_results.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp)]
    L.rk_batch_read.restype = ctypes.c_int
    L.rk_batch_read.argtypes = [vp, vp, u64, vp, vp, vp]
    L.rk_batch_autotune.restype = ctypes.c_int
    L.rk_batch_autotune.argtypes = [vp, u32, u32, ctypes.POINTER(ctypes.c_double), vp]
    L.rk_server_create.restype = ctypes.c_int
    L.rk_server_create.argtypes = [vp, ctypes.POINTER(ServerOpts), ctypes.POINTER(vp)]
    L.rk_server_destroy.restype = None
    L.rk_server_destroy.argtypes = [vp]
    L.rk_server_submit.restype = ctypes.c_int
    L.rk_server_submit.argtypes = [vp, u32, vp, u64, ctypes.POINTER(u64)]
    L.rk_server_take.restype = ctypes.c_int
    L.rk_server_take.argtypes = [vp, u64, ctypes.c_int, vp, u64, ctypes.POINTER(u64),
                                 ctypes.POINTER(RequestTimes)]
    L.rk_server_stats_get.restype = ctypes.c_int
    L.rk_server_stats_get.argtypes = [vp, ctypes.POINTER(ServerStats)]
    L.rk_paper_search_device.restype = ctypes.c_int
    L.rk_paper_search_device.argtypes = [vp, u64, vp, u32, vp, u32, vp]
    L.rk_debug_scan_withheld.restype = ctypes.c_int
    L.rk_debug_scan_withheld.argtypes = [vp, vp, u64, vp, u64, vp, u32, vp]
    L.rk_build_ptrs.restype = ctypes.c_int
    L.rk_build_ptrs.argtypes = [vp, vp, u32, ctypes.POINTER(BuildOpts), ctypes.POINTER(vp)]
    L.rk_search_matches.restype = ctypes.c_int
    L.rk_search_matches.argtypes = [vp, vp, u64, ctypes.POINTER(vp), ctypes.POINTER(u64)]
    L.rk_search_device_matches.restype = ctypes.c_int
    L.rk_search_device_matches.argtypes = [vp, vp, u64, vp, vp, u64, ctypes.POINTER(u64)]
    L.rk_free_matches.restype = None
    L.rk_free_matches.argtypes = [vp]
    L.rk_debug_binary_version.restype = ctypes.c_int
    L.rk_debug_binary_version.argtypes = [ctypes.POINTER(ctypes.c_int)]
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


def _buf(x, need: int, what: str, device: bool) -> int:
    """Address of a buffer argument, after the checks the binding can make: a
    tensor or array must be contiguous, hold `need` bytes and live where the
    call reads it (device memory for the d_ arguments, host memory for the h_
    ones: a host address handed to a kernel would fault the GPU).  A raw
    integer address is passed through, as the C contract allows."""
    if x is None or isinstance(x, int):
        return _ptr(x)
    if hasattr(x, "data_ptr") and hasattr(x, "is_cuda"):
        if bool(x.is_cuda) != device:
            raise RkError(RK_EINVAL, f"{what}: a {'CUDA' if device else 'host'} tensor is required")
        if not x.is_contiguous():
            raise RkError(RK_EINVAL, f"{what}: not contiguous")
        have = x.numel() * x.element_size()
    elif isinstance(x, np.ndarray):
        if device:
            raise RkError(RK_EINVAL, f"{what}: a numpy array is host memory")
        if not x.flags["C_CONTIGUOUS"]:
            raise RkError(RK_EINVAL, f"{what}: not contiguous")
        have = x.nbytes
    else:
        return _ptr(x)
    if have < need:
        raise RkError(RK_EINVAL, f"{what}: {have} bytes, the call needs {need}")
    return _ptr(x)


def _stream(stream) -> int:
    if stream is None:
        return 0
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


# ------------------------------------------------------------------ entry points

def rk_build(patterns: Sequence[bytes], base_log2: int = 0, filter: int = RK_FILTER_AUTO,
             filter_log2_bits: int = 0, warps: int = 0, tile_bytes: int = 0, stages: int = 0,
             ctas_per_sm: int = 0, sample: int = 0, role_step: int = 0) -> int:
    """Build a table from a sequence of byte strings; returns the handle."""
    L = load()
    lens = np.array([len(p) for p in patterns], dtype=np.uint32)
    cat = np.frombuffer(b"".join(bytes(p) for p in patterns) or b"\0", dtype=np.uint8).copy()
    opts = BuildOpts(base_log2, filter, filter_log2_bits, warps, tile_bytes, stages, ctas_per_sm,
                     sample, role_step)
    out = ctypes.c_void_p()
    _check(L.rk_build(cat.ctypes.data if len(patterns) else None,
                      lens.ctypes.data if len(patterns) else None,
                      len(patterns), ctypes.byref(opts), ctypes.byref(out)), "rk_build")
    return int(out.value)


#: opt-in shared memory per block of a GB300 (cudaDevAttrMaxSharedMemoryPerBlockOptin)
GB300_SMEM_OPTIN = 232448


def rk_plan(patterns: Sequence[bytes], smem_optin: int = GB300_SMEM_OPTIN, base_log2: int = 0,
            filter: int = RK_FILTER_AUTO, filter_log2_bits: int = 0, warps: int = 0,
            tile_bytes: int = 0, stages: int = 0, ctas_per_sm: int = 0, sample: int = 0,
            role_step: int = 0) -> dict:
    """What rk_build would give these patterns on a device with `smem_optin`
    bytes of opt-in shared memory per block, worked out on the host (no GPU);
    the keys of rk_table_info."""
    L = load()
    lens = np.array([len(p) for p in patterns], dtype=np.uint32)
    cat = np.frombuffer(b"".join(bytes(p) for p in patterns) or b"\0", dtype=np.uint8).copy()
    opts = BuildOpts(base_log2, filter, filter_log2_bits, warps, tile_bytes, stages, ctas_per_sm,
                     sample, role_step)
    info = TableInfo()
    _check(L.rk_plan(cat.ctypes.data if len(patterns) else None,
                     lens.ctypes.data if len(patterns) else None,
                     len(patterns), ctypes.byref(opts), smem_optin, ctypes.byref(info)), "rk_plan")
    return {name: getattr(info, name) for name, _ in TableInfo._fields_}


def rk_destroy(table: int) -> None:
    load().rk_destroy(table)


def rk_table_info(table: int) -> dict:
    info = TableInfo()
    _check(load().rk_table_info_get(table, ctypes.byref(info)), "rk_table_info_get")
    return {name: getattr(info, name) for name, _ in TableInfo._fields_}


def rk_workspace_bytes(table: int, capacity: int) -> int:
    return int(load().rk_workspace_bytes(table, capacity))


def rk_sort_launches(table: int, n: int, capacity: int) -> int:
    """Kernels rk_sort_device launches for a text of n bytes and `capacity` keys."""
    out = ctypes.c_uint32(0)
    rc = load().rk_sort_launches(table, n, capacity, ctypes.byref(out))
    if rc != RK_OK:
        raise RuntimeError(f"rk_sort_launches: {strerror(rc)}")
    return int(out.value)


def rk_scan_device(table: int, d_text, n: int, d_keys, capacity: int, d_info,
                   stream=None) -> None:
    _check(load().rk_scan_device(table, _buf(d_text, n, "d_text", True), n,
                                 _buf(d_keys, 8 * capacity, "d_keys", True), capacity,
                                 _buf(d_info, 16, "d_info", True),
                                 _stream(stream)), "rk_scan_device")


def rk_scan_workspace_bytes(table: int, n: int) -> int:
    """Workspace bytes of rk_scan_device_ws for a text of n bytes."""
    return int(load().rk_scan_workspace_bytes(table, n))


def rk_scan_launches(table: int, n: int, workspace_bytes: int) -> int:
    """Kernels rk_scan_device_ws launches for n text bytes and this workspace."""
    out = ctypes.c_uint32(0)
    rc = load().rk_scan_launches(table, n, workspace_bytes, ctypes.byref(out))
    if rc != RK_OK:
        raise RuntimeError(f"rk_scan_launches: {strerror(rc)}")
    return int(out.value)


def rk_scan_device_ws(table: int, d_text, n: int, d_keys, capacity: int, d_info, d_workspace,
                      workspace_bytes: int, stream=None) -> None:
    """rk_scan_device with the survivors verified by a second kernel."""
    _check(load().rk_scan_device_ws(table, _buf(d_text, n, "d_text", True), n,
                                    _buf(d_keys, 8 * capacity, "d_keys", True), capacity,
                                    _buf(d_info, 16, "d_info", True),
                                    _buf(d_workspace, workspace_bytes, "d_workspace", True),
                                    workspace_bytes, _stream(stream)),
           "rk_scan_device_ws")


def rk_scan_device_ws_split(table: int, d_text, n: int, d_keys, capacity: int, d_info,
                            d_workspace, workspace_bytes: int, stream=None, mid_event=None) -> None:
    """rk_scan_device_ws recording `mid_event` (a torch.cuda.Event that has
    been recorded once, so that it exists, or a raw cudaEvent_t) between the
    tile scan and the verification kernel."""
    ev = None
    if mid_event is not None:
        ev = int(getattr(mid_event, "cuda_event", mid_event))
        if not ev:
            raise ValueError("mid_event: the event has not been created (record it once first)")
    _check(load().rk_scan_device_ws_split(table, _buf(d_text, n, "d_text", True), n,
                                          _buf(d_keys, 8 * capacity, "d_keys", True), capacity,
                                          _buf(d_info, 16, "d_info", True),
                                          _buf(d_workspace, workspace_bytes, "d_workspace", True),
                                          workspace_bytes, _stream(stream), ev),
           "rk_scan_device_ws_split")


def rk_sort_device(table: int, n: int, d_keys, capacity: int, d_info, d_workspace,
                   workspace_bytes: int, stream=None) -> None:
    _check(load().rk_sort_device(table, n, _buf(d_keys, 8 * capacity, "d_keys", True), capacity,
                                 _buf(d_info, 16, "d_info", True),
                                 _buf(d_workspace, workspace_bytes, "d_workspace", True),
                                 workspace_bytes, _stream(stream)),
           "rk_sort_device")


def rk_search_device(table: int, d_text, n: int, d_keys, capacity: int, d_info, d_workspace,
                     workspace_bytes: int, stream=None) -> None:
    _check(load().rk_search_device(table, _buf(d_text, n, "d_text", True), n,
                                   _buf(d_keys, 8 * capacity, "d_keys", True), capacity,
                                   _buf(d_info, 16, "d_info", True),
                                   _buf(d_workspace, workspace_bytes, "d_workspace", True),
                                   workspace_bytes, _stream(stream)),
           "rk_search_device")


def rk_search(table: int, h_text, n: int, h_keys, capacity: int) -> Tuple[int, int]:
    """Host-buffer search.  Returns (status, n_matches); RK_ECAPACITY is
    returned, not raised, so the caller can retry with the reported count."""
    cnt = ctypes.c_uint64(0)
    rc = load().rk_search(table, _buf(h_text, n, "h_text", False), n,
                          _buf(h_keys, 8 * capacity, "h_keys", False), capacity, ctypes.byref(cnt))
    if rc not in (RK_OK, RK_ECAPACITY):
        raise RkError(rc, "rk_search")
    return rc, int(cnt.value)


def rk_build_ptrs(patterns: Sequence[bytes], **opts) -> int:
    """rk_build from one pointer per pattern (the bytes stay in Python
    buffers for the call); returns the handle."""
    L = load()
    bufs = [ctypes.create_string_buffer(bytes(p), max(len(p), 1)) for p in patterns]
    ptrs = (ctypes.c_void_p * max(len(bufs), 1))(*[ctypes.addressof(b) for b in bufs])
    lens = np.array([len(p) for p in patterns] or [0], dtype=np.uint32)
    o = BuildOpts(*(opts.get(name, 0) for name, _ in BuildOpts._fields_))
    out = ctypes.c_void_p()
    _check(L.rk_build_ptrs(ctypes.addressof(ptrs) if patterns else None,
                           lens.ctypes.data if patterns else None, len(patterns),
                           ctypes.byref(o), ctypes.byref(out)), "rk_build_ptrs")
    return int(out.value)


def rk_search_matches(table: int, h_text, n: int) -> np.ndarray:
    """Host-buffer search into library-allocated records; returns a copy as a
    numpy array of MATCH_DTYPE (the library's list is freed)."""
    L = load()
    out = ctypes.c_void_p()
    cnt = ctypes.c_uint64(0)
    _check(L.rk_search_matches(table, _buf(h_text, n, "h_text", False), n, ctypes.byref(out),
                               ctypes.byref(cnt)), "rk_search_matches")
    try:
        m = int(cnt.value)
        raw = ctypes.string_at(out.value, m * MATCH_DTYPE.itemsize) if m else b""
        return np.frombuffer(raw, dtype=MATCH_DTYPE).copy()
    finally:
        L.rk_free_matches(out)


def rk_search_device_matches(table: int, d_text, n: int, d_out, capacity: int,
                             stream=None) -> Tuple[int, int]:
    """Device-buffer search into records d_out[0..capacity).  Returns (status,
    n_matches); RK_ECAPACITY is returned, not raised."""
    cnt = ctypes.c_uint64(0)
    rc = load().rk_search_device_matches(table, _buf(d_text, n, "d_text", True), n,
                                         _stream(stream),
                                         _buf(d_out, MATCH_DTYPE.itemsize * capacity, "d_out", True),
                                         capacity, ctypes.byref(cnt))
    if rc not in (RK_OK, RK_ECAPACITY):
        raise RkError(rc, "rk_search_device_matches")
    return rc, int(cnt.value)


def rk_debug_binary_version() -> int:
    v = ctypes.c_int(0)
    _check(load().rk_debug_binary_version(ctypes.byref(v)), "rk_debug_binary_version")
    return int(v.value)


def rk_window_hashes_device(d_text, n: int, L: int, base_log2: int, d_hashes,
                            stream=None) -> None:
    windows = n - L + 1 if 1 <= L <= n else 0
    _check(load().rk_window_hashes_device(_buf(d_text, n if windows else 0, "d_text", True), n, L,
                                          base_log2, _buf(d_hashes, 8 * windows, "d_hashes", True),
                                          _stream(stream)), "rk_window_hashes_device")


def rk_search_device_noalloc(table: int, d_text, n: int, d_keys, capacity: int, d_info,
                             stream=None) -> None:
    """rk_search_device for callers that cannot allocate: the sort's scratch is
    a fixed array inside the library (capacity <= RK_NOALLOC_MAX_KEYS); calls
    that overlap on the GPU race on it."""
    _check(load().rk_search_device_noalloc(table, _buf(d_text, n, "d_text", True), n,
                                           _buf(d_keys, 8 * capacity, "d_keys", True), capacity,
                                           _buf(d_info, 16, "d_info", True), _stream(stream)),
           "rk_search_device_noalloc")


def rk_debug_scan_withheld(table: int, d_text, n: int, d_keys, capacity: int, d_info,
                           timeout_ms: int, stream=None) -> None:
    """Failure-detection diagnostics: a scan whose copies never arrive, so its
    bounded waits run out and d_info[1] becomes RK_ETIMEOUT."""
    _check(load().rk_debug_scan_withheld(table, _buf(d_text, n, "d_text", True), n,
                                         _buf(d_keys, 8 * capacity, "d_keys", True), capacity,
                                         _buf(d_info, 16, "d_info", True), timeout_ms,
                                         _stream(stream)),
           "rk_debug_scan_withheld")


def rk_paper_search_device(d_text, n: int, pattern: bytes, d_result, threads_per_block: int = 0,
                           stream=None) -> None:
    """The paper's one-thread-per-offset matcher for one pattern; d_result[x] = 1
    where a match starts."""
    pat = np.frombuffer(bytes(pattern), dtype=np.uint8).copy()
    _check(load().rk_paper_search_device(_buf(d_text, n, "d_text", True) if n else None, n,
                                         pat.ctypes.data, len(pattern),
                                         _buf(d_result, n, "d_result", True) if n else None,
                                         threads_per_block, _stream(stream)),
           "rk_paper_search_device")


# ------------------------------------------------------------------ batches

def rk_tableset_build(tables: Sequence[Sequence[bytes]], base_log2: int = 0,
                      filter: int = RK_FILTER_AUTO, filter_log2_bits: int = 0) -> int:
    """One table per pattern list; returns the table-set handle."""
    L = load()
    per = np.array([len(t) for t in tables], dtype=np.uint32)
    flat = [bytes(p) for t in tables for p in t]
    lens = np.array([len(p) for p in flat] or [0], dtype=np.uint32)
    cat = np.frombuffer(b"".join(flat) or b"\0", dtype=np.uint8).copy()
    opts = BuildOpts(base_log2, filter, filter_log2_bits, 0, 0, 0, 0)
    out = ctypes.c_void_p()
    _check(L.rk_tableset_build(len(tables), cat.ctypes.data, lens.ctypes.data, per.ctypes.data,
                               ctypes.byref(opts), ctypes.byref(out)), "rk_tableset_build")
    return int(out.value)


def rk_tableset_destroy(ts: int) -> None:
    load().rk_tableset_destroy(ts)


def rk_batch_create(ts: int, max_items: int, max_text_len: int, max_total_bytes: int,
                    capacity: int, warps: int = 0, tile_bytes: int = 0, stages: int = 0,
                    ctas_per_sm: int = 0, s2_in_smem: int = 0) -> int:
    opts = BatchOpts(max_items, max_text_len, max_total_bytes, capacity, warps, tile_bytes,
                     stages, ctas_per_sm, s2_in_smem)
    out = ctypes.c_void_p()
    _check(load().rk_batch_create(ts, ctypes.byref(opts), ctypes.byref(out)), "rk_batch_create")
    return int(out.value)


def rk_batch_destroy(b: int) -> None:
    load().rk_batch_destroy(b)


def rk_batch_info(b: int) -> dict:
    info = BatchInfo()
    _check(load().rk_batch_info_get(b, ctypes.byref(info)), "rk_batch_info_get")
    return {name: getattr(info, name) for name, _ in BatchInfo._fields_}


def rk_batch_set(b: int, table_of_item: Sequence[int], d_texts: Sequence, text_lens: Sequence[int],
                 stream=None) -> None:
    n = len(table_of_item)
    if len(d_texts) != n or len(text_lens) != n:
        raise ValueError("rk_batch_set: one table index, text and length per item")
    tabs = np.asarray(table_of_item, dtype=np.uint32)
    ptrs = np.array([_buf(t, int(L), "d_texts", True) for t, L in zip(d_texts, text_lens)]
                    or [0], dtype=np.uint64)
    lens = np.asarray(list(text_lens) or [0], dtype=np.uint64)
    _check(load().rk_batch_set(b, n, tabs.ctypes.data if n else None, ptrs.ctypes.data,
                               lens.ctypes.data, _stream(stream)), "rk_batch_set")


def rk_batch_run(b: int, stream=None) -> None:
    _check(load().rk_batch_run(b, _stream(stream)), "rk_batch_run")


def rk_batch_results(b: int) -> Tuple[int, int, int]:
    k, o, i = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
    _check(load().rk_batch_results(b, ctypes.byref(k), ctypes.byref(o), ctypes.byref(i)),
           "rk_batch_results")
    return int(k.value or 0), int(o.value or 0), int(i.value or 0)


def rk_batch_read(b: int, n_items: int, key_cap: int, stream=None):
    """(count, status, keys uint64[min(count, key_cap)], offsets uint64[n_items+1]).
    n_items must be the item count of the last rk_batch_set (the offsets
    buffer is sized from the batch itself)."""
    have = rk_batch_info(b)["n_items"]
    if n_items != have:
        raise ValueError(f"rk_batch_read: the batch holds {have} items, not {n_items}")
    keys = np.empty(max(key_cap, 1), dtype=np.uint64)
    offs = np.zeros(have + 1, dtype=np.uint64)
    info = np.zeros(2, dtype=np.uint64)
    _check(load().rk_batch_read(b, keys.ctypes.data, key_cap, offs.ctypes.data,
                                info.ctypes.data, _stream(stream)), "rk_batch_read")
    count, status = int(info[0]), int(info[1])
    return count, status, keys[:min(count, key_cap)], offs


def rk_batch_autotune(b: int, max_candidates: int = 0, reps: int = 3, stream=None) -> float:
    best = ctypes.c_double(0)
    _check(load().rk_batch_autotune(b, max_candidates, reps, ctypes.byref(best), _stream(stream)),
           "rk_batch_autotune")
    return best.value


def rk_server_create(ts: int, mem_cap: int, max_text_len: int, max_batch_bytes: int = 0,
                     batch_capacity: int = 0, engines: int = 0, max_batch_items: int = 0,
                     tile_bytes: int = 0, warps: int = 0) -> int:
    opts = ServerOpts(mem_cap, max_text_len, max_batch_bytes, batch_capacity, engines,
                      max_batch_items, tile_bytes, warps)
    out = ctypes.c_void_p()
    _check(load().rk_server_create(ts, ctypes.byref(opts), ctypes.byref(out)), "rk_server_create")
    return int(out.value)


def rk_server_destroy(s: int) -> None:
    load().rk_server_destroy(s)


def rk_server_submit(s: int, table: int, h_text, n: int) -> int:
    """The host buffer must stay alive and unchanged until the request is taken."""
    rid = ctypes.c_uint64(0)
    _check(load().rk_server_submit(s, table, _buf(h_text, n, "h_text", False) if n else None, n,
                                   ctypes.byref(rid)),
           "rk_server_submit")
    return int(rid.value)


def rk_server_take(s: int, request_id: int, timeout_ms: int = -1, key_cap: int = 1 << 16):
    """(status, keys uint64[], times dict); grows the buffer when it is too small.
    status RK_ETIMEOUT: not finished within timeout_ms."""
    L = load()
    while True:
        keys = np.empty(max(key_cap, 1), dtype=np.uint64)
        n = ctypes.c_uint64(0)
        t = RequestTimes()
        rc = L.rk_server_take(s, request_id, timeout_ms, keys.ctypes.data, key_cap,
                              ctypes.byref(n), ctypes.byref(t))
        if rc == RK_ECAPACITY and n.value > key_cap:
            key_cap = int(n.value)
            continue
        times = {name: getattr(t, name) for name, _ in RequestTimes._fields_}
        return rc, keys[:n.value].copy() if rc == RK_OK else keys[:0], times


def rk_server_stats(s: int) -> dict:
    st = ServerStats()
    _check(load().rk_server_stats_get(s, ctypes.byref(st)), "rk_server_stats_get")
    return {name: getattr(st, name) for name, _ in ServerStats._fields_}


def unpack_batch_keys(keys: np.ndarray, offset_bits: int, id_bits: int):
    """Split batch keys into (items, ids, offsets)."""
    keys = np.asarray(keys, dtype=np.uint64)
    offs = keys & np.uint64((1 << offset_bits) - 1)
    ids = ((keys >> np.uint64(offset_bits)) & np.uint64((1 << id_bits) - 1)).astype(np.uint32)
    items = (keys >> np.uint64(offset_bits + id_bits)).astype(np.uint32)
    return items, ids, offs


# ------------------------------------------------------------------ key packing

def unpack_keys(keys: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """Split keys (id << 40 | x) into (ids uint32, offsets uint64)."""
    keys = np.asarray(keys, dtype=np.uint64)
    ids = (keys >> np.uint64(RK_KEY_OFFSET_BITS)).astype(np.uint32)
    offs = keys & np.uint64((1 << RK_KEY_OFFSET_BITS) - 1)
    return ids, offs
