"""Oracle for multi-pattern Rabin-Karp matching: TEST INFRASTRUCTURE ONLY.

Only the tests, the smoke check and the bench's CPU-baseline and reference
legs may import this package.  The library under test never does.

Python front end over ``rk_oracle.c`` (compiled on first use with gcc):

* ``bruteforce(text, patterns)``  the definition of the result set
  M = {(p, x) : T[x .. x+len_p) == P_p} in ascending (p, x) order
  (problem statement of Section 1; per-offset windows of Section 3.1);
* ``rabin_karp(text, patterns, base)``  Section 3.1's hash-then-compare
  method over a pattern set, hashes mod 2^61 - 1;
* ``rk_hash(s, base)``, ``window_hashes(text, L, base)``, ``mulmod(a, b)``
  the Rabin hash h(s) = sum_i s[i] * B^(len-1-i) mod (2^61 - 1).

Both matchers return ``(pattern_ids: uint32[M], offsets: uint64[M])``.
"""

from __future__ import annotations

import ctypes
from typing import Dict, List, Sequence, Tuple

import numpy as np

from .build import build as _build

P61 = (1 << 61) - 1

_libs: Dict[int, ctypes.CDLL] = {}


def lib(mutant: int = 0) -> ctypes.CDLL:
    if mutant in _libs:
        return _libs[mutant]
    L = ctypes.CDLL(_build(mutant))
    u8p = ctypes.POINTER(ctypes.c_uint8)
    u32p = ctypes.POINTER(ctypes.c_uint32)
    u64p = ctypes.POINTER(ctypes.c_uint64)
    L.oracle_mulmod.restype = ctypes.c_uint64
    L.oracle_mulmod.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
    L.oracle_powmod.restype = ctypes.c_uint64
    L.oracle_powmod.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
    L.oracle_hash.restype = ctypes.c_uint64
    L.oracle_hash.argtypes = [u8p, ctypes.c_uint64, ctypes.c_uint64]
    L.oracle_window_hashes.restype = ctypes.c_uint64
    L.oracle_window_hashes.argtypes = [u8p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, u64p]
    L.oracle_bruteforce.restype = ctypes.c_int64
    L.oracle_bruteforce.argtypes = [u8p, ctypes.c_uint64, u8p, u32p, ctypes.c_uint32,
                                    u32p, u64p, ctypes.c_uint64]
    L.oracle_rabin_karp.restype = ctypes.c_int64
    L.oracle_rabin_karp.argtypes = [u8p, ctypes.c_uint64, u8p, u32p, ctypes.c_uint32,
                                    ctypes.c_uint64, u32p, u64p, ctypes.c_uint64]
    L.oracle_mutant_id.restype = ctypes.c_int
    _libs[mutant] = L
    return L


def _u8(a) -> Tuple[np.ndarray, "ctypes._Pointer"]:
    if isinstance(a, (bytes, bytearray, memoryview)):
        a = np.frombuffer(bytes(a), dtype=np.uint8)
    a = np.ascontiguousarray(a, dtype=np.uint8)
    if a.size == 0:
        a = np.zeros(1, dtype=np.uint8)[:0]
        buf = np.zeros(1, dtype=np.uint8)
        return a, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def _patterns(patterns: Sequence[bytes]):
    lens = np.array([len(p) for p in patterns], dtype=np.uint32)
    cat = np.frombuffer(b"".join(bytes(p) for p in patterns) or b"\0", dtype=np.uint8).copy()
    return cat, lens


def _run(fn_name: str, text, patterns: Sequence[bytes], extra: tuple, mutant: int):
    L = lib(mutant)
    t, tp = _u8(text)
    cat, lens = _patterns(patterns)
    k = len(patterns)
    lens_p = (lens if k else np.zeros(1, np.uint32)).ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))
    fn = getattr(L, fn_name)
    cap = 1 << 16
    while True:
        pid = np.empty(max(cap, 1), dtype=np.uint32)
        off = np.empty(max(cap, 1), dtype=np.uint64)
        cnt = fn(tp, t.size, cat.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), lens_p, k,
                 *extra, pid.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                 off.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), cap)
        if cnt < 0:
            raise MemoryError(f"{fn_name} ran out of memory")
        if cnt <= cap:
            return pid[:cnt].copy(), off[:cnt].copy()
        cap = int(cnt)


def bruteforce(text, patterns: Sequence[bytes], mutant: int = 0):
    """All (pattern id, offset) matches by direct comparison, ascending."""
    return _run("oracle_bruteforce", text, patterns, (), mutant)


def rabin_karp(text, patterns: Sequence[bytes], base: int = 256, mutant: int = 0):
    """All (pattern id, offset) matches by Rabin-Karp mod 2^61-1, ascending."""
    if not (2 <= base < P61):
        raise ValueError("base must be in [2, 2^61 - 1)")
    return _run("oracle_rabin_karp", text, patterns, (ctypes.c_uint64(base),), mutant)


def mulmod(a: int, b: int, mutant: int = 0) -> int:
    return int(lib(mutant).oracle_mulmod(a, b))


def powmod(b: int, e: int, mutant: int = 0) -> int:
    return int(lib(mutant).oracle_powmod(b, e))


def rk_hash(s, base: int = 256, mutant: int = 0) -> int:
    """h(s) = sum_i s[i] * base^(len-1-i) mod 2^61-1."""
    a, p = _u8(s)
    return int(lib(mutant).oracle_hash(p, a.size, base))


def window_hashes(text, L: int, base: int = 256, mutant: int = 0) -> np.ndarray:
    """Hash of every length-L window of text, by the rolling update."""
    t, tp = _u8(text)
    if L == 0 or L > t.size:
        return np.zeros(0, dtype=np.uint64)
    out = np.empty(t.size - L + 1, dtype=np.uint64)
    n = lib(mutant).oracle_window_hashes(tp, t.size, L, base,
                                         out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)))
    return out[:n]


def as_pairs(pids: np.ndarray, offs: np.ndarray) -> List[Tuple[int, int]]:
    return list(zip(pids.tolist(), offs.tolist()))
