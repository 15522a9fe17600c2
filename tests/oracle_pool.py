"""The oracle over a whole large text, split across host cores (test
infrastructure): the text goes once into shared memory, each worker process
runs the oracle's Rabin-Karp on one contiguous chunk plus the (longest
pattern - 1) bytes after it, and keeps the matches that start in its chunk,
so every match is found exactly once.  The oracle itself is unchanged; this
only cuts its input into pieces.

The pool uses the spawn start method, so it may be created after the parent
has initialised CUDA.
"""

from __future__ import annotations

import multiprocessing as mp
import os
from multiprocessing import shared_memory
from typing import Sequence, Tuple

import numpy as np

CHUNK = 32 << 20


def _chunk_job(args):
    shm_name, n, start, chunk, lmax, patterns = args
    import oracle  # worker process

    shm = shared_memory.SharedMemory(name=shm_name)
    try:
        text = np.ndarray((n,), dtype=np.uint8, buffer=shm.buf)
        end = min(n, start + chunk + lmax - 1)
        ids, offs = oracle.rabin_karp(np.array(text[start:end]), patterns)
        keep = offs < chunk
        return ids[keep].copy(), offs[keep].astype(np.uint64) + np.uint64(start)
    finally:
        del text
        shm.close()


def oracle_matches(text: np.ndarray, patterns: Sequence[bytes], start: int = 0,
                   procs: int = 0, chunk: int = CHUNK) -> Tuple[np.ndarray, np.ndarray]:
    """(ids, offsets) of every match starting at or after `start`, ascending
    by (id, offset), from the oracle's Rabin-Karp run on chunks in parallel."""
    n = int(text.size)
    if not patterns or n == 0:
        return np.zeros(0, np.uint32), np.zeros(0, np.uint64)
    lmax = max(len(p) for p in patterns)
    procs = procs or os.cpu_count() or 1
    shm = shared_memory.SharedMemory(create=True, size=max(n, 1))
    try:
        np.ndarray((n,), dtype=np.uint8, buffer=shm.buf)[:] = text
        jobs = [(shm.name, n, s, min(chunk, n - s), lmax, list(patterns))
                for s in range(start, n, chunk)]
        with mp.get_context("spawn").Pool(min(procs, len(jobs))) as pool:
            parts = pool.map(_chunk_job, jobs)
    finally:
        shm.close()
        shm.unlink()
    ids = np.concatenate([p[0] for p in parts]).astype(np.uint64)
    offs = np.concatenate([p[1] for p in parts])
    order = np.argsort((ids << np.uint64(40)) | offs, kind="stable")
    return ids[order].astype(np.uint32), offs[order]


def _item_job(args):
    text_bytes, patterns, keep_below, base = args
    import oracle  # worker process

    ids, offs = oracle.rabin_karp(np.frombuffer(text_bytes, dtype=np.uint8), patterns)
    keep = offs < keep_below
    return ids[keep].copy(), offs[keep].astype(np.uint64) + np.uint64(base)


def oracle_items(items, procs: int = 0, chunk: int = 4 << 20):
    """The oracle's (ids, offsets) for each (text, patterns) item, every item
    on its own; texts longer than `chunk` are cut into chunks with the same
    (longest pattern - 1)-byte overlap as oracle_matches, all on a spawn pool."""
    jobs, owner = [], []
    for i, (text, patterns) in enumerate(items):
        n = int(text.size)
        if not patterns or n == 0:
            continue
        lmax = max(len(p) for p in patterns)
        for s in range(0, n, chunk):
            jobs.append((text[s:min(n, s + chunk + lmax - 1)].tobytes(), list(patterns),
                         min(chunk, n - s), s))
            owner.append(i)
    procs = procs or os.cpu_count() or 1
    parts = []
    if jobs:
        with mp.get_context("spawn").Pool(min(procs, len(jobs))) as pool:
            parts = pool.map(_item_job, jobs, chunksize=1)
    out = [[] for _ in items]
    for i, p in zip(owner, parts):
        out[i].append(p)
    res = []
    for ps in out:
        if not ps:
            res.append((np.zeros(0, np.uint32), np.zeros(0, np.uint64)))
            continue
        ids = np.concatenate([p[0] for p in ps]).astype(np.uint64)
        offs = np.concatenate([p[1] for p in ps])
        order = np.argsort((ids << np.uint64(40)) | offs, kind="stable")
        res.append((ids[order].astype(np.uint32), offs[order]))
    return res
