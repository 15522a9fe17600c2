"""Seeded synthetic workloads shaped like the paper's experiments.

The paper (Section 3.3) scans random DNA text of 2 MB to 1 GB for short
patterns (m = 7 in Tables 1-2, m = 25..800 in Table 3).  Its files are not
available, so every input here is drawn from a seeded PCG64 generator with
the shapes below.  The recipe (draw order, distributions, planting) is fixed
so that any machine with the same NumPy produces the same bytes:

1. text, drawn in chunks of ``CHUNK`` bytes;
2. pattern lengths (all patterns), then pattern bytes (pattern by pattern);
3. plant offsets, pattern by pattern, uniform in ``[0, n - len]``; each plant
   overwrites the text with the pattern bytes, later plants over earlier ones.

Planted offsets are returned for diagnostics only: a later plant may destroy
an earlier one and natural occurrences exist, so the expected match list of a
workload is always computed from the final text.

Nothing in this module hashes or compares windows.
"""

from __future__ import annotations

import dataclasses
from typing import List, Optional, Sequence

import numpy as np

CHUNK = 1 << 26  # bytes drawn per generator call for large texts

#: English letter frequency rank order used for the Zipf text (rank 1 first).
ZIPF_ORDER = b"etaoinshrdlcumwfgypbvkjxqz"
#: probability that a position of the Zipf text is a space (mean word gap 6)
ZIPF_SPACE_P = 1.0 / 6.0
#: resolution of the symbol lookup table (probabilities are multiples of 2^-16)
LUT_BITS = 16


@dataclasses.dataclass
class Workload:
    """One synthetic search problem: a text and an ordered pattern list."""

    name: str
    text: np.ndarray  # uint8, 1-D, C-contiguous
    patterns: List[bytes]
    planted: List[np.ndarray]  # per pattern, planted offsets (diagnostic only)
    params: dict

    @property
    def n(self) -> int:
        return int(self.text.size)

    def pattern_lengths(self) -> np.ndarray:
        return np.array([len(p) for p in self.patterns], dtype=np.uint32)

    def concat_patterns(self) -> np.ndarray:
        if not self.patterns:
            return np.zeros(0, dtype=np.uint8)
        return np.frombuffer(b"".join(self.patterns), dtype=np.uint8).copy()


def _lut_from_weights(symbols: bytes, weights: Sequence[float]) -> np.ndarray:
    """Symbol lookup table of 2^16 entries: entry u holds the symbol whose
    cumulative-probability interval contains (u + 0.5) / 2^16."""
    w = np.asarray(weights, dtype=np.float64)
    cdf = np.cumsum(w / w.sum())
    size = 1 << LUT_BITS
    centres = (np.arange(size, dtype=np.float64) + 0.5) / size
    idx = np.searchsorted(cdf, centres, side="right")
    idx = np.minimum(idx, len(symbols) - 1)
    return np.frombuffer(symbols, dtype=np.uint8)[idx].copy()


def zipf_lut() -> np.ndarray:
    """Letters a-z with Zipf(s=1) weights over ``ZIPF_ORDER`` and a space with
    probability 1/6, quantised to a 2^16-entry table."""
    letters = ZIPF_ORDER
    lw = np.array([1.0 / r for r in range(1, len(letters) + 1)])
    lw = lw / lw.sum() * (1.0 - ZIPF_SPACE_P)
    return _lut_from_weights(letters + b" ", list(lw) + [ZIPF_SPACE_P])


def _draw_text_lut(rng: np.random.Generator, n: int, lut: np.ndarray) -> np.ndarray:
    text = np.empty(n, dtype=np.uint8)
    for s in range(0, n, CHUNK):
        e = min(n, s + CHUNK)
        text[s:e] = lut[rng.integers(0, 1 << LUT_BITS, e - s, dtype=np.uint16)]
    return text


def _draw_text_uniform(rng: np.random.Generator, n: int, alphabet: Optional[bytes]) -> np.ndarray:
    text = np.empty(n, dtype=np.uint8)
    if alphabet is None:
        for s in range(0, n, CHUNK):
            e = min(n, s + CHUNK)
            text[s:e] = rng.integers(0, 256, e - s, dtype=np.uint8)
    else:
        sym = np.frombuffer(alphabet, dtype=np.uint8)
        for s in range(0, n, CHUNK):
            e = min(n, s + CHUNK)
            text[s:e] = sym[rng.integers(0, len(sym), e - s, dtype=np.uint8)]
    return text


def _draw_patterns(rng, k, lmin, lmax, lut=None, alphabet=None) -> List[bytes]:
    lens = rng.integers(lmin, lmax + 1, k)
    pats = []
    for L in lens:
        L = int(L)
        if lut is not None:
            b = lut[rng.integers(0, 1 << LUT_BITS, L, dtype=np.uint16)]
        elif alphabet is None:
            b = rng.integers(0, 256, L, dtype=np.uint8)
        else:
            sym = np.frombuffer(alphabet, dtype=np.uint8)
            b = sym[rng.integers(0, len(sym), L, dtype=np.uint8)]
        pats.append(b.tobytes())
    return pats


def _plant(rng, text: np.ndarray, patterns: List[bytes], counts: Sequence[int]) -> List[np.ndarray]:
    n = text.size
    planted = []
    for pat, c in zip(patterns, counts):
        L = len(pat)
        if c <= 0 or L > n:
            planted.append(np.zeros(0, dtype=np.int64))
            continue
        pos = rng.integers(0, n - L + 1, int(c)).astype(np.int64)
        parr = np.frombuffer(pat, dtype=np.uint8)
        idx = (pos[:, None] + np.arange(L, dtype=np.int64)[None, :]).ravel()
        text[idx] = np.tile(parr, pos.size)
        planted.append(pos)
    return planted


def dna_single(seed: int = 0x5EED0000, n: int = 1 << 20, k: int = 8, m: int = 16,
               plants: int = 50) -> Workload:
    """Plain single search: uniform i.i.d. text over {A,C,G,T}, ``k`` patterns
    of length ``m`` over the same alphabet, each planted ``plants`` times."""
    rng = np.random.default_rng(seed)
    text = _draw_text_uniform(rng, n, b"ACGT")
    pats = _draw_patterns(rng, k, m, m, alphabet=b"ACGT")
    planted = _plant(rng, text, pats, [plants] * k)
    return Workload("dna_single", text, pats, planted,
                    dict(seed=seed, n=n, k=k, m=m, plants=plants))


def zipf_large(seed: int = 0x5EED0001, n: int = 1 << 30, k: int = 100, lmin: int = 4,
               lmax: int = 32, density: float = 1e-6) -> Workload:
    """Plain large scan: English-like Zipf letters with spaces; ``k`` patterns
    of lengths uniform in [lmin, lmax] from the same process, each planted
    round(density * n) times."""
    rng = np.random.default_rng(seed)
    lut = zipf_lut()
    text = _draw_text_lut(rng, n, lut)
    pats = _draw_patterns(rng, k, lmin, lmax, lut=lut)
    c = int(round(density * n))
    planted = _plant(rng, text, pats, [c] * k)
    return Workload("zipf_large", text, pats, planted,
                    dict(seed=seed, n=n, k=k, lmin=lmin, lmax=lmax, density=density))


def signature_set(seed: int = 0x5EED0002, n: int = 4 << 30, k: int = 10000, lmin: int = 8,
                  lmax: int = 64, plants: int = 1000) -> Workload:
    """Signature set: uniform random bytes; ``k`` random-byte patterns of
    lengths uniform in [lmin, lmax], each planted ``plants`` times."""
    rng = np.random.default_rng(seed)
    text = _draw_text_uniform(rng, n, None)
    pats = _draw_patterns(rng, k, lmin, lmax)
    planted = _plant(rng, text, pats, [plants] * k)
    return Workload("signature_set", text, pats, planted,
                    dict(seed=seed, n=n, k=k, lmin=lmin, lmax=lmax, plants=plants))


def random_small(seed: int, n: int, k: int, lmin: int, lmax: int,
                 alphabet: Optional[bytes] = b"ab", plants: int = 2) -> Workload:
    """Small fuzz case over a tiny alphabet (many natural, overlapping and
    duplicate matches)."""
    rng = np.random.default_rng(seed)
    text = _draw_text_uniform(rng, n, alphabet)
    pats = _draw_patterns(rng, k, lmin, lmax, alphabet=alphabet)
    planted = _plant(rng, text, pats, [plants] * k)
    return Workload("random_small", text, pats, planted,
                    dict(seed=seed, n=n, k=k, lmin=lmin, lmax=lmax, plants=plants))


@dataclasses.dataclass
class Batch:
    """Many independent search problems: texts[i] is searched with tables[table_of[i]]."""

    name: str
    texts: List[np.ndarray]
    tables: List[List[bytes]]
    table_of: List[int]
    params: dict

    @property
    def total_bytes(self) -> int:
        return int(sum(t.size for t in self.texts))


BATCH_ALPHABET = b"ABCDEFGHIJKLMNOPQRST"


def batched(seed: int = 0x5EED0003, n_items: int = 4096, min_len: int = 1 << 10,
            max_len: int = 1 << 24, k_min: int = 1, k_max: int = 256, lmin: int = 4,
            lmax: int = 48, alphabet: bytes = BATCH_ALPHABET, density: float = 1e-5) -> Batch:
    """Batched search: n_items texts with log-uniform lengths in [min_len,
    max_len] over `alphabet`, each with its own set of U{k_min..k_max}
    patterns of lengths U{lmin..lmax} over the same alphabet, each pattern
    planted round(density * len) times.  Draw order: all text lengths, then per
    item: text, pattern count, pattern lengths and bytes, plant offsets."""
    rng = np.random.default_rng(seed)
    lens = np.exp(rng.uniform(np.log(min_len), np.log(max_len), n_items)).astype(np.int64)
    texts, tables = [], []
    for n in lens:
        n = int(n)
        text = _draw_text_uniform(rng, n, alphabet)
        k = int(rng.integers(k_min, k_max + 1))
        pats = _draw_patterns(rng, k, lmin, lmax, alphabet=alphabet)
        _plant(rng, text, pats, [int(round(density * n))] * k)
        texts.append(text)
        tables.append(pats)
    return Batch("batched", texts, tables, list(range(n_items)),
                 dict(seed=seed, n_items=n_items, min_len=min_len, max_len=max_len, k_min=k_min,
                      k_max=k_max, lmin=lmin, lmax=lmax, density=density))


def serving_tables(seed: int = 0x5EED0004, n_tables: int = 64, k_max: int = 1024, lmin: int = 4,
                   lmax: int = 64) -> List[List[bytes]]:
    """Resident tables of the serving workload: table j holds U{1..k_max}
    uniform-byte patterns of lengths U{lmin..lmax}."""
    rng = np.random.default_rng(seed)
    tables = []
    for _ in range(n_tables):
        k = int(rng.integers(1, k_max + 1))
        tables.append(_draw_patterns(rng, k, lmin, lmax))
    return tables


def serving_texts(seed: int, n: int, tables: List[List[bytes]], min_len: int = 4 << 10,
                  max_len: int = 64 << 20, density: float = 1e-5):
    """n requests: (table id, text) with a uniform table choice, a log-uniform
    text length in [min_len, max_len] of uniform bytes, and every pattern of
    the table planted round(density * len) times."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        tid = int(rng.integers(0, len(tables)))
        L = int(np.exp(rng.uniform(np.log(min_len), np.log(max_len))))
        text = _draw_text_uniform(rng, L, None)
        _plant(rng, text, tables[tid], [int(round(density * L))] * len(tables[tid]))
        out.append((tid, text))
    return out


#: Full-size configurations: the 1 MiB DNA search, the 1 GiB Zipf scan and the
#: 4 GiB signature set.
FULL = {
    0: dict(fn=dna_single, seed=0x5EED0000),
    1: dict(fn=zipf_large, seed=0x5EED0001),
    2: dict(fn=signature_set, seed=0x5EED0002),
}


def make_config(i: int, n: Optional[int] = None, **overrides) -> Workload:
    """Workload of configuration ``i`` (0, 1 or 2), optionally with a smaller
    text.  For the Zipf scan the planting density stays 1e-6 per byte; for the
    signature set the plant count is scaled with the text length."""
    spec = FULL[i]
    kw = dict(seed=spec["seed"])
    if n is not None:
        kw["n"] = int(n)
        if i == 2 and "plants" not in overrides:
            kw["plants"] = max(1, int(round(1000 * n / (4 << 30))))
    kw.update(overrides)
    return spec["fn"](**kw)
