"""Pins of the oracle to facts outside it.

Each ``check_*`` raises AssertionError when the oracle (or a planted mutant of
it) disagrees with something the paper or mathematics fixes:

* the hand-worked examples in ``golden/hand_examples.txt``;
* Python's ``bytes.find`` and ``re`` overlapping search (library routines);
* brute force on exhaustive tiny inputs (two independent algorithms);
* closed forms of the hash: for base 256 the Rabin hash of s is the
  big-endian integer of s mod 2^61 - 1; for base 2 and short strings it is
  the paper's own shift-add hash (Section 3.1) with no reduction at all;
* number theory of the Mersenne prime p = 2^61 - 1: 2^61 = 1 (mod p) and
  Fermat's B^(p-1) = 1 (mod p);
* the rolling update agrees with per-window hashing and with the closed form.
"""

from __future__ import annotations

import itertools
import re

import numpy as np

import oracle
from golden_cases import load_hand_examples

P61 = (1 << 61) - 1


def check_hand_examples(mutant: int = 0) -> None:
    for case in load_hand_examples():
        for fn in (lambda t, p: oracle.bruteforce(t, p, mutant=mutant),
                   lambda t, p: oracle.rabin_karp(t, p, 256, mutant=mutant),
                   lambda t, p: oracle.rabin_karp(t, p, 2, mutant=mutant)):
            got = oracle.as_pairs(*fn(case.text, case.patterns))
            assert got == case.expect, (case.name, got, case.expect)


def _find_all(text: bytes, pat: bytes):
    out, i = [], text.find(pat)
    while i >= 0:
        out.append(i)
        i = text.find(pat, i + 1)
    return out


def check_bruteforce_vs_library(mutant: int = 0, trials: int = 60) -> None:
    rng = np.random.default_rng(1234)
    for t in range(trials):
        alpha = [b"ab", b"abc", b"ACGT", bytes(range(256))][t % 4]
        n = int(rng.integers(0, 300))
        text = bytes(rng.choice(list(alpha), n).astype(np.uint8)) if n else b""
        k = int(rng.integers(1, 8))
        pats = []
        for _ in range(k):
            m = int(rng.integers(1, 7))
            if n >= m and rng.random() < 0.5:  # a substring of the text
                s = int(rng.integers(0, n - m + 1))
                pats.append(text[s:s + m])
            else:
                pats.append(bytes(rng.choice(list(alpha), m).astype(np.uint8)))
        expect = [(p, x) for p, pat in enumerate(pats) for x in _find_all(text, pat)]
        expect_re = [(p, m.start()) for p, pat in enumerate(pats)
                     for m in re.finditer(b"(?=" + re.escape(pat) + b")", text)]
        assert expect == expect_re
        got = oracle.as_pairs(*oracle.bruteforce(text, pats, mutant=mutant))
        assert got == expect, (text, pats, got, expect)


def check_rk_vs_bruteforce_exhaustive(mutant: int = 0) -> None:
    """Every text of length <= 8 over {a, b} against all 30 patterns of
    length 1..4 over {a, b} at once, with base 256 and the paper's base 2."""
    pats = [bytes(p) for m in range(1, 5) for p in itertools.product(b"ab", repeat=m)]
    for n in range(0, 9):
        for tt in itertools.product(b"ab", repeat=n):
            text = bytes(tt)
            bf = oracle.as_pairs(*oracle.bruteforce(text, pats, mutant=mutant))
            for base in (256, 2):
                rk = oracle.as_pairs(*oracle.rabin_karp(text, pats, base, mutant=mutant))
                assert rk == bf, (text, base)


def check_rk_collisions(mutant: int = 0) -> None:
    """The paper's base-2 hash over bytes {0..3} collides constantly
    (e.g. 00 02 and 01 00 both hash to 2); verification must remove every
    false candidate, so the result must still equal brute force."""
    rng = np.random.default_rng(99)
    for _ in range(20):
        text = rng.integers(0, 4, 400, dtype=np.uint8)
        pats = [rng.integers(0, 4, int(rng.integers(2, 7)), dtype=np.uint8).tobytes()
                for _ in range(12)]
        bf = oracle.as_pairs(*oracle.bruteforce(text, pats, mutant=mutant))
        rk = oracle.as_pairs(*oracle.rabin_karp(text, pats, 2, mutant=mutant))
        assert rk == bf


def check_hash_closed_forms(mutant: int = 0) -> None:
    rng = np.random.default_rng(7)
    for L in list(range(0, 40)) + [64, 100, 333]:
        s = rng.integers(0, 256, L, dtype=np.uint8).tobytes()
        # base 256: the big-endian integer of the bytes, reduced mod p
        assert oracle.rk_hash(s, 256, mutant=mutant) == int.from_bytes(s, "big") % P61, L
        if L <= 53:
            # base 2, short strings: the paper's shift-add hash never reaches p
            h = 0
            for c in s:
                h = (h << 1) + c
            assert h < P61
            assert oracle.rk_hash(s, 2, mutant=mutant) == h, L


def check_hash_concatenation(mutant: int = 0) -> None:
    """h(s || t) = h(s) * B^|t| + h(t) mod p for any polynomial hash."""
    rng = np.random.default_rng(8)
    for _ in range(50):
        base = int(rng.integers(2, P61 - 1))
        s = rng.integers(0, 256, int(rng.integers(0, 30)), dtype=np.uint8).tobytes()
        t = rng.integers(0, 256, int(rng.integers(0, 30)), dtype=np.uint8).tobytes()
        lhs = oracle.rk_hash(s + t, base, mutant=mutant)
        rhs = (oracle.rk_hash(s, base, mutant=mutant) * pow(base, len(t), P61)
               + oracle.rk_hash(t, base, mutant=mutant)) % P61
        assert lhs == rhs


def check_modular_arithmetic(mutant: int = 0) -> None:
    edge = [0, 1, 2, 7, P61 - 2, P61 - 1, P61, P61 + 1, (1 << 62) + 5, (1 << 64) - 1]
    rng = np.random.default_rng(5)
    vals = edge + [int(x) for x in rng.integers(0, 1 << 63, 40, dtype=np.uint64)]
    for a in vals:
        for b in vals[:20]:
            assert oracle.mulmod(a, b, mutant=mutant) == (a * b) % P61, (a, b)
    assert oracle.powmod(2, 61, mutant=mutant) == 1
    for b in (2, 3, 256, 123456789):
        assert oracle.powmod(b, P61 - 1, mutant=mutant) == 1


def check_rolling(mutant: int = 0) -> None:
    rng = np.random.default_rng(11)
    for base in (256, 2, 1 << 13, 1000003, int(rng.integers(2, P61 - 1))):
        text = rng.integers(0, 256, 200, dtype=np.uint8)
        for L in (1, 2, 7, 8, 9, 31, 64, 200):
            hs = oracle.window_hashes(text, L, base, mutant=mutant)
            assert hs.size == text.size - L + 1
            direct = [oracle.rk_hash(text[x:x + L], base, mutant=mutant) for x in range(hs.size)]
            assert hs.tolist() == direct, (base, L)
            if base == 256:
                cf = [int.from_bytes(text[x:x + L].tobytes(), "big") % P61 for x in range(hs.size)]
                assert hs.tolist() == cf


ALL_CHECKS = [
    check_hand_examples,
    check_bruteforce_vs_library,
    check_rk_vs_bruteforce_exhaustive,
    check_rk_collisions,
    check_hash_closed_forms,
    check_hash_concatenation,
    check_modular_arithmetic,
    check_rolling,
]
