"""The oracle against its pins (CPU only), and the pins against planted mistakes."""

import numpy as np
import pytest

import oracle
import oracle_pins
from golden_cases import load_hand_examples


@pytest.mark.parametrize("check", oracle_pins.ALL_CHECKS, ids=lambda f: f.__name__)
def test_oracle_pin(check):
    check(0)


def test_hand_examples_parse():
    cases = load_hand_examples()
    assert len(cases) >= 8
    names = {c.name for c in cases}
    assert {"abracadabra", "overlap", "duplicates", "last_byte"} <= names


# Each mutant plants one plausible mistake in the oracle's C source:
#   1 drops the last window (the sequential listing's loop bound),
#   2 reports hash equality without comparing bytes,
#   3 removes the outgoing byte with B^L instead of B^(L-1),
#   4 never compares a pattern's last byte,
#   5 hashes the bytes in reverse order,
#   6 reports one pattern id per hash value (duplicate patterns collapsed),
#   7 takes the rolling update's incoming byte one position early,
#   8 reduces a product mod 2^61 - 1 by one fold without the final subtract.
@pytest.mark.parametrize("mutant", [1, 2, 3, 4, 5, 6, 7, 8])
def test_pins_catch_mutant(mutant):
    failed = []
    for check in oracle_pins.ALL_CHECKS:
        try:
            check(mutant)
        except AssertionError:
            failed.append(check.__name__)
    assert failed, f"mutant {mutant} passed every pin"


def test_rk_matches_bruteforce_on_workload_slices():
    from workloads import make_config
    for cfg in (0, 1, 2):
        w = make_config(cfg, n=1 << 14, **({"k": 40} if cfg == 2 else {}))
        bf = oracle.bruteforce(w.text, w.patterns)
        rk = oracle.rabin_karp(w.text, w.patterns)
        assert np.array_equal(bf[0], rk[0]) and np.array_equal(bf[1], rk[1])


def test_result_sorted_and_verified():
    from workloads import random_small
    w = random_small(3, 3000, 20, 1, 6, alphabet=b"abc")
    pid, off = oracle.rabin_karp(w.text, w.patterns)
    keys = list(zip(pid.tolist(), off.tolist()))
    assert keys == sorted(set(keys))
    t = w.text.tobytes()
    for p, x in keys:
        assert t[x:x + len(w.patterns[p])] == w.patterns[p]
