"""The chunked oracle run (tests/oracle_pool.py) finds what the oracle finds
on the whole text: chunks far smaller than the text, matches straddling
every chunk boundary, a start offset, and the text's ragged end."""

import numpy as np

import oracle
from oracle_pool import oracle_items, oracle_matches
from workloads import make_config, random_small


def test_chunks_equal_whole_text():
    w = make_config(1, n=3 << 20)
    # plant patterns across the chunk boundaries (64 KiB chunks below)
    text = w.text.copy()
    for i, b in enumerate(range(1 << 16, text.size, 1 << 16)):
        p = np.frombuffer(w.patterns[i % len(w.patterns)], np.uint8)
        s = b - 1 - (i % (p.size - 1 if p.size > 1 else 1))
        text[s:s + p.size] = p
    expect = oracle.rabin_karp(text, w.patterns)
    got = oracle_matches(text, w.patterns, procs=3, chunk=1 << 16)
    assert np.array_equal(got[0], expect[0]) and np.array_equal(got[1], expect[1])


def test_start_offset_and_tiny_alphabet():
    w = random_small(5, 200_003, 20, 1, 9, alphabet=b"ab", plants=30)
    ids, offs = oracle.bruteforce(w.text, w.patterns)
    for start in (0, 1, 77_777):
        keep = offs >= start
        got = oracle_matches(w.text, w.patterns, start=start, procs=2, chunk=4093)
        assert np.array_equal(got[0], ids[keep]) and np.array_equal(got[1], offs[keep])


def test_items_equal_each_item_alone():
    """oracle_items: every item against its own set, long items in chunks
    (matches across the chunk boundaries), empty texts and empty sets."""
    items = []
    for i, n in enumerate((0, 5, 9000, 70_001, 30_000)):
        w = random_small(40 + i, n, 6 + i, 1, 12, alphabet=b"abc", plants=20)
        items.append((w.text, w.patterns))
    items.append((items[2][0], []))
    got = oracle_items(items, procs=3, chunk=4096)
    assert len(got) == len(items)
    for (text, pats), (gi, go) in zip(items, got):
        ei, eo = oracle.rabin_karp(text, pats) if pats else (np.zeros(0), np.zeros(0))
        assert np.array_equal(gi, ei) and np.array_equal(go, eo)
