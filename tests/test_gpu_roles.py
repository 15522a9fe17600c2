"""GPU parity of the role filter (stage 1 looks up only every 2nd or 4th
position's 4-byte gram; its roles, with those of the gram 4 bytes on, decide
which windows survive; at step 4 a side set covers patterns under 7 bytes)
against the oracle, bit-exact, through the scan that verifies its survivors
itself and through the deferred scan, with its edge cases: 4-byte patterns
at odd offsets (found through a gram that holds one text byte past the
pattern, or the side set), windows at tile boundaries and at the text end
(found through the first sampled position of the next chunk or tile), the
last chunk of a warp's round (whose second grams belong to another warp),
every window a candidate (the per-lane path when the warp's queue is full),
and the paper's base-2 hash (hash collisions)."""

import numpy as np
import pytest

import oracle
from workloads import make_config, random_small

pytestmark = pytest.mark.gpu

from gpu_util import assert_same, deferred_search, gpu_search, require_gpu  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


from paper_1810_01051_gb300 import rk  # noqa: E402

OPTS = [
    dict(),
    dict(tile_bytes=1024, stages=2, warps=2),   # many tiles: boundaries everywhere
    dict(tile_bytes=1040, stages=3, warps=5),   # a tile not a multiple of the warp rounds
    dict(warps=16, tile_bytes=4096),
    dict(warps=31, stages=3),
    dict(base_log2=1),                          # the paper's hash: collisions to verify
]


def role_step(patterns, **opts):
    t = rk.rk_build(list(patterns), **opts)
    try:
        return rk.rk_table_info(t)["role_step"]
    finally:
        rk.rk_destroy(t)


def both_paths(patterns, text, mis, what, **opts):
    expect = oracle.rabin_karp(text, patterns)
    assert_same(gpu_search(patterns, text, mis, **opts), expect, f"single kernel {what}")
    assert_same(deferred_search(patterns, text, mis, **opts), expect, f"deferred {what}")


@pytest.mark.parametrize("seed", range(24))
def test_fuzz_roles(seed):
    rng = np.random.default_rng(7700 + seed)
    alpha = [b"ab", b"abc", b"ACGT", b"ABCDEFGHIJKLMNOPQRST", None][seed % 5]
    n = int(rng.integers(0, 60000))
    k = int(rng.integers(1, 60))
    lmin = int(rng.integers(4, 10))
    lmax = lmin + int(rng.integers(0, 40))
    w = random_small(seed + 700, n, k, lmin, lmax, alphabet=alpha, plants=5)
    opts = dict(OPTS[seed % len(OPTS)])
    forced = [0, 2, 4][seed % 3]  # the builder's choice, step 2, step 4 (with a side set
    if forced:                    # when some pattern is shorter than 7 bytes)
        opts["role_step"] = forced
    step = role_step(w.patterns, **opts)
    assert step in ((2, 4) if not forced else (forced, 0)), (step, forced)
    both_paths(w.patterns, w.text, int(rng.integers(0, 16)), f"seed {seed} {opts}", **opts)


@pytest.mark.parametrize("forced", [2, 4])
def test_forced_step(forced):
    """A set of 7+ byte patterns under either step; step 2 on it takes no
    4-byte wildcard grams."""
    w = random_small(31, 50000, 40, 7, 30, alphabet=b"abc", plants=6)
    assert role_step(w.patterns, role_step=forced) == forced
    for opts in (dict(role_step=forced), dict(role_step=forced, tile_bytes=1024, warps=2)):
        both_paths(w.patterns, w.text, 7, f"step {forced} {opts}", **opts)


def test_four_byte_patterns_at_every_offset():
    """4-byte patterns planted at every offset modulo 16 and across 1 KiB tile
    boundaries: odd offsets are found only through the gram P[1..4) plus the
    next text byte."""
    rng = np.random.default_rng(5)
    n = 20000
    text = rng.integers(0, 4, n, dtype=np.uint8) + ord("a")
    pats = [b"wxyz", b"zzzz", b"wxyw", b"abcdefgh", b"xyzwa"]
    for i, x in enumerate(list(range(1, 64)) + [1023, 1024, 1025, 2045, 2046, 2047, 4095,
                                                n - 4, n - 5]):
        p = pats[i % 3]
        text[x:x + 4] = np.frombuffer(p, dtype=np.uint8)
    assert role_step(pats) == 2 and role_step(pats, role_step=4) == 4
    for rs in (4, 2):  # the side set, or the wildcard grams at step 2
        for opts in (dict(), dict(tile_bytes=1024, stages=2, warps=2),
                     dict(tile_bytes=1040, warps=3)):
            for mis in (0, 1, 6):
                both_paths(pats, text, mis, f"{opts} mis {mis} step {rs}", role_step=rs, **opts)


@pytest.mark.parametrize("tail", range(0, 17))
def test_text_end_offsets(tail):
    """Windows that end with the text, for text ends at every offset of a
    chunk; 4-byte and longer patterns."""
    rng = np.random.default_rng(80 + tail)
    n = 8192 + tail
    text = rng.integers(0, 3, n, dtype=np.uint8) + ord("a")
    pats = [bytes(text[n - L:].tolist()) for L in (4, 5, 7, 8, 11, 19)]
    pats += [bytes(text[s:s + 9].tolist()) for s in (0, 1, 2, 3)]
    for opts in (dict(), dict(tile_bytes=2048, stages=2, warps=2)):
        for mis in (0, 5, 12):
            both_paths(pats, text, mis, f"tail {tail} {opts} mis {mis}", **opts)


def test_side_set_on_zipf_text():
    """A set shaped like the full Zipf one (two 4-byte patterns) under
    step 4 with a side set over 6 MiB of Zipf text: the side set's windows
    found through the positions 2 mod 4, and a misaligned text."""
    full = make_config(1, n=6 << 20)
    rng = np.random.default_rng(12)
    # a set shaped like the full one: lengths 4..32 with two 4-byte patterns
    pats = [bytes(full.text[s:s + L].tolist())
            for s, L in zip(rng.integers(0, full.n - 40, 60), [4, 4, 5, 5, 6, 6] + [7 + i % 26 for i in range(54)])]
    assert role_step(pats, role_step=4) == 4
    expect = oracle.rabin_karp(full.text, pats)
    for opts in (dict(role_step=4), dict(role_step=4, warps=12),
                 dict(role_step=4, tile_bytes=4096, warps=3)):
        for mis in (0, 7):
            assert_same(deferred_search(pats, full.text, mis, **opts), expect, f"{opts} {mis}")
            assert_same(gpu_search(pats, full.text, mis, **opts), expect, f"{opts} {mis}")


def test_every_window_a_candidate():
    """A text of one letter: every sampled position survives, more than a
    warp's queue takes in one round, and every window matches."""
    n = 1 << 18
    text = np.full(n, ord("a"), dtype=np.uint8)
    text[::997] = ord("b")
    for pats in ([b"aaaa", b"aaaaa", b"aaaaaaaaa", b"baaa"],
                 [b"aaaaaaa", b"aaaaaaaa", b"aaaaaaaaaaaa", b"baaaaaa"]):
        for opts in (dict(), dict(tile_bytes=1024, warps=2), dict(role_step=2)):
            both_paths(pats, text, 3, f"{pats} {opts}", **opts)


def test_workload_sets():
    """A Zipf set (step 2; step 4 with a side set for its patterns under 7
    bytes when asked for) and the DNA set (step 4) at reduced sizes: the role
    filters, the prefix filter (role_step = 1) and the oracle agree."""
    for cfg, n, step in ((1, 6 << 20, 2), (0, 1 << 20, 4)):
        w = make_config(cfg, n=n)
        assert role_step(w.patterns) == step
        expect = oracle.rabin_karp(w.text, w.patterns)
        for opts in (dict(), dict(role_step=4), dict(role_step=1)):
            assert_same(deferred_search(w.patterns, w.text, 1, **opts), expect, f"cfg {cfg} {opts}")
            assert_same(gpu_search(w.patterns, w.text, 2, **opts), expect, f"cfg {cfg} {opts}")
