"""GPU parity of the sampled deferred scan (every pattern at least 7 bytes:
stage 1 tests every 4th position against the patterns' 4-byte grams at
offsets 0..3; tables built without a role filter, role_step = 1) against the
oracle, bit-exact, with the edge cases of the sampling: windows ending at
tile boundaries (found through the next tile's first word), grams repeated
at several offsets, the shortest allowed patterns, and texts ending at every
offset of a 16-byte chunk.  The edge cases also run with the builder's
choice, which for these small sets is the role filter with step 4."""

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
    dict(tile_bytes=1040, stages=3, warps=5),   # tile not a multiple of the warp rounds
    dict(filter=rk.RK_FILTER_FLAT, filter_log2_bits=10),  # a crowded bit set
    dict(filter=rk.RK_FILTER_REPLICATED),
    dict(base_log2=1),
]


def sample_step(patterns, **opts):
    t = rk.rk_build(list(patterns), **opts)
    try:
        return rk.rk_table_info(t)["sample_step"]
    finally:
        rk.rk_destroy(t)


@pytest.mark.parametrize("seed", range(18))
def test_fuzz_sampled(seed):
    rng = np.random.default_rng(9100 + seed)
    alpha = [b"ab", b"abc", b"ACGT", None][seed % 4]
    n = int(rng.integers(0, 40000))
    k = int(rng.integers(1, 60))
    lmin = int(rng.integers(7, 12))
    lmax = lmin + int(rng.integers(0, 60))
    w = random_small(seed + 900, n, k, lmin, lmax, alphabet=alpha, plants=4)
    opts = dict(OPTS[seed % len(OPTS)], role_step=1)
    assert sample_step(w.patterns, **opts) == 4
    expect = oracle.rabin_karp(w.text, w.patterns)
    mis = int(rng.integers(0, 16))
    assert_same(deferred_search(w.patterns, w.text, mis, **opts), expect,
                f"seed {seed} opts {opts}")


def test_repeated_grams_and_shortest_patterns():
    """Grams that start a pattern at several offsets (masks with more than
    one bit), patterns of exactly 7 bytes, and a periodic text full of
    overlapping matches."""
    text = np.frombuffer((b"abababab" * 700 + b"aaaaaaaaaaaa" * 300 + b"abcabcabcab" * 400),
                         dtype=np.uint8)
    pats = [b"abababa", b"bababab", b"aaaaaaa", b"aaaaaaaa", b"abcabca", b"cabcabcabca",
            b"ababababab", b"aaaaaaaaaaab", b"xyzxyzx"]
    assert sample_step(pats, role_step=1) == 4
    expect = oracle.bruteforce(text, pats)
    for opts in (dict(role_step=1), dict(tile_bytes=1024, stages=2, warps=2, role_step=1),
                 dict(), dict(tile_bytes=1024, stages=2, warps=2)):
        for mis in (0, 1, 2, 3, 9):
            assert_same(deferred_search(pats, text, mis, **opts), expect, f"{opts} mis {mis}")


@pytest.mark.parametrize("tail", range(0, 17))
def test_text_end_offsets(tail):
    """Windows that end with the text, for text ends at every offset of a
    chunk, found through the last sampled positions."""
    rng = np.random.default_rng(50 + tail)
    n = 8192 + tail
    text = rng.integers(0, 3, n, dtype=np.uint8) + ord("a")
    pats = [bytes(text[n - L:].tolist()) for L in (7, 8, 11, 19)]
    pats += [bytes(text[s:s + 9].tolist()) for s in (0, 1, 2, 3)]
    expect = oracle.bruteforce(text, pats)
    for opts in (dict(role_step=1), dict(tile_bytes=2048, stages=2, warps=2, role_step=1),
                 dict(), dict(tile_bytes=2048, stages=2, warps=2)):
        for mis in (0, 5, 12):
            assert_same(deferred_search(pats, text, mis, **opts), expect,
                        f"tail {tail} {opts} mis {mis}")


def test_sampling_off_same_list():
    """The same table without sampling (sample = 1) gives the same list, and
    the single-kernel scan of a sampled table is unchanged."""
    w = make_config(2, n=6 << 20)
    expect = oracle.rabin_karp(w.text, w.patterns)
    assert sample_step(w.patterns, sample=1) == 1
    assert_same(deferred_search(w.patterns, w.text, 3, sample=1), expect, "unsampled")
    assert_same(deferred_search(w.patterns, w.text, 3), expect, "sampled")
    assert_same(gpu_search(w.patterns, w.text, 3), expect, "single kernel")


def test_short_pattern_disables_sampling():
    assert sample_step([b"abcdefg", b"abcdef"], role_step=1) == 1
    assert sample_step([b"abcdefg", b"abcdefgh"], role_step=1) == 4
    assert sample_step([b"abcdefg"], filter=rk.RK_FILTER_NONE, role_step=1) == 1


def test_list_overflow_sampled():
    """Sampled stage 1 with every window a candidate: each sampled position
    offers the windows at all four of its gram's offsets, the list (n / 64 +
    4096 entries) fills, and the rest are verified inside the scan."""
    n = 1 << 20
    text = np.full(n, ord("a"), dtype=np.uint8)
    text[::1009] = ord("b")
    pats = [b"aaaaaaa", b"aaaaaaaa", b"aaaaaaaaaaa", b"aaaaaaaaaaaab", b"baaaaaa"]
    assert sample_step(pats, role_step=1) == 4
    expect = oracle.bruteforce(text, pats)
    assert expect[0].size > n // 64 + 4096
    for mis in (0, 3):
        for opts in (dict(role_step=1), dict()):
            assert_same(deferred_search(pats, text, mis, **opts), expect,
                        f"overflow mis {mis} {opts}")
