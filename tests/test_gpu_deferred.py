"""GPU parity of the deferred scan: survivors listed by the tile scan and
hashed, probed and verified by a second kernel (rk_scan_device_ws, and
rk_search_device given room for the list), against the oracle, bit-exact."""

import numpy as np
import pytest

import oracle
from workloads import make_config, random_small

pytestmark = pytest.mark.gpu

from gpu_util import assert_same, deferred_search, require_gpu  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


from paper_1810_01051_gb300 import rk  # noqa: E402

OPTS = [
    dict(),
    dict(filter=rk.RK_FILTER_FLAT, filter_log2_bits=12),
    dict(base_log2=1),
    dict(base_log2=13, filter=rk.RK_FILTER_FLAT),
    dict(tile_bytes=1024, stages=2, warps=2),
    dict(filter=rk.RK_FILTER_NONE),  # no prefilter: runs the in-scan path
]


@pytest.mark.parametrize("seed", range(16))
def test_fuzz_small(seed):
    rng = np.random.default_rng(7000 + seed)
    alpha = [b"ab", b"abc", b"ACGT", None][seed % 4]
    n = int(rng.integers(0, 30000))
    k = int(rng.integers(1, 40))
    lmin = int(rng.integers(1, 9))
    lmax = lmin + int(rng.integers(0, 70))
    w = random_small(seed + 500, n, k, lmin, lmax, alphabet=alpha, plants=3)
    expect = oracle.rabin_karp(w.text, w.patterns)
    opts = OPTS[seed % len(OPTS)]
    mis = int(rng.integers(0, 16))
    assert_same(deferred_search(w.patterns, w.text, mis, via_search=True, **opts), expect,
                f"search seed {seed} opts {opts}")
    assert_same(deferred_search(w.patterns, w.text, mis, via_search=False, **opts), expect,
                f"scan_ws seed {seed} opts {opts}")


@pytest.mark.parametrize("cfg,n", [(0, None), (1, 6 << 20), (2, 24 << 20)])
def test_configs_reduced(cfg, n):
    w = make_config(cfg, n=n)
    expect = oracle.rabin_karp(w.text, w.patterns)
    assert_same(deferred_search(w.patterns, w.text, 5), expect, f"config {cfg}")


def test_list_overflow_verified_in_scan():
    """Every window is a candidate: the list (n / 64 + 4096 entries) fills,
    and the rest are verified inside the scan."""
    n = 1 << 20
    text = np.full(n, ord("a"), dtype=np.uint8)
    text[::997] = ord("b")
    pats = [b"aaaa", b"aaaaa", b"aaaaaaa", b"aaaaaaaaaa", b"aaab"]
    expect = oracle.bruteforce(text, pats)
    assert expect[0].size > n // 64 + 4096
    assert_same(deferred_search(pats, text, 3), expect, "overflow")


@pytest.mark.parametrize("tail", [1, 5, 12, 15, 16, 17])
def test_text_end_reads(tail):
    """Windows that end at the text end, with the text ending just past a
    16-byte boundary: the second kernel reads them from global memory."""
    rng = np.random.default_rng(tail)
    n = 4096 + tail
    text = rng.integers(0, 4, n, dtype=np.uint8) + ord("A")
    pats = [bytes(text[n - L:].tolist()) for L in (1, 3, 8, 9, 16)] + [b"ABCA", b"CC"]
    expect = oracle.bruteforce(text, pats)
    for mis in (0, 7, 13):
        assert_same(deferred_search(pats, text, mis), expect, f"tail {tail} mis {mis}")
