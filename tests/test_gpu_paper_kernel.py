"""The paper's own one-thread-per-offset GPU matcher (kept for comparison)
against the oracle, including the long patterns of the paper's Table 3
(m = 25 .. 800) on DNA-like text, and the long-pattern path of the tiled
scan on the same inputs."""

import numpy as np
import pytest

import oracle
from workloads import dna_single

pytestmark = pytest.mark.gpu

from gpu_util import assert_same, gpu_search, require_gpu, to_device  # noqa: E402
from paper_1810_01051_gb300 import rk  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def paper_offsets(text: np.ndarray, pat: bytes, tpb: int = 0, misalign: int = 0) -> np.ndarray:
    import torch
    d = to_device(text, misalign)
    res = torch.full((max(text.size, 1),), 7, dtype=torch.uint8, device="cuda")
    rk.rk_paper_search_device(d, text.size, pat, res, tpb)
    torch.cuda.synchronize()
    r = res.cpu().numpy()[:text.size]
    assert set(np.unique(r).tolist()) <= {0, 1}
    return np.flatnonzero(r).astype(np.uint64)


@pytest.mark.parametrize("tpb", [32, 256, 1024])
def test_paper_kernel_matches_oracle(tpb):
    rng = np.random.default_rng(tpb)
    for m in (1, 2, 7, 16, 63, 64, 65, 300):
        text = rng.integers(0, 3, 20000, dtype=np.uint8)
        pat = rng.integers(0, 3, m, dtype=np.uint8).tobytes()
        if m < 100:
            s = int(rng.integers(0, text.size - m))
            text[s:s + m] = np.frombuffer(pat, np.uint8)
        ids, offs = oracle.bruteforce(text, [pat])
        assert np.array_equal(paper_offsets(text, pat, tpb, misalign=m % 5), offs), m


def test_paper_kernel_last_window_and_edges():
    text = np.frombuffer(b"xxabcab", np.uint8)
    assert paper_offsets(text, b"ab").tolist() == [2, 5]  # x = n - m counts
    assert paper_offsets(text, b"xxabcabz").size == 0   # longer than the text
    assert paper_offsets(np.zeros(0, np.uint8), b"a").size == 0


@pytest.mark.parametrize("m", [25, 50, 100, 200, 800])
def test_table3_pattern_lengths_both_kernels(m):
    """Table 3's pattern lengths on 2 MB of DNA-like text (its file size is not
    stated; about 2 MB by inference), one planted pattern set."""
    w = dna_single(seed=0x5EED0100 + m, n=2 << 20, k=4, m=m, plants=20)
    expect = oracle.rabin_karp(w.text, w.patterns)
    assert_same(gpu_search(w.patterns, w.text, misalign=1), expect, f"tiled m={m}")
    for p, pat in enumerate(w.patterns):
        assert np.array_equal(paper_offsets(w.text, pat), expect[1][expect[0] == p])
