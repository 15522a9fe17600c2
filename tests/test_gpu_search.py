"""GPU parity: the CUDA path through the C ABI against the oracle, element by
element (integer work, so bit-exact: the identical sorted (id, offset) list)."""

import numpy as np
import pytest

import oracle
from golden_cases import load_hand_examples
from workloads import make_config, random_small

pytestmark = pytest.mark.gpu

from gpu_util import assert_same, gpu_search, keys_to_pairs, require_gpu, search_table, to_device  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


from paper_1810_01051_gb300 import rk  # noqa: E402

# Table options exercised: default, each prefilter layout, no prefilter (every
# window hashed at every length), the paper's base-2 hash (constant
# collisions), a non-byte base, small tiles (many tiles, halo crossings).
OPTS = [
    dict(),
    dict(filter=rk.RK_FILTER_REPLICATED),
    dict(filter=rk.RK_FILTER_FLAT, filter_log2_bits=12),
    dict(filter=rk.RK_FILTER_NONE),
    dict(base_log2=1),
    dict(base_log2=13, filter=rk.RK_FILTER_FLAT),
    dict(tile_bytes=1024, stages=2, warps=2),
    dict(tile_bytes=1040, stages=4, warps=5, filter=rk.RK_FILTER_REPLICATED, filter_log2_bits=10),
]


@pytest.mark.parametrize("opts", OPTS, ids=lambda o: ",".join(f"{k}={v}" for k, v in o.items()) or "default")
def test_hand_examples(opts):
    for case in load_hand_examples():
        text = np.frombuffer(case.text, dtype=np.uint8)
        for mis in (0, 3):
            ids, offs = gpu_search(case.patterns, text, misalign=mis, **opts)
            assert list(zip(ids.tolist(), offs.tolist())) == case.expect, (case.name, mis)


@pytest.mark.parametrize("seed", range(24))
def test_fuzz_small(seed):
    rng = np.random.default_rng(1000 + seed)
    alpha = [b"ab", b"abc", b"ACGT", None][seed % 4]
    n = int(rng.integers(0, 20000))
    k = int(rng.integers(1, 40))
    lmin = int(rng.integers(1, 9))
    lmax = lmin + int(rng.integers(0, 70))
    w = random_small(seed, n, k, lmin, lmax, alphabet=alpha, plants=3)
    opts = OPTS[seed % len(OPTS)]
    expect = oracle.rabin_karp(w.text, w.patterns)
    got = gpu_search(w.patterns, w.text, misalign=int(rng.integers(0, 16)), **opts)
    assert_same(got, expect, f"seed {seed} opts {opts}")


@pytest.mark.parametrize("cfg", [0, 1, 2])
@pytest.mark.parametrize("opts", [dict(), dict(tile_bytes=4096)], ids=["default", "tile4k"])
def test_configs_reduced(cfg, opts):
    """Each configuration at about 1 MiB plus a ragged tail: 30+ tiles."""
    n = (1 << 20) + 12345
    w = make_config(cfg, n=n)
    expect = oracle.rabin_karp(w.text, w.patterns)
    got = gpu_search(w.patterns, w.text, misalign=5, **opts)
    assert_same(got, expect, f"config {cfg}")
    assert got[0].size > 0


def test_config0_full_size():
    """The 1 MiB DNA search at full size, whole list against brute force."""
    w = make_config(0)
    expect = oracle.bruteforce(w.text, w.patterns)
    got = gpu_search(w.patterns, w.text)
    assert_same(got, expect, "config 0")
    assert got[0].size >= 8 * 40  # 50 plants per pattern, few destroyed


@pytest.mark.parametrize("base_log2", [1, 8, 13, 60])
def test_window_hashes(base_log2):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(base_log2)
    text = rng.integers(0, 256, 5000, dtype=np.uint8)
    d = to_device(text, 7)
    for L in (1, 2, 7, 8, 9, 33, 64, 100, 4096):
        out = torch.zeros(text.size - L + 1, dtype=torch.int64, device="cuda")
        rk.rk_window_hashes_device(d, text.size, L, base_log2, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy().view(np.uint64)
        expect = oracle.window_hashes(text, L, 1 << base_log2)
        assert np.array_equal(got, expect), (base_log2, L)


def test_edge_cases():
    # empty text; pattern longer than text; q = 1, 2, 3 prefixes; zero bytes
    # (prefix key 0); whole-text match; longest pattern allowed
    assert gpu_search([b"a"], np.zeros(0, np.uint8))[0].size == 0
    assert gpu_search([b"abcdef"], np.frombuffer(b"abc", np.uint8))[0].size == 0
    rng = np.random.default_rng(5)
    for pats in ([b"a", b"ab"], [b"ab", b"ba", b"abc"], [b"abc", b"bca", b"abcabc"],
                 [b"\0\0\0\0", b"\0\0\0\0\0", b"\0"]):
        for alpha in (b"abc", bytes([0, 1])):
            text = np.frombuffer(bytes(rng.choice(list(alpha), 3000).astype(np.uint8)), np.uint8)
            assert_same(gpu_search(pats, text), oracle.bruteforce(text, pats), str(pats))
    text = rng.integers(0, 256, 20000, dtype=np.uint8)
    long_pat = text[7000:7000 + rk.RK_MAX_PATTERN_LEN].tobytes()
    pats = [long_pat, text[:100].tobytes(), text[-50:].tobytes()]
    assert_same(gpu_search(pats, text), oracle.bruteforce(text, pats), "long")
    whole = text[:300]
    assert_same(gpu_search([whole.tobytes()], whole), (np.array([0], np.uint32), np.array([0], np.uint64)))


def test_empty_table_and_duplicates():
    text = np.frombuffer(b"abababab", np.uint8)
    assert gpu_search([], text)[0].size == 0
    got = gpu_search([b"aba", b"aba", b"b"], text)
    assert_same(got, oracle.bruteforce(text, [b"aba", b"aba", b"b"]), "dups")


def test_capacity_overflow_reports_count():
    text = np.frombuffer(b"a" * 10000, np.uint8)
    table = rk.rk_build([b"a", b"aa"])
    try:
        d = to_device(text)
        keys, count, status = search_table(table, d, text.size, 100)
        assert status == rk.RK_OK and count == 10000 + 9999
        keys, count, status = search_table(table, d, text.size, count)
        ids, offs = keys_to_pairs(keys[:count])
        assert_same((ids, offs), oracle.bruteforce(text, [b"a", b"aa"]), "after retry")
    finally:
        rk.rk_destroy(table)


def test_host_path_matches_device_path():
    w = make_config(1, n=(3 << 20) + 77)
    table = rk.rk_build(w.patterns)
    try:
        expect = oracle.rabin_karp(w.text, w.patterns)
        out = np.empty(expect[0].size + 10, dtype=np.uint64)
        rc, cnt = rk.rk_search(table, w.text, w.text.size, out, out.size)
        assert rc == rk.RK_OK and cnt == expect[0].size
        assert_same(rk.unpack_keys(out[:cnt]), expect, "host path")
        small = np.empty(3, dtype=np.uint64)
        rc, cnt2 = rk.rk_search(table, w.text, w.text.size, small, 3)
        assert rc == rk.RK_ECAPACITY and cnt2 == cnt
    finally:
        rk.rk_destroy(table)


def test_scan_then_sort_equals_search():
    torch = pytest.importorskip("torch")
    w = make_config(2, n=1 << 20, k=500)
    table = rk.rk_build(w.patterns)
    try:
        d = to_device(w.text)
        cap = 1 << 16
        keys = torch.empty(cap, dtype=torch.int64, device="cuda")
        info = torch.zeros(2, dtype=torch.int64, device="cuda")
        rk.rk_scan_device(table, d, w.text.size, keys, cap, info)
        torch.cuda.synchronize()
        count = int(info[0])
        unsorted = keys[:count].cpu().numpy().view(np.uint64).copy()
        wsb = rk.rk_workspace_bytes(table, cap)
        ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
        rk.rk_sort_device(table, w.text.size, keys, cap, info, ws, wsb)
        torch.cuda.synchronize()
        srt = keys[:count].cpu().numpy().view(np.uint64)
        assert np.array_equal(np.sort(unsorted), srt)
        assert_same(rk.unpack_keys(srt), oracle.rabin_karp(w.text, w.patterns), "scan+sort")
    finally:
        rk.rk_destroy(table)


@pytest.mark.parametrize("n,k,lmin,lmax", [(1 << 20, 12, 2, 6), ((1 << 22) + 5, 300, 8, 12)],
                         ids=["4-passes", "5-passes"])
def test_sort_paths_agree(n, k, lmin, lmax):
    """The cooperative single-launch sort (small capacity) and the per-pass
    look-back kernels (capacity beyond 32 tiles per resident CTA) give the
    oracle's list on the same keys, with odd and even pass counts and with
    several tiles per CTA (more than two tiles per SM of matches)."""
    torch = pytest.importorskip("torch")
    w = random_small(77 + k, n, k, lmin, lmax, alphabet=b"ab", plants=0)
    expect = oracle.rabin_karp(w.text, w.patterns)
    m = int(expect[0].size)
    assert m > 2048 * 2 * 152, m  # more tiles than resident CTAs of the fused sort
    table = rk.rk_build(w.patterns)
    try:
        d = to_device(w.text)
        for cap, fused in ((m + 100, True), (1 << 24, True), (1 << 25, False)):
            launches = rk.rk_sort_launches(table, n, cap)
            assert (launches == 1) == fused, (cap, launches)
            keys, count, status = search_table(table, d, n, cap)
            assert status == rk.RK_OK and count == m
            assert_same(keys_to_pairs(keys[:count]), expect, f"cap {cap}")
    finally:
        rk.rk_destroy(table)


def test_matcher_wrapper():
    """The convenience wrapper (deferred scan through its workspace) gives the
    oracle's list, grows a one-key output until it fits, and handles an
    empty text."""
    torch = pytest.importorskip("torch")
    from paper_1810_01051_gb300.matcher import Matcher
    w = make_config(1, n=3 << 20)
    expect = oracle.rabin_karp(w.text, w.patterns)
    m = Matcher(w.patterns)
    try:
        d = to_device(w.text)
        for cap in (None, 1):
            keys = m.search(d, capacity=cap)
            assert_same(keys_to_pairs(keys), expect, f"capacity {cap}")
        assert m.search(torch.zeros(0, dtype=torch.uint8, device="cuda")).numel() == 0
    finally:
        m.close()


def test_c_example_program(tmp_path):
    """The C example (tests/c_api_example.c) built against the header and
    library prints the oracle's list."""
    import subprocess
    from test_abi import compile_c_example
    exe = compile_c_example(tmp_path)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    text = np.frombuffer(b"xxGATTACAxACGTxxGATTACA", np.uint8)
    ids, offs = oracle.bruteforce(text, [b"GATTACA", b"ACGT"])
    expect = [f"{i} {o}" for i, o in zip(ids.tolist(), offs.tolist())]
    assert expect == ["0 2", "0 16", "1 10"]
    assert r.stdout.split("\n")[:-1] == expect
