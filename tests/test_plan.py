"""The table builder's host logic through rk_plan (CPU only: rk_plan makes
no CUDA call).  The pattern statistics are recounted here in Python; the
launch shape is checked against the builder's rules: the stage-1 bit set's
layout and size, sampling, the halo, and the shrinking of stages and tiles
until the CTA's shared memory fits."""

import ctypes

import numpy as np
import pytest

from paper_1810_01051_gb300 import build_lib, rk
from workloads import make_config, random_small

OPTIN = rk.GB300_SMEM_OPTIN


@pytest.fixture(scope="module", autouse=True)
def lib():
    build_lib.build()
    return rk.load()


def ceil_log2(x):
    return max(0, int(x - 1).bit_length())


def stats(patterns):
    lens = [len(p) for p in patterns]
    q = min(4, min(lens))
    return dict(n_patterns=len(patterns), min_len=min(lens), max_len=max(lens),
                n_lengths=len(set(lens)), gram_len=q, n_grams=len({p[:q] for p in patterns}),
                halo_bytes=(max(max(lens) - 1, 1) + 15) // 16 * 16)


def sampled_grams(patterns):
    return len({p[j:j + 4] for p in patterns for j in range(4)})


def pattern_sets():
    z = make_config(1, n=1 << 16).patterns           # 100 Zipf patterns, 4..32 bytes
    s = make_config(2, n=1 << 16, k=2000).patterns   # 2000 random-byte patterns, 8..64
    d = make_config(0, n=1 << 12).patterns           # 8 DNA patterns of 16 bytes
    r = random_small(4, 10, 30, 1, 3, alphabet=b"abc").patterns
    longp = [bytes([i % 251]) * 4096 for i in range(3)] + [b"abcdefgh"]
    return dict(zipf=z, signature=s, dna=d, short=r, long=longp)


@pytest.mark.parametrize("name", ["zipf", "signature", "dna", "short", "long"])
def test_pattern_statistics(name):
    pats = pattern_sets()[name]
    info = rk.rk_plan(pats)
    for key, val in stats(pats).items():
        assert info[key] == val, key
    assert info["base_log2"] == 8
    if info["role_step"]:
        # role filter: 16 stage-1 warps, 6 survivor warps, 48 KiB tiles, two stages
        assert (info["warps"], info["survivor_warps"]) == (16, 6)
        assert info["tile_bytes"] <= 49152 and info["stages"] == 2
    else:
        assert info["warps"] == 24 and info["survivor_warps"] == 0
    assert info["sm_count"] == 0 and info["device"] == 0xFFFFFFFF


@pytest.mark.parametrize("name", ["zipf", "signature", "dna", "short", "long"])
def test_filter_layout_and_size(name):
    pats = pattern_sets()[name]
    info = rk.rk_plan(pats)
    D = info["n_grams"]
    if D <= 256:
        # replicated into the 32 banks: 2^14 bits per copy
        assert info["filter"] == rk.RK_FILTER_REPLICATED
        assert info["filter_log2_bits"] == 14
        assert info["filter_smem_bytes"] == (1 << 14) // 8 * 32
    else:
        # flat: about 32 bits per prefix, 2^15..2^20 bits
        assert info["filter"] == rk.RK_FILTER_FLAT
        assert info["filter_log2_bits"] == min(20, max(15, ceil_log2(32 * D)))
        assert info["filter_smem_bytes"] == (1 << info["filter_log2_bits"]) // 8
    none = rk.rk_plan(pats, filter=rk.RK_FILTER_NONE)
    assert none["filter"] == rk.RK_FILTER_NONE and none["filter_log2_bits"] == 0
    assert none["filter_smem_bytes"] == 0 and none["sample_step"] == 1
    flat = rk.rk_plan(pats, filter=rk.RK_FILTER_FLAT, filter_log2_bits=12)
    assert flat["filter"] == rk.RK_FILTER_FLAT and flat["filter_smem_bytes"] == (1 << 12) // 8
    rep = rk.rk_plan(pats, filter=rk.RK_FILTER_REPLICATED, filter_log2_bits=11)
    assert rep["filter_smem_bytes"] == (1 << 11) // 8 * 32


def role_keys(patterns, step):
    """Role-filter keys for sampling step `step` counted in Python: per
    pattern, the gram at each offset j < step (and the one 4 bytes on when the
    pattern has j + 8 bytes), or for a 4-byte pattern at j = 1 the 256 grams
    P[1..4) + any byte.  Step 4 over patterns shorter than 7 bytes gives those
    only their grams at offsets 0 and 1, in the main set and in a side set
    of at most 1024 grams.  None when the step does not apply."""
    lens = [len(p) for p in patterns]
    if min(lens) < 4 or sum(L == 4 for L in lens) > 64:
        return None
    side = step == 4 and min(lens) < 7
    n = ns = 0
    for L in lens:
        if side and L < 7:
            k = 2 if L >= 5 else 257
            n += k
            ns += k
            continue
        for j in range(step):
            if j + 4 <= L:
                n += 2 if L >= j + 8 else 1
            else:
                n += 256
    if ns > 1024:
        return None
    return n


def role_rule(patterns, role_step=0, filter=rk.RK_FILTER_AUTO):
    """(step, log2 bits) of the role filter the builder should choose: its
    own choice only with the prefilter's (RK_FILTER_AUTO)."""
    if min(len(p) for p in patterns) < 4 or filter == rk.RK_FILTER_NONE:
        return 0, 0
    if role_step == 0 and filter != rk.RK_FILTER_AUTO:
        return 0, 0
    for step in (4, 2):
        if role_step not in (0, step):
            continue
        if role_step == 0 and step == 4 and min(len(p) for p in patterns) < 7:
            continue  # the builder's own choice takes no side set
        nk = role_keys(patterns, step)
        if nk is None:
            continue
        bits = min(19, max(15, ceil_log2(nk * 512)))
        if nk * 16 <= 1 << bits:
            return step, bits
    return 0, 0


@pytest.mark.parametrize("name", ["zipf", "signature", "dna", "short", "long"])
def test_sampling_rule(name):
    pats = pattern_sets()[name]
    info = rk.rk_plan(pats)
    step, bits = role_rule(pats)
    assert (info["role_step"], info["role_filter_log2_bits"]) == (step, bits)
    want_side = 0  # only a forced step 4 takes a side set
    assert info["role_side_log2_bits"] == want_side
    none = rk.rk_plan(pats, role_step=1)
    assert none["role_step"] == 0 and none["role_filter_log2_bits"] == 0
    for forced in (2, 4):
        want = role_rule(pats, forced)
        got = rk.rk_plan(pats, role_step=forced)
        assert (got["role_step"], got["role_filter_log2_bits"]) == want
    for filt in (rk.RK_FILTER_FLAT, rk.RK_FILTER_REPLICATED):
        assert rk.rk_plan(pats, filter=filt)["role_step"] == 0
        got = rk.rk_plan(pats, filter=filt, role_step=4)
        assert (got["role_step"], got["role_filter_log2_bits"]) == role_rule(pats, 4, filt)
    for opts, has_role in ((dict(), step != 0), (dict(role_step=1), False)):
        info = rk.rk_plan(pats, **opts)
        if min(len(p) for p in pats) >= 7 and not has_role:
            # every window holds one position = 0 mod 4 within its first 7 bytes
            assert info["sample_step"] == 4
            G = sampled_grams(pats)
            want = 14 if G <= 256 else min(19, max(15, ceil_log2(32 * G)))
            assert info["sample_filter_log2_bits"] == want
            off = rk.rk_plan(pats, sample=1, **opts)
            assert off["sample_step"] == 1 and off["sample_filter_log2_bits"] == 0
        else:
            # a role filter replaces the sampled grams' structures
            assert info["sample_step"] == 1 and info["sample_filter_log2_bits"] == 0


def test_role_filter_choice():
    """The workloads' sets take the filter the rule predicts: a Zipf set (a
    few patterns under 7 bytes) step 2 (step 4 with a side set when asked
    for), the DNA set step 4, 2,000
    signature patterns (about 16,000 role keys) step 4, the full 10,000 (about
    79,000) none; patterns below 4 bytes, RK_FILTER_NONE, or more than 64
    four-byte patterns rule it out."""
    sets = pattern_sets()
    z = rk.rk_plan(sets["zipf"])
    assert (z["role_step"], z["role_filter_log2_bits"], z["role_side_log2_bits"]) == (2, 19, 0)
    z4 = rk.rk_plan(sets["zipf"], role_step=4)
    assert (z4["role_step"], z4["role_side_log2_bits"]) == (4, 14)
    assert rk.rk_plan(sets["dna"])["role_step"] == 4
    assert rk.rk_plan(sets["signature"])["role_step"] == 4
    big = make_config(2, n=1 << 16, k=10000).patterns
    assert rk.rk_plan(big)["role_step"] == 0
    assert rk.rk_plan(sets["short"])["role_step"] == 0
    assert rk.rk_plan(sets["zipf"], filter=rk.RK_FILTER_NONE)["role_step"] == 0
    many4 = [bytes([65 + i % 26, 66 + i // 26, 67, 68]) for i in range(65)]
    assert rk.rk_plan(many4)["role_step"] == 0
    assert rk.rk_plan(many4[:64])["role_step"] == 2
    assert rk.rk_plan(many4[:3], role_step=4)["role_side_log2_bits"] == 14
    with pytest.raises(rk.RkError):
        rk.rk_plan(sets["zipf"], role_step=3)


def test_shared_memory_fits_every_request():
    pats = pattern_sets()
    rng = np.random.default_rng(3)
    for _ in range(60):
        name = ["zipf", "signature", "dna", "short", "long"][int(rng.integers(0, 5))]
        opts = dict(warps=int(rng.integers(1, 32)), stages=int(rng.integers(2, 9)),
                    tile_bytes=16 * int(rng.integers(64, 4097)),
                    ctas_per_sm=int(rng.choice([1, 2, 4])))
        optin = int(rng.choice([OPTIN, 101376, 166912, 65536]))
        try:
            info = rk.rk_plan(pats[name], smem_optin=optin, **opts)
        except rk.RkError as e:
            assert e.code == rk.RK_EINVAL
            continue
        limit = optin // opts["ctas_per_sm"] - 1024
        assert info["smem_bytes"] <= limit, (name, opts, optin)
        assert info["tile_bytes"] % 16 == 0 and info["tile_bytes"] >= 1024
        assert 2 <= info["stages"] <= opts["stages"]
        assert info["tile_bytes"] <= opts["tile_bytes"]
        if info["role_step"]:
            # stage-1 warps plus 1..6 survivor warps within 31
            sv = min(6, max(1, 31 - opts["warps"]))
            assert info["survivor_warps"] == sv
            assert info["warps"] == min(opts["warps"], 31 - sv)
        else:
            assert info["warps"] == opts["warps"] and info["survivor_warps"] == 0
        assert info["ctas_per_sm"] == opts["ctas_per_sm"]
        # asking for the chosen pipeline gives it again; only the survivor
        # tables may now move to shared memory (their place is decided
        # before the tile shrinks)
        again = rk.rk_plan(pats[name], smem_optin=optin, warps=info["warps"],
                           stages=info["stages"], tile_bytes=info["tile_bytes"],
                           ctas_per_sm=info["ctas_per_sm"])
        assert (again["tile_bytes"], again["stages"]) == (info["tile_bytes"], info["stages"])
        assert again["smem_bytes"] <= limit
        if info["s2_smem_bytes"]:
            assert again == info


@pytest.mark.parametrize("role_step,optin", [(1, 166912), (0, 120000)])
def test_stages_then_tiles_shrink(role_step, optin):
    pats = pattern_sets()["zipf"]
    full = rk.rk_plan(pats, stages=2, role_step=role_step)
    # more stages than fit: stages drop first, the tile stays
    many = rk.rk_plan(pats, stages=8, role_step=role_step)
    assert many["tile_bytes"] == full["tile_bytes"] and many["stages"] < 8
    # a device with less shared memory: the tile halves until it fits
    small = rk.rk_plan(pats, smem_optin=optin, role_step=role_step)
    assert small["stages"] == 2 and small["tile_bytes"] < full["tile_bytes"]
    assert full["tile_bytes"] % small["tile_bytes"] == 0
    assert small["smem_bytes"] <= optin - 1024


def test_survivor_tables_in_shared_memory_only_when_they_fit():
    pats = pattern_sets()
    zipf = rk.rk_plan(pats["zipf"])
    assert zipf["s2_smem_bytes"] > 0  # small tables travel to shared memory
    sig = rk.rk_plan(pats["signature"])
    assert sig["s2_smem_bytes"] == 0  # 2000 patterns: read from L2
    # more CTAs per SM leave less room: never more staged than with one
    two = rk.rk_plan(pats["zipf"], ctas_per_sm=2)
    assert two["s2_smem_bytes"] in (0, zipf["s2_smem_bytes"])


def test_device_bytes():
    pats = pattern_sets()
    for name, p in pats.items():
        info = rk.rk_plan(p)
        assert info["device_bytes"] % 256 == 0
        assert info["device_bytes"] >= sum((len(x) + 7) // 8 * 8 for x in p), name
    a = rk.rk_plan(pats["signature"][:500])["device_bytes"]
    b = rk.rk_plan(pats["signature"])["device_bytes"]
    assert b > a


def test_empty_set_and_rejections(lib):
    info = rk.rk_plan([])
    assert info["n_patterns"] == 0 and info["sample_step"] == 1
    for bad in (dict(base_log2=61), dict(filter=9), dict(tile_bytes=1000), dict(stages=1),
                dict(warps=40), dict(sample=2), dict(role_step=3), dict(ctas_per_sm=9)):
        with pytest.raises(rk.RkError) as e:
            rk.rk_plan([b"ab"], **bad)
        assert e.value.code == rk.RK_EINVAL, bad
    for pats in ([b"ab", b""], [b"x" * (rk.RK_MAX_PATTERN_LEN + 1)]):
        with pytest.raises(rk.RkError):
            rk.rk_plan(pats)
    with pytest.raises(rk.RkError):
        rk.rk_plan([b"ab"], smem_optin=1024)
    with pytest.raises(rk.RkError):
        # a 4096-byte halo per stage cannot fit in 16 KiB
        rk.rk_plan([b"y" * 4096], smem_optin=16384)
    cat = np.frombuffer(b"ab", dtype=np.uint8).copy()
    ln = np.array([2], dtype=np.uint32)
    assert lib.rk_plan(cat.ctypes.data, ln.ctypes.data, 1, None, OPTIN, None) == rk.RK_EINVAL
    info_c = rk.TableInfo()
    assert lib.rk_plan(cat.ctypes.data, ln.ctypes.data, 1, None, OPTIN,
                       ctypes.byref(info_c)) == rk.RK_OK
    assert info_c.n_patterns == 1 and info_c.min_len == 2


def test_plan_is_deterministic_and_order_free_in_shape():
    pats = pattern_sets()["signature"]
    a = rk.rk_plan(pats)
    b = rk.rk_plan(list(reversed(pats)))
    assert a == rk.rk_plan(pats)
    # ids follow input order, but the table's shape does not depend on it
    assert a == b
