"""The seeded input generator against its recipe (CPU only): alphabets,
letter weights, size and length ranges, plant counts, determinism, and that
the module holds none of the matching arithmetic."""

import ast
import inspect
import os

import numpy as np

import workloads
from workloads import gen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_same_seed_same_bytes():
    a = gen.zipf_large(n=1 << 16)
    b = gen.zipf_large(n=1 << 16)
    c = gen.zipf_large(seed=1, n=1 << 16)
    assert np.array_equal(a.text, b.text) and a.patterns == b.patterns
    assert not np.array_equal(a.text, c.text)


def test_full_size_defaults():
    # the configurations' sizes live in the defaults; nothing is drawn here
    def defaults(fn):
        return {k: v.default for k, v in inspect.signature(fn).parameters.items()}
    d = defaults(gen.dna_single)
    assert (d["n"], d["k"], d["m"], d["plants"]) == (1 << 20, 8, 16, 50)
    z = defaults(gen.zipf_large)
    assert (z["n"], z["k"], z["lmin"], z["lmax"], z["density"]) == (1 << 30, 100, 4, 32, 1e-6)
    s = defaults(gen.signature_set)
    assert (s["n"], s["k"], s["lmin"], s["lmax"], s["plants"]) == (4 << 30, 10000, 8, 64, 1000)
    b = defaults(gen.batched)
    assert (b["n_items"], b["min_len"], b["max_len"], b["k_min"], b["k_max"], b["lmin"],
            b["lmax"], b["density"]) == (4096, 1 << 10, 1 << 24, 1, 256, 4, 48, 1e-5)
    t = defaults(gen.serving_tables)
    assert (t["n_tables"], t["k_max"], t["lmin"], t["lmax"]) == (64, 1024, 4, 64)
    assert [gen.FULL[i]["seed"] for i in (0, 1, 2)] == [0x5EED0000, 0x5EED0001, 0x5EED0002]


def test_zipf_lut_weights():
    lut = gen.zipf_lut()
    assert lut.size == 1 << gen.LUT_BITS
    counts = np.bincount(lut, minlength=256)
    syms = set(np.nonzero(counts)[0].tolist())
    assert syms == set(gen.ZIPF_ORDER) | {ord(" ")}
    h = sum(1.0 / r for r in range(1, 27))
    q = 1.0 / (1 << gen.LUT_BITS)
    assert abs(counts[ord(" ")] * q - 1 / 6) <= q
    for r, c in enumerate(gen.ZIPF_ORDER, start=1):
        # letter of rank r: (1/r) / H_26 of the 5/6 that are not spaces
        assert abs(counts[c] * q - (5 / 6) / (r * h)) <= q, chr(c)


def test_zipf_text_frequencies():
    w = gen.zipf_large(n=1 << 22, k=10)
    counts = np.bincount(w.text, minlength=256)
    lut_p = np.bincount(gen.zipf_lut(), minlength=256) / (1 << gen.LUT_BITS)
    # planted bytes are a few hundred of 4 Mi; every frequency within 5 sigma
    n = w.n
    for c in np.nonzero(lut_p)[0]:
        sigma = np.sqrt(n * lut_p[c] * (1 - lut_p[c]))
        assert abs(counts[c] - n * lut_p[c]) < 5 * sigma + 400, chr(c)
    assert counts.sum() == counts[np.nonzero(lut_p)[0]].sum()
    assert all(set(p) <= set(gen.ZIPF_ORDER) | {ord(" ")} for p in w.patterns)
    assert all(4 <= len(p) <= 32 for p in w.patterns)
    assert all(len(pl) == round(1e-6 * n) for pl in w.planted)


def test_dna_single_shape():
    w = gen.dna_single(n=1 << 18)
    assert w.text.dtype == np.uint8 and w.text.flags["C_CONTIGUOUS"]
    assert set(np.unique(w.text).tolist()) == set(b"ACGT")
    counts = np.bincount(w.text)[list(b"ACGT")]
    assert np.all(np.abs(counts - w.n / 4) < 5 * np.sqrt(w.n * 3 / 16))
    assert len(w.patterns) == 8 and all(len(p) == 16 and set(p) <= set(b"ACGT")
                                        for p in w.patterns)
    assert all(len(pl) == 50 for pl in w.planted)


def test_plants_are_written_in_order():
    # later plants overwrite earlier ones, so the last pattern's plants are
    # all intact and every plant lies inside the text
    w = gen.random_small(5, 2000, 6, 3, 9, alphabet=b"xyz", plants=7)
    t = w.text.tobytes()
    for p, pl in zip(w.patterns, w.planted):
        assert pl.size == 7 and np.all(pl >= 0) and np.all(pl <= w.n - len(p))
    last, pl = w.patterns[-1], w.planted[-1]
    assert all(t[x:x + len(last)] == last for x in pl.tolist())


def test_signature_set_scaling():
    w = workloads.make_config(2, n=1 << 20, k=50)
    assert len(w.patterns) == 50 and all(8 <= len(p) <= 64 for p in w.patterns)
    # plants scale with the text: 1000 per pattern at 4 GiB
    assert all(len(pl) == max(1, round(1000 * (1 << 20) / (4 << 30))) for pl in w.planted)
    vals = np.bincount(w.text, minlength=256)
    assert vals.min() > 0 and abs(vals.mean() - w.n / 256) < 1


def test_batched_shape():
    b = gen.batched(n_items=64, max_len=1 << 14)
    assert len(b.texts) == len(b.tables) == 64 and b.table_of == list(range(64))
    sizes = np.array([t.size for t in b.texts])
    assert sizes.min() >= 1 << 10 and sizes.max() <= 1 << 14
    alpha = set(gen.BATCH_ALPHABET)
    for t, pats in zip(b.texts, b.tables):
        assert set(np.unique(t).tolist()) <= alpha
        assert 1 <= len(pats) <= 256
        assert all(4 <= len(p) <= 48 and set(p) <= alpha for p in pats)
    assert b.total_bytes == sizes.sum()


def test_batched_lengths_log_uniform():
    b = gen.batched(n_items=2000, min_len=1 << 4, max_len=1 << 12, k_max=1)
    logs = np.log2([t.size for t in b.texts])
    # log2 of the sizes is uniform on [4, 12]: mean 8, deciles evenly spaced
    assert abs(logs.mean() - 8.0) < 0.15
    dec = np.percentile(logs, np.arange(10, 100, 10))
    assert np.all(np.abs(dec - (4 + 0.8 * np.arange(1, 10))) < 0.3)


def test_serving_shape():
    tables = gen.serving_tables(n_tables=8, k_max=40)
    assert len(tables) == 8
    assert all(1 <= len(t) <= 40 and all(4 <= len(p) <= 64 for p in t) for t in tables)
    reqs = gen.serving_texts(3, 20, tables, min_len=1 << 10, max_len=1 << 14)
    assert len(reqs) == 20
    for tid, text in reqs:
        assert 0 <= tid < 8 and (1 << 10) <= text.size <= (1 << 14)


def test_generator_holds_no_matching_arithmetic():
    # the inputs are shared by the oracle and the GPU path: the generator
    # imports neither and never compares or hashes windows
    for name in ("__init__.py", "gen.py"):
        tree = ast.parse(open(os.path.join(ROOT, "workloads", name)).read())
        for node in ast.walk(tree):
            mods = []
            if isinstance(node, ast.Import):
                mods = [a.name for a in node.names]
            elif isinstance(node, ast.ImportFrom):
                mods = [node.module or ""]
            for m in mods:
                assert not m.startswith(("oracle", "paper_1810_01051_gb300")), (name, m)
    src = open(os.path.join(ROOT, "workloads", "gen.py")).read()
    for word in ("hash", "find(", "memcmp", "2**61", "1 << 61"):
        assert word not in src.split('"""', 2)[-1], word
