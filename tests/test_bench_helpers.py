"""The bench's host-side helpers on CPU: the committed profile's figures are
used only while they were taken on the current scan sources, the oracle's
CPU sample covers every window it times, and the peak falls back when no
measured figure exists."""

import os
import shutil

import numpy as np
import pytest

import bench


def test_profile_figures_follow_the_source_hash(tmp_path, monkeypatch):
    """A profile summary is read only under the SHA-256 of the current scan
    sources: a copy of the committed summary carrying the current hash gives
    its figures, any edit of a source voids them, and so does a missing file."""
    txt = open(bench.PROFILE).read()
    import re
    cur = re.sub(r"scan_sources_sha256:\s*[0-9a-f]{64}",
                 "scan_sources_sha256: " + bench.scan_sources_sha256(), txt)
    prof_file = tmp_path / "profile.md"
    prof_file.write_text(cur)
    monkeypatch.setattr(bench, "PROFILE", str(prof_file))
    prof = bench.read_profile()
    assert prof is not None
    assert prof["dram_bytes_per_full_launch"] > 1 << 29  # at least the text, read once
    for key in ("tile_scan_alu_pipe_frac", "tile_scan_fmaheavy_pipe_frac",
                "tile_scan_issue_active_frac"):
        assert 0.0 < prof[key] <= 1.0, key
    # any change to a scan source invalidates the figures
    srcs = []
    for f in bench.SCAN_SRCS:
        dst = tmp_path / os.path.basename(f)
        shutil.copy(f, dst)
        srcs.append(str(dst))
    with open(srcs[0], "a") as fh:
        fh.write("\n// edited\n")
    monkeypatch.setattr(bench, "SCAN_SRCS", srcs)
    assert bench.read_profile() is None
    # and a missing profile gives none
    monkeypatch.setattr(bench, "PROFILE", str(tmp_path / "absent.md"))
    assert bench.read_profile() is None


def test_cpu_slices_carry_the_halo():
    text = np.random.default_rng(1).integers(0, 256, 1 << 16, dtype=np.uint8)
    tb = text.tobytes()
    slices = bench.cpu_slices(text, lmax=32, per_core=1000, cores=5)
    assert len(slices) == 5
    for s in slices:
        # a contiguous piece of the text: every window starting in its first
        # per_core bytes is complete (longest pattern - 1 extra bytes)
        assert len(s) == 1000 + 31
        at = tb.find(s)
        assert at >= 0 and at + len(s) <= len(tb)


def test_hbm_peak_fallback(monkeypatch, tmp_path):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.hbm_peak() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text('{"hbm_gbs": 6785.9}')
    assert bench.hbm_peak() == (6785.9, "measured")


def test_config_names_the_workload():
    cfg = bench.config_dict(1 << 30, 100)
    assert cfg["workload"] == bench.WORKLOAD and cfg["text_bytes"] == 1 << 30
    assert "L2" in cfg["l2"]
    assert not any(k in cfg for k in ("model", "seq_len"))


@pytest.mark.parametrize("argv", [["--warmup", "2"]])
def test_warmup_floor(argv, monkeypatch):
    monkeypatch.setattr("sys.argv", ["bench.py"] + argv)
    with pytest.raises(SystemExit):
        bench.main()
