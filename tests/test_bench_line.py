"""The bench's main arm end to end on CPU, with the GPU layer replaced by a
fake that answers as the library would (the oracle's match count), so that
the JSON line's assembly — every key the contract asks for, the roofline
with the profile's figures, the e2e and CPU-baseline objects — is exercised
before a GPU run depends on it."""

import json
import sys
import types

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import bench  # noqa: E402
import oracle  # noqa: E402
import workloads  # noqa: E402


CANDS = 1234  # candidate windows the fake tile scan reports


class FakeEvent:
    clock = 0.0

    def __init__(self, enable_timing=False):
        self.t = 0.0

    def record(self, stream=None):
        FakeEvent.clock += 0.5  # 0.5 ms between consecutive records
        self.t = FakeEvent.clock

    def elapsed_time(self, other):
        return other.t - self.t


class FakeStream:
    def __init__(self, device=None):
        self.cuda_stream = 0

    def synchronize(self):
        pass


def fake_rk(expect_m):
    rk = types.SimpleNamespace(RK_OK=0)
    state = {}

    def rk_search_device(table, d_text, n, keys, cap, info, ws, wsb, st=None):
        info[0] = expect_m
        info[1] = 0

    rk.rk_build = lambda patterns: 1
    rk.rk_destroy = lambda t: None
    rk.rk_table_info = lambda t: {"filter": 1, "filter_log2_bits": 14, "warps": 16,
                                  "tile_bytes": 49152, "stages": 2, "ctas_per_sm": 1,
                                  "smem_bytes": 216704, "s2_smem_bytes": 14080, "sm_count": 152,
                                  "role_step": 2, "role_filter_log2_bits": 19,
                                  "survivor_warps": 6, "sample_step": 1,
                                  "sample_filter_log2_bits": 0}

    def split(t, d, n, keys, cap, info, sws, scan_b, st, mid):
        state.setdefault("scans", []).append(1)
        sws[:8].view(torch.int64)[0] = CANDS
        mid.record(st)
    rk.rk_scan_workspace_bytes = lambda t, n: 256 + (n // 64 + 4096) * 16
    rk.rk_workspace_bytes = lambda t, cap: 16 * cap + 4096
    rk.rk_search_device = rk_search_device
    rk.rk_scan_launches = lambda t, n, b: 2
    rk.rk_sort_launches = lambda t, n, cap: 1
    rk.rk_scan_device_ws = lambda *a: state.setdefault("scans", []).append(1)
    rk.rk_scan_device_ws_split = split
    rk.rk_sort_device = lambda *a: None
    rk.rk_search = lambda t, h_text, n, h_keys, cap: (0, expect_m)
    rk.strerror = lambda rc: "ok"
    return rk, state


def fake_gpu(monkeypatch, rk, small):
    """Replace the library, CUDA streams, events and device placement with
    CPU stand-ins, and every configuration with the small workload."""
    pkg = types.SimpleNamespace(rk=rk, build_lib=types.SimpleNamespace(build=lambda: None))
    monkeypatch.setitem(sys.modules, "paper_1810_01051_gb300", pkg)
    monkeypatch.setattr(workloads, "make_config", lambda i, n=None, **k: small)
    monkeypatch.setattr(bench, "CPU_SAMPLE_PER_CORE", 64 << 10)
    real_device, real_empty = torch.device, torch.empty
    monkeypatch.setattr(torch, "device",
                        lambda *a, **k: real_device("cpu") if a and a[0] == "cuda" else
                        real_device(*a, **k))
    monkeypatch.setattr(torch, "empty",
                        lambda *a, pin_memory=False, **k: real_empty(*a, **k))
    monkeypatch.setattr(torch.cuda, "set_device", lambda d: None)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a: None)
    monkeypatch.setattr(torch.cuda, "Stream", FakeStream)
    monkeypatch.setattr(torch.cuda, "Event", FakeEvent)
    monkeypatch.setattr(torch.cuda, "get_device_properties",
                        lambda d: types.SimpleNamespace(uuid="fake"))
    monkeypatch.setattr(bench.time, "sleep", lambda s: None)


@pytest.mark.parametrize("cpu_baseline", [False, True])
def test_bench_line(monkeypatch, capsys, cpu_baseline):
    small = workloads.make_config(1, n=1 << 20)
    expect_m = int(oracle.rabin_karp(small.text, small.patterns)[0].size)
    rk, state = fake_rk(expect_m)
    fake_gpu(monkeypatch, rk, small)
    argv = ["bench.py", "--steps", "4", "--warmup", "3", "--no-extras", "--e2e-steps", "2"]
    if not cpu_baseline:
        argv.append("--no-cpu-baseline")
    monkeypatch.setattr(sys, "argv", argv)
    assert bench.main() == 0
    out = [line for line in capsys.readouterr().out.splitlines() if line.startswith("{")]
    assert len(out) == 1
    line = json.loads(out[0])

    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "roofline", "e2e", "gpu_launches", "clocks", "cpu_baseline"):
        assert key in line, key
    assert line["n_gpus"] == 1 and line["steps"] == 4 and line["warmup"] == 3
    assert line["config"]["workload"] == bench.WORKLOAD and "model" not in line["config"]
    assert line["matches"] == expect_m and line["dtype"] == "u8"
    assert len(state["scans"]) == 4 + 3  # warm-up and timed steps
    assert line["gpu_launches"] == 4 * (2 + 1)
    # each step spans three 0.5 ms event intervals (tile scan, verification,
    # sort) on the fake clock
    assert line["scan_ms"] == pytest.approx(1.0) and line["sort_ms"] == pytest.approx(0.5)
    assert line["tile_scan_ms"] == pytest.approx(0.5) and line["verify_ms"] == pytest.approx(0.5)
    assert line["candidates"] == CANDS
    roof = line["roofline"]
    assert roof["bound"] == "hbm" and roof["unit"] == "GB/s"
    assert roof["kernel"] == "rk_scan_rf_kernel"
    assert roof["algorithmic_bytes_per_launch"] == small.n + 16 * CANDS
    assert roof["achieved"] == pytest.approx((small.n + 16 * CANDS) / 0.5e-3 / 1e9)
    assert roof["frac"] == pytest.approx(roof["achieved"] / roof["peak"])
    assert roof["scan_step_frac"] == pytest.approx(
        (small.n + 8 * expect_m) / 1.0e-3 / 1e9 / roof["peak"])
    pk = roof["per_kernel"]
    assert set(pk) == {"tile_scan", "verify", "sort"}
    assert pk["verify"]["algorithmic_bytes"] == 16 * CANDS + 8 * expect_m
    assert pk["sort"]["algorithmic_bytes"] == 16 * expect_m
    for row in pk.values():
        assert row["ms"] == pytest.approx(0.5)
        assert row["frac"] == pytest.approx(row["algorithmic_bytes"] / 0.5e-3 / 1e9 / roof["peak"])
    prof = bench.read_profile()
    if prof is None:  # figures taken on other sources are not reported
        assert roof["traffic"] is None and roof["integer_pipes"] is None
    else:
        assert roof["traffic"] == prof["dram_bytes_per_full_launch"]
        assert roof["integer_pipes"]["alu_pipe_frac"] == prof["tile_scan_alu_pipe_frac"]
    e2e = line["e2e"]
    assert e2e["h2d_bytes_per_step"] == small.n and e2e["d2h_bytes_per_step"] == 16 + 8 * expect_m
    if cpu_baseline:
        cpu = line["cpu_baseline"]
        assert cpu["kind"] == "oracle" and cpu["cores"] >= 1 and cpu["value"] > 0
        assert cpu["value_one_core"] > 0 and "slices" in cpu["sample"]
        assert cpu["build"].startswith("gcc -O3")
    else:
        assert line["cpu_baseline"] is None
    assert np.isfinite(line["value"]) and line["value"] > 0


def test_signature_line(monkeypatch, capsys):
    """`--workload signature`: the signature-set object as a line of its own,
    with its per-kernel roofline (on the small workload and the fake GPU)."""
    small = workloads.make_config(1, n=1 << 20)
    expect_m = int(oracle.rabin_karp(small.text, small.patterns)[0].size)
    rk, state = fake_rk(expect_m)
    fake_gpu(monkeypatch, rk, small)
    monkeypatch.setattr(sys, "argv", ["bench.py", "--workload", "signature", "--steps", "3",
                                      "--warmup", "3"])
    assert bench.main() == 0
    out = [line for line in capsys.readouterr().out.splitlines() if line.startswith("{")]
    assert len(out) == 1
    line = json.loads(out[0])
    assert line["steps"] == 3 and line["n_gpus"] == 1 and line["dtype"] == "u8"
    assert line["config"]["text_bytes"] == small.n
    sig = line["signature_set"]
    assert sig["matches"] == expect_m and sig["candidates"] == CANDS
    roof = line["roofline"]
    assert roof is sig["roofline"] or roof == sig["roofline"]
    assert set(roof["per_kernel"]) == {"tile_scan", "verify", "sort"}
    assert roof["algorithmic_bytes_per_launch"] == small.n + 16 * CANDS
    assert roof["frac"] == pytest.approx(roof["achieved"] / roof["peak"])
    assert line["gpu_launches"] == 3 * (2 + 1)
    assert len(state["scans"]) == 3 + 3  # warm-up and timed steps (split or plain)
