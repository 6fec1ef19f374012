"""Host logic of bench.py: the compulsory-byte model of one MTTKRP, the
recorded-traffic lookup (only while the kernel source is unchanged), and the
parsing of the nvidia-smi clock samples taken during the timed region."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_mttkrp_compulsory_bytes():
    # stream (key 8 + value 4 per nonzero), every distinct input row once,
    # every distinct output row once
    b = bench.mttkrp_bytes(nnz=1000, key_bytes=8, val_bytes=4, distinct=[10, 20, 30], R=16, fbytes=2, obytes=4, n=1)
    assert b == 1000 * 12 + (10 + 30) * 16 * 2 + 20 * 16 * 4


def test_recorded_traffic_needs_matching_source(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    entry = {"source_hash": bench.kernel_source_hash(), "bytes_per_launch": {"0": 100, "1": 300}}
    (prof / "mttkrp_dram_traffic.json").write_text(json.dumps({"w/f32": entry}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    # the hash is computed from the kernel sources under ROOT: point it back
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: entry["source_hash"])
    assert bench.recorded_traffic("w", "f32", [1, 3]) == (100 * 1 + 300 * 3) / 4
    assert bench.recorded_traffic("w", "bf16", [1, 3]) is None
    entry["source_hash"] = "changed"
    (prof / "mttkrp_dram_traffic.json").write_text(json.dumps({"w/f32": entry}))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "current")
    assert bench.recorded_traffic("w", "f32", [1, 3]) is None


def test_clock_parsing():
    lines = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
             "0, 2055, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
             "0, 2070, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active",
             "garbage"]
    c = bench.ClockSampler.parse(lines)
    assert c == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    hot = bench.ClockSampler.parse(["0, 1500, 2070, 1400, 0x8, Active, Not Active, Active, Not Active"])
    assert hot["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    assert bench.ClockSampler.parse([]) is None
