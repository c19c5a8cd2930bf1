"""Host helpers of bench.py (CPU): the committed DRAM-traffic record is reported
only for the kernel source and workload it was taken on, the printed count is
compared with the oracle's stored values, and the clock record flags throttling."""
import json

import bench


def test_recorded_traffic_only_for_its_source_and_workload(monkeypatch, tmp_path):
    sha = "ab" * 32
    rec = {"records": [{"workload": "rmat-s23", "p": 4, "kernel": "auto", "source_sha256": sha,
                        "dram_bytes_per_launch": 123}]}
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "k_count_traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: sha)
    assert bench.recorded_traffic("rmat-s23", 4, "auto") == 123
    assert bench.recorded_traffic("rmat-s23", 8, "auto") is None
    assert bench.recorded_traffic("rmat-s23", 4, "hashmap") is None
    assert bench.recorded_traffic("chunglu-friendster", 4, "auto") is None
    # a changed kernel source invalidates the record
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "cd" * 32)
    assert bench.recorded_traffic("rmat-s23", 4, "auto") is None


def test_golden_triangles_of_the_bench_workloads():
    assert bench.golden_triangles("chunglu-friendster") == 193731339
    assert bench.golden_triangles("rmat-s23") == 4673989558
    assert bench.golden_triangles("no-such-workload") is None


def test_clock_summary_flags_throttle_reasons(tmp_path):
    s = bench.ClockSampler(0)
    s.proc = object()  # samples already written
    lines = [
        "0, 2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 2070, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 1980, 2070, 1395.0, 0x4, Not Active, Not Active, Not Active, Active",
        "malformed",
    ]
    with open(s.path, "w") as f:
        f.write("\n".join(lines) + "\n")
    out = s.summary()
    assert out["samples"] == 3
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]
    s2 = bench.ClockSampler(0)
    s2.proc = object()
    with open(s2.path, "w") as f:
        f.write("0, 1500, 2070, 800.0, 0x8, Active, Not Active, Not Active, Not Active\n")
    assert s2.summary()["reasons"] == ["hw_slowdown"]
