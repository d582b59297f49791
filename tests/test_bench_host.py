"""Host logic of the benchmark that needs no GPU: the clock record taken during the timed
region (median SM clock, throttle reasons) and the per-launch DRAM traffic, which is
reported only while the measured kernel's sources are the ones that were captured."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


class _FakeProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _clocks_from(tmp_path, rows):
    path = tmp_path / "clocks.csv"
    path.write_text("\n".join(rows) + "\n")
    s = bench.ClockSampler(0)
    s.proc = _FakeProc()
    s.file = open(path, "r+")
    return s.stop()


def test_clock_record_median_and_reasons(tmp_path):
    rows = [
        "0, 2070, 2070, 250.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 610.4, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 300.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
    ]
    clk = _clocks_from(tmp_path, rows)
    assert clk["sm_mhz"] == 2070.0
    assert clk["sm_max_mhz"] == 2070.0
    assert clk["reasons"] == ["sw_power_cap"]
    assert clk["samples"] == 3
    assert clk["power_w_max"] == pytest.approx(610.4)
    assert not os.path.exists(tmp_path / "clocks.csv")   # the sample file is removed


def test_clock_record_flags_thermal_slowdown(tmp_path):
    rows = ["0, 1500, 2070, 900.0, 0x68, Active, Active, Active, Not Active"]
    clk = _clocks_from(tmp_path, rows)
    assert clk["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]


def test_clock_record_without_samples(tmp_path):
    clk = _clocks_from(tmp_path, ["[N/A], [N/A], x, y, z, a, b, c, d"])
    assert clk["sm_mhz"] is None and clk["reasons"] == ["no samples"]
    assert bench.ClockSampler(0).stop()["reasons"] == ["nvidia-smi unavailable"]


def _traffic_table(tmp_path, rows):
    path = tmp_path / "traffic.md"
    path.write_text("| kernel | traffic bytes per launch | capture | source |\n"
                    "|---|---|---|---|\n" + "".join(f"| {' | '.join(r)} |\n" for r in rows))
    return str(path)


def test_traffic_reported_only_for_the_captured_sources(tmp_path, monkeypatch):
    now = bench.source_hash(bench.KERNEL_SOURCES["direct laplacian3"])
    monkeypatch.setattr(bench, "TRAFFIC_FILE", _traffic_table(tmp_path, [
        ("direct laplacian3", "616133632", "read 1 + write 2 B", now),
        ("separable gaussian5", "616420352", "read 3 + write 4 B", "0000000000000000"),
    ]))
    assert bench.captured_traffic("direct laplacian3") == (616133632.0, "read 1 + write 2 B")
    # a capture taken from other sources is not reported
    assert bench.captured_traffic("separable gaussian5") == (None, "kernel changed since the capture")


def test_traffic_missing_capture(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "TRAFFIC_FILE", _traffic_table(tmp_path, []))
    assert bench.captured_traffic("direct laplacian3") == (None, "kernel not captured")
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(tmp_path / "absent.md"))
    assert bench.captured_traffic("direct laplacian3") == (None, "no capture summary")



def test_reference_arm_line(monkeypatch, capsys):
    """The reference arm times the FP64 oracle on the host and prints one JSON line with the
    same metric and unit as the GPU arm, a cpu_baseline and a zero-copy e2e entry (here on a
    small stand-in volume and a few hundred voxels per step, to keep the test short)."""
    import json

    import numpy as np
    import synth
    small = synth.volume("blobs", synth.U8, (32, 24, 16), synth.BASE_SEED + 1)
    monkeypatch.setattr(bench, "workload_host", lambda: small)
    monkeypatch.setattr(bench, "oracle_sample_rate", lambda vol, seconds: (1e6, 300, 0.1))
    for var in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(var, raising=False)

    class Args:
        steps, warmup = 3, 1

    bench.run_reference(Args())
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == "Gvoxel/s"
    assert d["higher_is_better"] is True and d["n_gpus"] == 1
    assert d["steps"] == 3 and d["warmup"] == 1
    assert d["value"] > 0 and np.isfinite(d["value"])
    assert d["config"]["workload"] == bench.WORKLOAD
    cpu = d["cpu_baseline"]
    assert cpu["kind"] == "oracle" and cpu["value"] == d["value"] and cpu["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": "Gvoxel/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
