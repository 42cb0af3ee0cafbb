"""Host-side pieces of the benchmark line: committed DRAM-traffic figures count only while the
kernel sources they were measured on are unchanged, the peak comes from the measured file when
present, and the reference arm's contract keys are in place (no GPU needed)."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_traffic_follows_the_kernel_sources(monkeypatch):
    with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
        d = json.load(f)
    for step in ("forward_step", "adjoint_step"):
        assert step in bench.STEP_SOURCES
        v = bench.ncu_traffic(step)
        if d[step]["sources_sha1"] == bench.kernel_sources_sha1(bench.STEP_SOURCES[step]):
            assert v == float(d[step]["dram_bytes_per_launch"])
            assert v > 0
        else:
            assert v is None
    # any change to a source of the step voids its figure
    monkeypatch.setattr(bench, "kernel_sources_sha1", lambda names: "0" * 40)
    assert bench.ncu_traffic("forward_step") is None
    assert bench.ncu_traffic("adjoint_step") is None


def test_traffic_is_close_to_the_byte_model():
    """The committed per-launch traffic of the fused 3D steps sits at the algorithmic bytes
    (32 B per node forward, 44 B per node for the adjoint step's byte model) within 25 %."""
    nodes = 256 ** 3
    with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
        d = json.load(f)
    fw = d["forward_step"]["dram_bytes_per_launch"] / (32.0 * nodes)
    adj = d["adjoint_step"]["dram_bytes_per_launch"] / (44.0 * nodes)
    assert 0.95 < fw < 1.05
    assert 1.0 < adj < 1.25


def test_peak_from_the_measured_file():
    peak, kind = bench.peaks()
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            assert peak == float(json.load(f)["hbm_gbs"])
        assert kind == "measured"
    else:
        assert kind == "fallback" and peak > 0
