"""The bench's reference arm (the FP64 oracle on the host cores) runs without a
GPU: its one JSON line carries the fields the measurement contract names, and
the timing rules are enforced on the command line."""
import json
import os
import subprocess
import sys

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args):
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT,
                          capture_output=True, text=True, timeout=600)


def test_reference_arm_json_line():
    r = _run("--impl", "reference", "--steps", "1", "--warmup", "3")
    assert r.returncode == 0, r.stderr[-2000:]
    line = [ln for ln in r.stdout.splitlines() if ln.startswith("{")][-1]
    d = json.loads(line)
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "dof-updates/s"
    assert d["value"] > 0 and d["higher_is_better"] is True and d["n_gpus"] == 1
    assert d["steps"] == 1 and d["warmup"] == 3 and d["ms_per_step"] > 0
    assert d["scaling"] == "weak" and d["vs_baseline"] is None and d["dtype"] == "f64"
    assert "workload" in d["config"] and d["config"]["nodes"] == 64 ** 3 * 6 ** 3 and "sample" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_timing_rules_on_the_command_line():
    assert _run("--impl", "reference", "--steps", "1", "--warmup", "2").returncode == 2


def test_captured_counters_follow_the_kernel_sources(monkeypatch):
    """The DRAM traffic and the SR stage kernel's flop counts come from ncu captures
    of the committed kernels; they are reported only while the kernels' sources
    hash as they did at capture, and dropped (null) once a source changes."""
    assert bench._traffic() == bench.TRAFFIC_BYTES_PER_LAUNCH
    roof = bench._alu_roofline(0.2)
    assert roof["bound"] == "alu" and roof["fp64"]["flops_per_launch"] == bench.SR_STAGE_FLOPS["fp64"]
    assert abs(roof["frac"] - bench.SR_STAGE_FLOPS["fp64"] / 0.2e-3 / 1e12 / bench.FP64_PEAK_TFLOPS) < 1e-12
    monkeypatch.setattr(bench, "TRAFFIC_SOURCES_SHA256", "0" * 64)
    monkeypatch.setattr(bench, "SR_STAGE_SOURCES_SHA256", "0" * 64)
    assert bench._traffic() is None
    assert bench._alu_roofline(0.2)["achieved"] is None


def test_roofline_arithmetic():
    """64 B per dof-update in the FP64-state model: 320 B per node-step, a mean of
    106.7 B per node and stage launch; the ensemble's HBM fraction is those bytes
    over the step time against the measured peak."""
    assert abs(bench.FP64_STATE_BYTES_PER_NODE_STAGE * 3 - 320.0) < 1e-12
    r = bench._ensemble_roofline(1_000_000, 1.0)
    assert abs(r["achieved"] - 320.0) < 1e-9 and abs(r["frac"] - 320.0 / r["peak"]) < 1e-12
