"""The benchmark's reference arm (the CPU oracle timed on the host) prints
one JSON line with the fields the benchmark contract names."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "2", "--warmup", "3"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["metric"] == "cell-updates/s" and d["value"] > 0 and d["steps"] == 2
    assert d["config"]["workload"] == "aco_2048x2048_100k_agents"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


def test_warmup_below_three_is_refused():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "2", "--warmup", "2"],
                         capture_output=True, text=True, timeout=120, cwd=ROOT)
    assert out.returncode != 0


def test_traffic_figure_only_for_the_profiled_kernel_source(tmp_path, monkeypatch):
    """roofline.traffic comes from the committed ncu summary only while the
    summary's kernel-source hash matches the current kernel sources."""
    sys.path.insert(0, ROOT)
    import bench
    cur = bench.kernel_source_hash()
    f = tmp_path / "traffic.md"
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(f))
    f.write_text(f"kernel_source_sha256_16: {cur}\ndram_bytes_per_launch: 73932672\n")
    assert bench.recorded_traffic() == 73932672.0
    f.write_text("kernel_source_sha256_16: 0000000000000000\ndram_bytes_per_launch: 73932672\n")
    assert bench.recorded_traffic() is None             # stale: taken on other sources
    f.write_text(f"kernel_source_sha256_16: {cur}\n")
    assert bench.recorded_traffic() is None             # no figure recorded
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(tmp_path / "missing.md"))
    assert bench.recorded_traffic() is None
    # the committed summary names its own hash and figure
    monkeypatch.undo()
    text = open(bench.TRAFFIC_FILE).read()
    assert "kernel_source_sha256_16:" in text and "dram_bytes_per_launch:" in text
