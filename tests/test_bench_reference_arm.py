"""bench.py --impl reference (the FP64 oracle timed on the host cores) runs
without a GPU and prints one JSON line with the contract's keys and the
same config as the GPU arm reports."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e", "impl"):
        assert k in d, k
    assert d["impl"] == "reference" and d["higher_is_better"] is False
    assert d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    sys.path.insert(0, ROOT)
    import argparse
    import bench
    a = argparse.Namespace(config="cl50k", outer=30, tol=1e-4, check_every=5)
    assert d["config"] == bench._config(a, 1)


def test_sweep_traffic_is_reported_only_for_the_captured_kernel_and_width(tmp_path, monkeypatch):
    """roofline.traffic comes from the committed ncu record only while the
    sweep's source hashes to the recorded value and the row width is the
    captured one; it scales with the rows."""
    import argparse
    sys.path.insert(0, ROOT)
    import bench
    rec = json.load(open(os.path.join(ROOT, "profiles", "k_sweep_traffic.json")))
    a = argparse.Namespace(dtype="bf16")
    got = bench._ncu_traffic(a, 50_000, 50_000)
    if rec["source_sha256"] == bench.sweep_source_hash():
        assert got == rec["bf16"]["dram_bytes_per_launch_captured"] * 10
        assert abs(got - 5.0e9) / 5.0e9 < 0.02          # the algorithmic bytes
        assert bench._ncu_traffic(a, 25_000, 50_000) == got // 2
    else:
        assert got is None
    assert bench._ncu_traffic(a, 100_000, 80_000) is None   # another launch shape
    monkeypatch.setattr(bench, "sweep_source_hash", lambda: "0" * 64)
    assert bench._ncu_traffic(a, 50_000, 50_000) is None    # another kernel source
