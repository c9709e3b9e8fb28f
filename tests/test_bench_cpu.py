"""The benchmark's reference arm (the CPU oracle timed on a bounded sample) runs without a GPU
and prints one JSON line with the keys the benchmark contract names."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--small",
                          "--steps", "2", "--warmup", "1", "--cpu-iters", "2"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr
    lines = [l for l in out.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 2 and d["warmup"] == 1
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert "workload" in d["config"]


def test_group_sweep_rejects_sizes_outside_the_group():
    """The grouping sweep checks its sizes against the group's systems before any device work."""
    for bad in ("0", "1,129", ","):
        out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--group-sweep", bad],
                             capture_output=True, text=True, timeout=600, cwd=ROOT)
        assert out.returncode != 0 and "--group-sweep sizes must lie in 1..128" in out.stderr, (bad, out.stderr)
