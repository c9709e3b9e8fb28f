"""The benchmark's reference arm (the CPU oracle timed on a bounded sample) runs without a GPU
and prints one JSON line with the keys the benchmark contract names."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--small",
                          "--steps", "2", "--warmup", "1", "--cpu-seconds", "0.5"],
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


def test_clock_sampler_parses_speeds_and_throttle_reasons(tmp_path):
    """The clock record of the timed region: median SM clock, the maximum, and every throttle
    reason seen Active in any sample (malformed lines are skipped, the sample file removed)."""
    sys.path.insert(0, ROOT)
    import bench

    class Done:
        def terminate(self):
            pass

        def wait(self):
            return 0

    c = bench.Clocks(0)
    c.path = str(tmp_path / "clocks.csv")
    with open(c.path, "w") as fh:
        fh.write("2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                 "1995, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active\n"
                 "garbage line\n"
                 "[N/A], 2070, 10.0, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                 "2040, 2070, 1200.0, 0x40, Not Active, Active, Not Active, Not Active\n")
    c.p, c.out = Done(), open(os.devnull, "w")
    rec = c.stop()
    assert rec["sm_mhz"] == 2040.0 and rec["sm_max_mhz"] == 2070.0 and rec["samples"] == 3
    assert rec["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    assert not os.path.exists(c.path)
    c2 = bench.Clocks(0)
    assert c2.stop()["reasons"] == ["nvidia-smi unavailable"]       # sampler never started


def test_algorithmic_bytes_per_node_system_by_configuration():
    """The roofline's byte model of one CGLS iteration per node and system: phase 1 reads s, p_old
    and writes p, t1 (32 B) plus x in and out (16 B) when it updates x, and m - 1 older directions
    (8 B each) in the iteration that adds the steps of m iterations; phase 2 reads r1, t1 and writes
    r1, s (32 B).  One update per iteration: 80 B; every second iteration (configurations 22, 23):
    76 B; every fourth (24): 74 B."""
    import types
    sys.path.insert(0, ROOT)
    import bench

    def b(kernel):
        return bench.bytes_per_node_sys(types.SimpleNamespace(kernel=kernel))

    for m, cfgs in ((1, (8, 9, 18, 20, 21)), (2, (22, 23)), (4, (24,))):
        per_iter = 32 + 32 + (16 + 8 * (m - 1)) / m
        for c in cfgs:
            assert b(2 + c) == per_iter, (c, b(2 + c), per_iter)
    assert b(0) == b(1) == 80.0
    assert (b(2 + 18), b(2 + 22), b(2 + 24)) == (80.0, 76.0, 74.0)
