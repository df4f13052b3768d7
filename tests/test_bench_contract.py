"""The benchmark's reference arm (the oracle on the host) prints one JSON line
with the keys the benchmark contract names; runs without a GPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3",
                          "--cpu-sample", "40"], cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["unit"] == "sweeps/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["warmup"] >= 3 and d["steps"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == os.cpu_count()
    assert 0.5 < d["cpu_baseline"]["exponent"] < 2.0  # the fitted growth of the oracle's time with N
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert "workload" in d["config"]


def test_committed_traffic_is_reported_only_for_the_captured_launch():
    """The ncu DRAM traffic in the row-sweep and gate-kernel summaries belongs to
    the default workload and launch shape; any other bench configuration
    reports null."""
    sys.path.insert(0, ROOT)
    import bench
    for kernel, name in (("row_sweep", "row_sweep_so52_e12_N1e6.md"), ("ansatz", "ansatz_so52_e12_N1e6.md")):
        text = open(os.path.join(ROOT, "profiles", name)).read()
        committed = int(text.split("traffic_bytes_per_launch:")[1].split()[0])
        assert bench.measured_traffic(kernel, bench.parse([])) in (committed, None)
        for argv in (["--n-keep", "300000"], ["--threads", "512"], ["--cluster", "2"], ["--rows-l2", "1"],
                     ["--sweep", "1"]):
            assert bench.measured_traffic(kernel, bench.parse(argv)) is None, argv
    assert bench.measured_traffic("energy", bench.parse([])) is None


def test_scaling_exponent_recovers_a_power_law():
    sys.path.insert(0, ROOT)
    import bench
    assert abs(bench.scaling_exponent(100, 2.0, 400, 2.0 * 4 ** 1.25) - 1.25) < 1e-12
