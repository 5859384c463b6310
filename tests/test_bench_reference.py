"""bench.py's reference arm (the CPU oracle, bounded samples) prints one JSON
line with the keys of the benchmark contract (CPU only, a small workload)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_line():
    out = subprocess.run(
        [sys.executable, "bench.py", "--impl", "reference", "--workload", "ising_chi4_L2_fp64",
         "--steps", "1", "--warmup", "3", "--ref-seconds", "0.2"],
        cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["metric"] == "MERA grad evals/s"
    assert line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["config"]["workload"] == "ising_chi4_L2_fp64"


def test_reference_line_whole_evaluations():
    """Workloads of the widened rows time whole oracle evaluations (here the
    Z2-symmetric ternary MERA at the size of the paper's Fig. 2)."""
    out = subprocess.run(
        [sys.executable, "bench.py", "--impl", "reference", "--workload", "ternary_ising_chi8_L2_fp64_z2",
         "--steps", "1", "--warmup", "3", "--ref-seconds", "0.2"],
        cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["value"] > 0 and line["value"] == line["cpu_baseline"]["value"]
    assert "energy/gradient evaluations" in line["cpu_baseline"]["sample"]
