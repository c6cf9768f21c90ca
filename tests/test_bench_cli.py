"""The benchmark's CPU-side legs, run on the smallest workload: the reference
arm (full oracle solves, capped step count, one JSON line with the keys the
benchmark contract names) and the all-core oracle column."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                          "16x16x4_b4", "--steps", "5", "--warmup", "2"], capture_output=True, text=True,
                         timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "config",
              "cpu_baseline", "e2e", "impl"):
        assert k in d, k
    assert d["impl"] == "reference" and d["higher_is_better"] is False
    assert d["steps"] == 3 and d["warmup"] == 1 and d["steps_requested"] == 5
    assert d["cpu_baseline"]["detail"]["converged"] and d["cpu_baseline"]["detail"]["true_relres"] <= 1e-6
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


def test_all_core_oracle_column():
    sys.path.insert(0, ROOT)
    import bench
    col = bench.oracle_all_cores("16x16x4_b4", 1e-6, 30, 4104)
    assert col["cores"] >= 1 and col["value"] > 0.0 and col["iters"] == [10]
