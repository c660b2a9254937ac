"""Host-side pieces of bench.py that need no GPU: which workloads the oracle's bounded
CPU sample covers, and the JSON the reference arm prints where it does not."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_oracle_sample_bounds():
    import bench
    assert bench.oracle_feasible("hubbard-L12-fp64")          # the default workload
    assert bench.oracle_feasible("hubbard-L8-fp64")
    assert not bench.oracle_feasible("hubbard-L14-mixed")     # D = 11.8 M
    assert not bench.oracle_feasible("hubbard-L10-11-12-clusters-mixed")
    r = bench.run_cpu_baseline("hubbard-L14-fp64")
    assert r["value"] is None and r["kind"] == "oracle" and "not sampled" in r["sample"]


def test_reference_arm_unavailable_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                          "hubbard-L14-mixed", "--steps", "1", "--warmup", "0"],
                         capture_output=True, text=True, timeout=300, env=dict(os.environ, CUDA_VISIBLE_DEVICES=""))
    assert out.returncode == 0, out.stderr
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and "unavailable" in line
