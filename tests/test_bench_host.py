"""Host-side pieces of bench.py that need no GPU: the oracle baseline on the host cores
(the whole map of a small workload, rows over a process pool), which workloads it
covers, and the JSON the reference arm prints where it does not."""
import json
import os
import subprocess
import sys


ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_full_oracle_map_on_the_host_cores():
    import bench
    import workloads
    from oracle import rixs as orixs
    wl = workloads.tiny(6, 3, 3)
    r = bench.cpu_full_map(wl, return_map=True)
    assert r["kind"] == "oracle" and r["cores"] >= 1 and r["value"] > 0
    ref = orixs.rixs_map(6, 3, 3, 1.0, 8.0, 4.0, 0, wl.Gamma, wl.eta, wl.w_in, wl.w,
                         gs_start=workloads.lanczos_start(400, wl.lanczos_seed))
    assert orixs.relative_l2(r["map"], ref.I) <= 1e-10


def test_baseline_coverage():
    import bench
    r = bench.run_cpu_baseline("hubbard-L10-11-12-clusters-mixed")
    assert r["value"] is None and r["kind"] == "oracle" and "not sampled" in r["sample"]
    assert bench.DEFAULT == "hubbard-L14-mixed"
    assert bench.host_cores() >= 1


def test_reference_arm_unavailable_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                          "solve-sweep-L12", "--steps", "1", "--warmup", "0"],
                         capture_output=True, text=True, timeout=300, env=dict(os.environ, CUDA_VISIBLE_DEVICES=""))
    assert out.returncode == 0, out.stderr
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and "unavailable" in line


def test_traffic_only_for_the_captured_launch_shape():
    """The measured DRAM traffic of a capture scales to the bench's launches only when the
    bench ran the launch shape that was captured."""
    import json
    import bench
    rec = json.load(open(os.path.join(ROOT, "profiles", "ncu_traffic.json")))
    for wl, shape in (("hubbard-L14-mixed", 1), ("hubbard-L12-fp64", 128)):
        r = rec[wl]["cf_apply"]
        assert r["shape"] == shape and r["dram_bytes"] > 0
        t = bench.measured_traffic(wl, "cf_apply", 1e9, shape)
        assert t == r["dram_bytes"] / r["alg_bytes"] * 1e9
        # DRAM bytes over algorithmic bytes: below 1 where the captured columns' V_k stays
        # in L2 across the launch (the 8-column L = 12 capture), above 1 for partner rows
        # evicted and read again (L = 14)
        assert 0.8 <= t / 1e9 < 1.3
        assert bench.measured_traffic(wl, "cf_apply", 1e9, shape + 1) is None
    assert bench.measured_traffic("no-such-workload", "cf_apply", 1e9, 1) is None
