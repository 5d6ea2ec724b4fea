"""bench.py's reference arm (the FP64 oracle timed on the host) prints the
JSON line the benchmark contract asks for; run here on a small L-shape."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_line_has_the_contract_keys():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "lshape", "--N", "33", "--steps", "2", "--warmup", "3"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads([l for l in out.stdout.splitlines() if l.startswith("{")][-1])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["steps"] == 2 and line["warmup"] == 3
    assert line["value"] > 0 and line["higher_is_better"] is True
    assert "workload" in line["config"]
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_other_ranks_exit_quietly():
    """Under torchrun only rank 0 runs the reference arm; other ranks exit 0."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "lshape", "--N", "33", "--steps", "1", "--warmup", "0",
                          "--gpus", "2"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    assert not [l for l in out.stdout.splitlines() if l.startswith("{")]


def test_cpu_baseline_one_core_and_all_cores():
    """The CPU baseline times the oracle on one host core and on every core, and
    records the host CPU as lscpu reports it."""
    import argparse
    sys.path.insert(0, ROOT)
    import bench
    from paper_2001_11533_gb300 import workloads as W
    args = argparse.Namespace(hessian_levels=0, coarse_max=1000, degree=2, inner_tol=1e-10, cpu_budget=0.2)
    cb = bench.cpu_baseline(W.lshape_checkerboard(N=33), args)
    assert cb["kind"] == "oracle" and cb["value"] > 0 and cb["unit"] == bench.UNIT
    assert cb["cores"] == (os.cpu_count() or 1)
    assert cb["single_core"]["cores"] == 1 and cb["single_core"]["value"] > 0
    assert cb["host"]["nproc"] == os.cpu_count()
