"""The benchmark's contract on the host: the reference arm (the oracle,
timed on the host cores) prints one JSON line with every field of the output
contract; ranks other than 0 print nothing; the GPU arm refuses to run without
a CUDA device instead of falling back to the CPU."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(args, env=None, timeout=300):
    e = dict(os.environ)
    e.update(env or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, cwd=ROOT,
                          env=e, capture_output=True, text=True, timeout=timeout)


def test_reference_arm_prints_one_contract_line():
    r = _run(["--impl", "reference", "--workload", "box_sphere_motion_64", "--steps", "1",
              "--warmup", "0"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["metric"] == "residual samples/s"
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["config"]["workload"] == "box_sphere_motion_64"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_exit_quietly():
    r = _run(["--impl", "reference", "--steps", "1", "--warmup", "0"],
             env={"RANK": "1", "LOCAL_RANK": "1", "WORLD_SIZE": "2"}, timeout=120)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""


def test_gpu_arm_refuses_without_a_device():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    r = _run(["--steps", "1", "--warmup", "0"], timeout=300)
    assert r.returncode != 0
    assert "CUDA device" in (r.stderr + r.stdout)


def test_multicore_oracle_timing_uses_disjoint_ranges():
    sys.path.insert(0, ROOT)
    import bench
    d = bench.cpu_baseline_multicore("box_sphere_motion_64", 16, 64, 1 << 16, cores=2)
    assert d["kind"] == "oracle" and d["cores"] == 2 and d["value"] > 0
    assert "1024 residual samples" in d["sample"]


def test_peak_probe_builds():
    """The bench's device-peak probe compiles for sm_103a (it runs only on a
    GPU)."""
    sys.path.insert(0, ROOT)
    import bench
    exe = bench.build_peak_probe()
    assert os.path.exists(exe) and os.access(exe, os.X_OK)


def test_record_comparison_counts_mismatches():
    """compare_records (the bench's oracle_error) matches samples by key and
    flags a moved pixel, a value beyond the tolerance and a missing sample."""
    sys.path.insert(0, ROOT)
    import numpy as np
    import bench
    from paper_2406_16302_gb300.rp import RECORD_DTYPE
    a = np.zeros(5, dtype=RECORD_DTYPE)
    a["root"] = np.arange(5)
    a["tech"] = 1
    a["frame"] = 2
    a["pix_a"] = 7
    a["pix_b"] = -1
    a["va"] = 1.0
    b = a.copy()
    b["va"][0] += 0.5e-4            # within 1e-4 of the magnitude
    b["va"][1] += 3e-4              # beyond it
    b["pix_a"][2] = 8               # another pixel
    good, total, worst = bench.compare_records(b[:4], a)
    assert (good, total) == (2, 5)
    assert abs(worst - 3e-4) < 1e-6
