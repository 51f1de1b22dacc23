"""bench.py's reference arm (the FP64 oracle on the host cores) runs without
a GPU and prints one JSON line with the contract's keys; the profile
summary it reads the DRAM traffic from matches the kernel source."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    # a small workload keeps the CPU suite short; the default is the full channel
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "3",
                          "--warmup", "3", "--workload", "neon_argon_2048x32"], cwd=ROOT,
                         capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr
    lines = [l for l in out.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "dtype", "config", "cpu_baseline", "e2e"):
        assert key in rec, key
    assert rec["impl"] == "reference" and rec["metric"] == "MLUPS" and rec["value"] > 0
    assert rec["cpu_baseline"]["kind"] == "oracle" and rec["cpu_baseline"]["cores"] >= 1
    assert rec["e2e"]["h2d_bytes_per_step"] == 0 and rec["e2e"]["value"] == rec["value"]
    assert rec["config"]["workload"] == "neon_argon_2048x32"
    assert rec["config"]["nodes_updated"] == 32 * (2048 - 2)


def test_profile_summary_traffic_is_current():
    sys.path.insert(0, ROOT)
    import bench
    t = bench.profiled_traffic()
    if t is None:
        pytest.skip("the committed profile predates the current step-kernel source")
    # the traffic is within 10 % of the 144 B per updated node it has to move
    assert abs(t / (144 * 16776192) - 1) < 0.1
