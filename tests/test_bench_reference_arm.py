"""The reference arm of bench.py on CPU: `--impl reference` times the oracle and prints one
JSON line with the GPU arm's metric, unit, direction and config (one solve of the step's
workload per step), an oracle cpu_baseline and an e2e block that moves no bytes.  Run on a
32 x 32 crossbar so it takes a second."""
import argparse
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--size", "32", "--steps", "2", "--warmup", "1"],
                       capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [x for x in r.stdout.splitlines() if x.strip().startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    sys.path.insert(0, ROOT)
    import bench
    ours = bench.step_config(argparse.Namespace(size=32, handles=2, batch=64, restart=30,
                                                precision="bf16split", device="sinh",
                                                neg_ratio=0.5))
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == "solves/s"
    assert d["higher_is_better"] is True and d["steps"] == 2 and d["warmup"] == 1
    assert d["config"] == ours                 # the GPU arm's config, key for key
    assert d["value"] > 0 and d["ms_per_step"] > 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "solves/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_oracle_once_times_one_converged_solve():
    sys.path.insert(0, ROOT)
    import bench
    t = bench.oracle_once(32)
    assert 0.0 < t < 60.0


def test_secondary_leg_records_a_failure_in_line():
    sys.path.insert(0, ROOT)
    import bench
    out = {}
    bench.secondary_leg(out, "ok", lambda: {"value": 1.0})

    def fails():
        raise RuntimeError("side figure failed")
    bench.secondary_leg(out, "bad", fails)
    assert out["ok"] == {"value": 1.0}
    assert out["bad"] == {"error": "RuntimeError: side figure failed"}
