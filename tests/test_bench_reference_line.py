"""bench.py --impl reference: the oracle timed on the host cores prints one JSON line
with the contract's keys, the same metric, unit and config as the GPU arm (built by the
same host-side function), and an e2e object with no host-device traffic."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    env = dict(os.environ)
    env.pop("RANK", None)
    env.pop("WORLD_SIZE", None)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--oracle-rows", "4", "--oracle-steps", "1"],
                       capture_output=True, text=True, cwd=ROOT, env=env, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    sys.path.insert(0, ROOT)
    import argparse
    import bench
    args = argparse.Namespace(workload="cube96_p2", nsteps=0, nshot=1, cg_rtol=1e-6, solve="persistent", cg_guess=3)
    assert line["impl"] == "reference"
    assert line["metric"] == bench.METRIC and line["unit"] == "shot-steps/s" and line["higher_is_better"] is True
    assert line["config"] == bench.workload_config(args)
    assert line["value"] > 0 and line["cpu_baseline"]["value"] == line["value"]
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"] == {"value": line["value"], "unit": "shot-steps/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_pcg_algorithmic_bytes_match_the_documented_count():
    """Roofline numerator of the persistent PCG: 536 B per row and launch (two 63-field
    FP32 applies + vectors) and 316 B per row and iteration on the 3-D p = 2 operator;
    the FP64 path doubles field and vector bytes (the residual is FP64 in both)."""
    sys.path.insert(0, ROOT)
    import bench
    assert bench.cg_bytes(63, 1, 4) == (536, 316)
    assert bench.cg_bytes(63, 1, 8) == (2 * 63 * 8 + 8 + 48, 63 * 8 + 8 + 104)
    # R right-hand sides share the field stream
    init4, it4 = bench.cg_bytes(63, 4, 4)
    assert it4 - 63 * 4 - 4 == 4 * (316 - 63 * 4 - 4)
