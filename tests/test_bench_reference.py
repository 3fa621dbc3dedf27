"""The reference arm of bench.py (the CPU oracle, timed on the host cores) on
CPU: one JSON line with the contract's keys, the same metric, unit and
config as the CUDA arm's line, no host-device bytes; under a multi-rank
launch only rank 0 prints."""

import json
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _run(extra_env, *args):
    env = dict(os.environ, **extra_env)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", *args],
                          capture_output=True, text=True, env=env, cwd=ROOT, timeout=600)


def test_reference_line_matches_the_cuda_arms_contract():
    sys.path.insert(0, ROOT)
    import bench
    r = _run({}, "--steps", "1", "--warmup", "0", "--workload", "d2_256x256_i64_add_k16")
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["higher_is_better"] is True and d["value"] > 0
    assert d["config"] == bench.workload_config("d2_256x256_i64_add_k16", (256, 256), (16, 16), "add", 1)
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0


def test_reference_other_ranks_print_nothing():
    r = _run({"RANK": "1", "LOCAL_RANK": "1", "WORLD_SIZE": "2"}, "--gpus", "2", "--steps", "1",
             "--warmup", "0", "--workload", "d2_256x256_i64_add_k16")
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""
