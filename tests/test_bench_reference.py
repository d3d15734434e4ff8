"""The benchmark's reference arm (the oracle on the host cores) on a small field:
one JSON line with the contract's keys on rank 0, nothing on the other ranks."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ARGS = [sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0",
        "--shape", "32", "32", "32", "--oracle-sample", "8192"]


def _run(env_extra):
    env = dict(os.environ)
    env.update(env_extra)
    return subprocess.run(ARGS, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_reference_arm_line():
    r = _run({"RANK": "0", "WORLD_SIZE": "1"})
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["value"] > 0 and d["unit"] == "GB/s" and d["higher_is_better"] is True
    assert d["config"]["workload"].startswith("grf3d_32x32x32")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert "sample" in cb
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_silent():
    r = _run({"RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_reference_sample_sizing():
    """The reference arm's sample is whole 64-value blocks between 2^16 and
    2^24 values per field, smaller when more steps share the time budget."""
    sys.path.insert(0, ROOT)
    import numpy as np

    import bench

    rng = np.random.default_rng(0)
    A = rng.normal(size=1 << 18).astype(np.float32)
    B = rng.normal(size=1 << 18).astype(np.float32)
    few, many = bench.reference_sample(A, B, 1), bench.reference_sample(A, B, 100_000)
    for n in (few, many):
        assert n % 64 == 0 and (1 << 16) <= n <= (1 << 24)
    assert many == 1 << 16 and few >= many
