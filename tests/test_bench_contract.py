"""The reference arm of bench.py on CPU: the literal FP64 oracle timed on the
host cores prints one JSON line with the benchmark's metric, its own
cpu_baseline and an end-to-end figure with no host-device traffic; under a
multi-rank launch only rank 0 prints."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(n, steps, warmup, env_extra=None):
    env = dict(os.environ)
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        env.pop(k, None)
    env.update(env_extra or {})
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--n", str(n),
                        "--steps", str(steps), "--warmup", str(warmup)],
                       capture_output=True, text=True, timeout=300, env=env, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    return [ln for ln in r.stdout.splitlines() if ln.strip()]


def test_reference_arm_line():
    lines = _run(192, 2, 1)
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"].startswith("evals/s")
    assert d["unit"] == "evals/s" and d["higher_is_better"] is True
    assert d["n_gpus"] == 1 and d["steps"] == 2 and d["warmup"] == 1
    assert d["value"] > 0
    # two evaluations (FP32 and FP64 inputs) per step
    assert abs(d["value"] * d["ms_per_step"] - 2000.0) < 1e-6 * 2000.0
    assert "192x192" in d["config"]["workload"] and d["config"]["evals_per_step"] == 2
    cpu = d["cpu_baseline"]
    assert cpu["kind"] == "oracle" and cpu["value"] == d["value"] and cpu["unit"] == "evals/s"
    assert cpu["cores"] >= 1 and cpu["nproc"] >= 1 and cpu["cpu_model"]
    assert cpu["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    assert d["vs_baseline"] is None


def test_reference_arm_other_ranks_print_nothing():
    assert _run(64, 1, 0, {"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}) == []
