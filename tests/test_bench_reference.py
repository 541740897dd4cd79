"""bench.py --impl reference on CPU: the oracle arm's one JSON line (the same
metric, unit and config keys as the CUDA arm, the oracle described as its own
cpu_baseline, an e2e with no copies), rank 0 alone under a multi-rank launch,
and the unavailable line for an ensemble workload."""
import json
import os
import subprocess
import sys

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_bench(*args, env=None):
    oracle.build()
    e = dict(os.environ)
    e.update(env or {})
    e.setdefault("OMP_NUM_THREADS", "2")
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", *args],
                          cwd=ROOT, env=e, capture_output=True, text=True, timeout=300)


def test_reference_arm_prints_one_line_of_the_contract():
    p = run_bench("--workload", "brownian_64", "--steps", "2", "--warmup", "1")
    assert p.returncode == 0, p.stderr
    lines = [ln for ln in p.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["unit"] == "MLUPS" and d["higher_is_better"] is True
    assert d["n_gpus"] == 1 and d["steps"] == 2 and d["warmup"] == 1
    assert d["dtype"] == "f64" and d["data"] == "synthetic"
    assert d["config"]["workload"] == "brownian_64^3_256p"
    assert d["config"]["nodes_per_rank"] == 64 ** 3 and d["config"]["particles_per_rank"] == 256
    assert d["value"] > 0
    # value = nodes per second over the timed steps, in millions
    assert d["value"] == pytest.approx(64 ** 3 / (d["ms_per_step"] * 1e-3) / 1e6, rel=1e-9)
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["unit"] == "MLUPS"
    assert cb["cores"] >= 1 and "oracle steps" in cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert d["vs_baseline"] is None


def test_reference_arm_runs_on_rank_0_only():
    p = run_bench("--workload", "brownian_64", "--steps", "1", "--warmup", "1",
                  env={"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert p.returncode == 0, p.stderr
    assert p.stdout.strip() == ""


def test_reference_arm_states_what_it_does_not_time():
    p = run_bench("--workload", "ensemble_68", "--steps", "1", "--warmup", "1")
    assert p.returncode == 0, p.stderr
    d = json.loads(p.stdout.strip())
    assert d["impl"] == "reference" and d["unavailable"]
