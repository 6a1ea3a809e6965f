"""bench.py on the CPU: the reference arm times the FP64 oracle on a
bounded pair sample and prints one JSON line with the keys of the bench
contract (under torchrun, ranks other than 0 exit without output); the GPU
arm has no CPU fallback and fails without a GPU."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(extra_env=None):
    env = dict(os.environ, **(extra_env or {}))
    cmd = [sys.executable, "bench.py", "--impl", "reference", "--workload", "yule1k_n64",
           "--steps", "1", "--warmup", "1", "--ref-seconds", "1"]
    return subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)


def test_reference_line():
    p = _run()
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 1
    assert d["config"]["workload"] == "yule1k_n64"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"],
                        "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_other_ranks_print_nothing():
    p = _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert p.returncode == 0, p.stderr[-2000:]
    assert p.stdout.strip() == ""


def test_gpu_arm_fails_loudly_without_a_gpu():
    # no CPU fallback: without a GPU the default arm exits non-zero and prints no line
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    p = subprocess.run([sys.executable, "bench.py", "--steps", "1", "--warmup", "1", "--workload", "yule1k_n64"],
                       cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert p.returncode != 0
    assert p.stdout.strip() == ""


def test_striped_loop_rate_on_a_slice():
    # the plain striped CPU loop of the CPU-baseline leg: one stripe per host
    # thread on [0, k), the step's methods; on the first samples of the table
    # when one stripe of the whole table is too much work
    import bench
    import oracle
    from synth import workload
    tree_s, table_s = workload("yule1k_n64")
    rate, used, k, dt, n_used = bench.oracle_striped_rate(tree_s, table_s)
    assert rate > 0 and dt > 0 and n_used == table_s.n_samples
    assert k == min(table_s.n_samples // 2, oracle.host_cores()) and used == k
    rate, used, k, dt, n_used = bench.oracle_striped_rate(tree_s, table_s, max_updates_per_thread=1.0)
    assert n_used == min(256, table_s.n_samples) and rate > 0


def test_sub_table_keeps_the_first_samples():
    import bench
    from synth import workload
    _, t = workload("yule1k_n64")
    s = bench.sub_table(t, 10)
    assert s.n_samples == 10 and s.n_features == t.n_features
    assert (s.dense() == t.dense()[:10]).all()
