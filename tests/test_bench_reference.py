"""The benchmark's reference arm (the CPU oracle on the benchmark workload)
keeps the JSON-line contract, alone and under torchrun with two ranks (rank
0 prints the one line, timed on all the host cores it may use; the other
rank exits without work). Runs on the CPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KEYS = {"impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
        "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
        "cpu_baseline", "e2e"}


def run(cmd, env=None):
    p = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, p.stdout
    return json.loads(lines[0])


def check(d, n):
    assert KEYS <= set(d)
    assert d["impl"] == "reference" and d["metric"] == "spgemm_gflops"
    assert d["unit"] == "GFLOP/s" and d["higher_is_better"] is True
    assert d["n_gpus"] == n and d["steps"] == 1 and d["vs_baseline"] is None
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["config"]["workload"] == "rmat20_ef16_AxA_plus_StAS"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1
    assert cb["cores"] == len(os.sched_getaffinity(0))
    assert d["e2e"] == {"value": d["value"], "unit": "GFLOP/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_reference_arm_one_process():
    check(run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
               "--warmup", "0"]), 1)


def test_reference_arm_under_torchrun():
    env = dict(os.environ, OMP_NUM_THREADS="1")
    d = run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
             "--master-addr", "127.0.0.1", "--master-port", "29561", "bench.py", "--impl",
             "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"], env=env)
    check(d, 2)
