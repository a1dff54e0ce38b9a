"""bench.py's output contract, checked on the CPU: the reference arm (the
oracle timed on the host cores) prints one JSON line with every key the
measurement contract asks for, and the GPU arm fails loudly without a GPU
instead of falling back to the CPU."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_bench(*args, timeout=300):
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT,
                          capture_output=True, text=True, timeout=timeout)


def test_reference_arm_prints_the_contract_line():
    r = run_bench("--impl", "reference", "--workload", "c2s", "--steps", "1", "--warmup", "0")
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["unit"] == "eigenpairs/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["ms_per_step"] > 0 and d["n_gpus"] == 1
    assert "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    # a step is a timed iteration of the oracle's own solve; the solve time is
    # an explicit projection of it, and a step fits in the run's wall time
    pr = d["projection"]
    assert pr["iterations_per_solve"] > 0
    assert abs(d["value"] - 64 / (d["ms_per_step"] / 1e3 * pr["iterations_per_solve"])) <= 1e-9 * d["value"]
    assert d["ms_per_step"] / 1e3 * (d["steps"] + d["warmup"]) <= d["wall_s"] + 1e-6


def test_gpu_arm_fails_loudly_without_a_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    r = run_bench("--workload", "c2s", "--steps", "1", "--warmup", "3", timeout=120)
    assert r.returncode != 0
    assert not [l for l in r.stdout.splitlines() if l.startswith("{")]
