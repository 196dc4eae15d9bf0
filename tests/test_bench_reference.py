"""The reference arm of bench.py on the CPU: the oracle timed on a bounded
sample prints one JSON line with the contract's keys, and under torchrun only
rank 0 runs it (the other ranks exit 0 without work)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CMD = [sys.executable, "bench.py", "--impl", "reference", "--workload", "uniform-16k", "--steps", "2",
       "--warmup", "1"]


def _env(**kw):
    env = {k: v for k, v in os.environ.items() if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK")}
    env.update(kw)
    return env


def test_reference_line_keeps_the_contract():
    r = subprocess.run(CMD, cwd=ROOT, env=_env(), capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    d = json.loads(r.stdout.strip().splitlines()[-1])
    assert d["impl"] == "reference" and d["metric"] == "input Mpoints/s" and d["unit"] == "Mpoints/s"
    assert d["value"] > 0 and d["higher_is_better"] is True and d["n_gpus"] == 1
    assert d["steps"] == 2 and d["warmup"] >= 3  # at least three warm-up steps, whatever was asked
    assert d["config"]["workload"] == "uniform-16k" and d["data"] == "synthetic"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["vs_baseline"] is None


def test_other_ranks_exit_without_work():
    r = subprocess.run(CMD, cwd=ROOT, env=_env(RANK="1", LOCAL_RANK="1", WORLD_SIZE="2"),
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""
