"""The reference arm of bench.py (the float64 oracle timed on the host cores)
keeps the benchmark line's contract; it needs no GPU, so it is checked here."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CMD = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
       "--warmup", "0", "--cpu-seconds", "1"]


def _run(env_extra=None):
    env = dict(os.environ, **(env_extra or {}))
    r = subprocess.run(CMD, capture_output=True, text=True, timeout=600, cwd=ROOT, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    return r.stdout


def test_reference_line_has_the_contract_keys():
    sys.path.insert(0, ROOT)
    import bench
    lines = [ln for ln in _run().splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == "MLUPS" and d["higher_is_better"] is True
    assert d["n_gpus"] == 1 and d["steps"] == 2 and d["warmup"] == 0
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["config"] == bench.workload_config(2048, 4096, 1)   # the same workload as our arm
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] > 0 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_prints_only_on_rank_0():
    assert _run({"RANK": "1", "WORLD_SIZE": "2"}).strip() == ""
