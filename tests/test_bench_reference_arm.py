"""The reference arm of bench.py (the oracle on the host cores) keeps the
JSON contract: one line with impl, metric, unit, value, steps, warm-up,
a cpu_baseline describing the run and an e2e entry with no copies.  Runs on
the small 48^3 workload, on the CPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--config", "blobs48", "--steps", "2",
                        "--warmup", "1"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 1 and d["steps"] == 2 and d["warmup"] == 1
    assert d["unit"] == "voxels/s" and d["higher_is_better"] is True and d["value"] > 0
    assert d["metric"].startswith("invasion voxels/s")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"] == "blobs48"


def test_reference_arm_under_two_ranks_prints_once():
    base = [sys.executable, "bench.py", "--impl", "reference", "--config", "blobs48", "--steps", "1", "--warmup", "0",
            "--gpus", "2"]
    outs = []
    for rank in (0, 1):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank))
        r = subprocess.run(base, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
        assert r.returncode == 0, r.stderr[-2000:]
        outs.append([ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")])
    assert len(outs[0]) == 1 and outs[1] == []
    assert json.loads(outs[0][0])["n_gpus"] == 2
