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


def test_oracle_sample_is_a_corner_cube_of_large_images(monkeypatch):
    """Images above the full-pass limit are timed on their corner cube, with
    the workload's faces and radii of the cube's own largest distance."""
    sys.path.insert(0, ROOT)
    import numpy as np

    import bench
    import oracle as O
    from paper_2101_03240_gb300 import synth
    w = synth.c1_blobs48()
    sw, levels, desc = bench.oracle_sample(w, 40)
    assert sw.image is w.image and "full pass" in desc
    monkeypatch.setattr(bench, "ORACLE_FULL_MAX_VOXELS", 1000)
    monkeypatch.setattr(bench, "ORACLE_CROP_EDGE", 20)
    sw, levels, desc = bench.oracle_sample(w, 40)
    assert sw.image.shape == (20, 20, 20) and np.array_equal(sw.image, w.image[:20, :20, :20])
    assert sw.inlet == w.inlet and sw.outlet == w.outlet and sw.name == "blobs48_corner20"
    d = O.edt(sw.image)
    assert levels == synth.mio_levels(int(d[sw.image > 0].max()), 40)


def test_traffic_is_null_when_sources_or_workload_differ(monkeypatch):
    """The bench line's ncu traffic holds only for the captured workload and
    the sources it was captured on (checked by their SHA-256)."""
    sys.path.insert(0, ROOT)
    import bench
    for c, t in bench.NCU_TRAFFIC.items():
        assert t["workload"] == "blobs512" and t["src"] and t["bytes_per_voxel"] > 0
        assert bench.traffic_per_launch(c, 1000) == t["bytes_per_voxel"] * 1000
        assert bench.traffic_per_launch(c, 1000, "spheres200") is None
    assert bench.traffic_per_launch("no_such_class", 1000) is None
    monkeypatch.setattr(bench, "source_sha16", lambda rel: "0" * 16)
    assert all(bench.traffic_per_launch(c, 1000) is None for c in bench.NCU_TRAFFIC)
