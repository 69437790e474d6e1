"""bench.py's reference arm on the host cores: one JSON line with the contract's keys, on the same
workload, metric and unit as the GPU arm (run here on the 589-node bucket3_depth6 game)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                        "bucket3_depth6", "--steps", "3", "--warmup", "1"], capture_output=True, text=True,
                       timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 1 and d["steps"] == 3 and d["warmup"] == 1
    assert d["unit"] == "node-updates/s" and d["higher_is_better"] is True and d["value"] > 0
    assert d["config"]["workload"].startswith("bucket3_depth6 (seed 0): 6 ordered deals")
    assert d["config"]["nodes"] == 589
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["gpu_launches"] == 0


def test_every_named_workload_has_its_description():
    sys.path.insert(0, ROOT)
    import bench
    import gamegen

    assert set(bench.WORKLOAD_TEXT) == set(gamegen.CONFIGS)
