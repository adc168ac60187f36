"""bench.py's reference arm (the CPU oracle) and its JSON line, on the host:
the contract keys, complete measured oracle steps, and the silent non-zero
ranks."""
import json
import math
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(args, env=None):
    e = dict(os.environ)
    e.update(env or {})
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, cwd=ROOT, env=e,
                       capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    return [ln for ln in p.stdout.splitlines() if ln.strip()]


def test_reference_arm_prints_one_contract_line():
    sys.path.insert(0, ROOT)
    import bench
    lines = _run(["--impl", "reference", "--n", "32", "--steps", "2", "--warmup", "1"])
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["higher_is_better"] is False and d["n_gpus"] == 1
    assert d["steps"] == 2 and d["warmup"] == 1
    assert d["value"] > 0 and math.isfinite(d["value"])
    assert d["ms_per_step"] == d["value"] * 1e3
    assert d["config"]["grid"] == [32, 32, 32]
    assert "smaller than L2" in d["config"]["l2"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert "32x32x32" in cb["sample"] and "not scaled" in cb["sample"]
    # each timed step is a complete oracle step, so the line's per-step times
    # add up to no more than the run took
    assert len(d["per_step_s"]) == 2
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_reference_arm_prints_nothing_on_other_ranks():
    lines = _run(["--impl", "reference", "--n", "32", "--steps", "1", "--warmup", "0"],
                 env={"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert lines == []
