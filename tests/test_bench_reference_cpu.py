"""The benchmark's reference arm: the oracle timed on the host cores, printing the
same JSON line as the GPU arm (metric, unit, direction, config of the workload) with
impl = reference, its cpu_baseline description and an e2e object without transfers.
Under torchrun only rank 0 works and prints; the other ranks exit 0 silently.  Run
on the small 64 x 128 workload so that it takes seconds."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CMD = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "cfg1_axisym_64x128",
       "--steps", "2", "--warmup", "3"]


def _run(env_extra):
    env = dict(os.environ, **env_extra)
    return subprocess.run(CMD, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_reference_arm_line():
    r = _run({"RANK": "0"})
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == "Mcell-steps/s" and d["unit"] == "Mcell-steps/s" and d["higher_is_better"] is True
    assert d["steps"] == 2 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["config"]["workload"] == "cfg1_axisym_64x128" and d["config"]["cells"] == 64 * 128
    assert d["value"] > 0.0 and d["ms_per_step"] > 0.0
    assert abs(d["value"] - 64 * 128 / (d["ms_per_step"] * 1e-3) / 1e6) < 1e-9 * d["value"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_silent():
    r = _run({"RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""


def test_reference_arm_default_3d_workload_samples_a_downscale():
    """The default workload (3D 256^3, plain FP64) is beyond the oracle's direct
    solves: each reference step is one oracle step of the same case on 20^3 cells,
    the value counts those cells, and the line says so."""
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1", "--warmup", "3"]
    r = subprocess.run(cmd, cwd=ROOT, env=dict(os.environ, RANK="0"), capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    d = json.loads([ln for ln in r.stdout.splitlines() if ln.strip()][-1])
    assert d["config"]["workload"] == "cfg3_cart3d_256_fp64" and d["config"]["cells"] == 256 ** 3
    assert d["dtype"] == "f64"
    assert abs(d["value"] - 20 ** 3 / (d["ms_per_step"] * 1e-3) / 1e6) < 1e-9 * d["value"]
    assert "20^3" in d["cpu_baseline"]["sample"]
