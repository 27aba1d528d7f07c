"""bench.py's reference arm (the FP64 oracle timed on the host cores): one JSON line with the
contract's keys on rank 0, nothing on the other ranks."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(env_extra):
    env = dict(os.environ, **env_extra)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "2cam",
                           "--steps", "2", "--warmup", "1"], cwd=ROOT, env=env, capture_output=True, text=True,
                          timeout=600)


def test_reference_arm_prints_the_contract_line():
    p = _run({"RANK": "0"})
    assert p.returncode == 0, p.stderr
    line = json.loads(p.stdout.strip().splitlines()[-1])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["steps"] == 2 and line["warmup"] == 1 and line["value"] > 0
    assert line["config"]["workload"] and line["higher_is_better"] is True
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == line["value"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_exit_quietly():
    p = _run({"RANK": "1"})
    assert p.returncode == 0, p.stderr
    assert p.stdout.strip() == ""


import pytest  # noqa: E402


@pytest.mark.gpu
def test_gpu_arm_prints_the_contract_line():
    """The product arm on the small 2-camera workload: the keys of the bench contract, with the
    roofline, end-to-end, clock and launch-count fields filled in."""
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--workload", "2cam", "--steps", "5",
                        "--warmup", "3", "--no-plain", "--no-fp16", "--no-batch", "--no-lorb", "--no-seam",
                        "--no-accuracy", "--no-backward", "--e2e-steps", "3"], cwd=ROOT, capture_output=True,
                       text=True, timeout=900)
    assert p.returncode == 0, p.stderr[-2000:]
    line = json.loads(p.stdout.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e", "clocks", "gpu_launches"):
        assert k in line, k
    assert line["n_gpus"] == 1 and line["steps"] == 5 and line["warmup"] == 3 and line["value"] > 0
    assert line["config"]["workload"].startswith("2cam")
    rf = line["roofline"]
    assert rf["bound"] in ("hbm", "tensor", "alu") and rf["peak"] > 0 and rf["achieved"] > 0
    assert abs(rf["frac"] - rf["achieved"] / rf["peak"]) < 1e-9
    e2e = line["e2e"]
    assert e2e["value"] > 0 and e2e["h2d_bytes_per_step"] > 0 and e2e["d2h_bytes_per_step"] > 0
    assert line["gpu_launches"] >= 5 and line["cpu_baseline"]["kind"] == "oracle"
    assert "sm_mhz" in line["clocks"] and "reasons" in line["clocks"]
    fm = line["frame_ms"]
    assert fm["frames"] == 5 and 0 < fm["p10"] <= fm["median"] <= fm["p90"]
