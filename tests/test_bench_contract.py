"""bench.py's one-line JSON contract: the reference arm (the CPU oracle, no
GPU) on CPU, and the default arm on the GPU, each run as its own process
the way the round-end runs launch them."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
BASE_KEYS = {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
             "vs_baseline", "dtype", "data", "config", "e2e"}


def _run(args, timeout):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True, text=True,
                       timeout=timeout, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    return json.loads(lines[0])


def test_reference_arm_line():
    j = _run(["--impl", "reference", "--steps", "1", "--warmup", "0"], timeout=300)
    assert BASE_KEYS <= set(j)
    assert j["impl"] == "reference" and j["value"] > 0 and j["higher_is_better"] is True
    assert j["config"]["workload"] == "latent_192x32x48_k3_s1024"
    assert j["cpu_baseline"]["kind"] == "oracle" and j["cpu_baseline"]["cores"] >= 1
    host = j["cpu_baseline"]["host"]
    assert host["nproc"] == j["cpu_baseline"]["cores"] and host["model"]
    assert j["cpu_baseline"]["single_thread"]["cores"] == 1 and j["cpu_baseline"]["single_thread"]["value"] > 0
    sys.path.insert(0, ROOT)
    import bench
    assert j["config"] == bench.workload_config(294912, 3, 1024)
    assert j["e2e"]["h2d_bytes_per_step"] == 0 and j["e2e"]["d2h_bytes_per_step"] == 0


@pytest.mark.gpu
def test_default_arm_line():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    j = _run(["--steps", "20", "--warmup", "3", "--no-cpu-baseline", "--no-throughput", "--e2e-steps", "4"],
             timeout=900)
    assert BASE_KEYS <= set(j)
    assert j["n_gpus"] == 1 and j["steps"] == 20 and j["warmup"] >= 3 and j["scaling"] == "weak"
    assert j["value"] > 0 and abs(j["value"] - 294912 / (j["ms_per_step"] * 1e-3) / 1e6) < 1e-6 * j["value"]
    assert j["config"]["workload"] == "latent_192x32x48_k3_s1024" and "l2" in j["config"]
    sys.path.insert(0, ROOT)
    import bench
    assert j["config"] == bench.workload_config(294912, 3, 1024)   # the reference arm prints the same dict
    e = j["e2e"]
    assert e["value"] > 0 and e["h2d_bytes_per_step"] > 0 and e["d2h_bytes_per_step"] > 0
    r = j["roofline"]
    assert {"bound", "achieved", "peak", "unit", "frac", "traffic"} <= set(r)
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-9 and 0 < r["frac"] < 1
    assert r["peak_source"].startswith("measured") and 0.5 * r["peak_derived"] < r["peak"] < 1.2 * r["peak_derived"]
    assert j["gpu_launches"] == 5 * 20
    assert j["serial"]["value"] > 0 and set(j["concurrent_decodes"]) == {"2", "3"}
    assert j["table_coder"]["stream_identical"] is True
