"""bench.py's output contract on a small run: one JSON line with the metric,
the whole-step value and timing, the roofline of the dominant kernel, the
CPU-oracle baseline, the end-to-end number through host buffers, the clocks
sampled during the timed region and the count of library launches; and the
reference arm (the oracle) with its own line."""
import json
import os
import subprocess
import sys

import pytest
import torch

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def run_bench(*args):
    out = subprocess.run([sys.executable, "bench.py", *args], cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1, out.stdout[-2000:]
    return json.loads(lines[0])


def test_cuda_arm_prints_the_contract_line():
    # 5000 steps of the N = 256 case (~0.1 ms each) outlast several clock samples (every 100 ms)
    d = run_bench("--case", "small", "--steps", "5000", "--warmup", "3", "--latency-samples", "20",
                  "--no-serving", "--no-learned", "--no-large", "--no-packed")
    assert d["metric"] and d["unit"] == "Gpixel-frames/s" and d["higher_is_better"] is True
    assert d["n_gpus"] == 1 and d["steps"] == 5000 and d["warmup"] == 3
    assert d["value"] > 0 and d["ms_per_step"] > 0 and d["scaling"] == "weak"
    assert "workload" in d["config"] and d["dtype"] and d["data"]
    r = d["roofline"]
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak"] > 0
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-9
    assert "traffic" in r  # the ncu figure for this kernel and workload, or null
    c = d["cpu_baseline"]
    assert c["kind"] == "oracle" and c["value"] > 0 and c["cores"] >= 1 and c["sample"]
    e = d["e2e"]
    assert e["value"] > 0 and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] > 0 and e["d2h_bytes_per_step"] > 0
    assert d["clocks"] and {"sm_mhz", "sm_max_mhz", "reasons"} <= set(d["clocks"])
    assert d["gpu_launches"] >= 5000  # at least one library launch per timed step


def test_reference_arm_prints_its_line():
    d = run_bench("--impl", "reference", "--steps", "1", "--warmup", "3")
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "Gpixel-frames/s"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
