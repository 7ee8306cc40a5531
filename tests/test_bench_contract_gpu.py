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
    # 20 timed steps of the N = 256 case (a few ms): the clock record still has
    # samples, taken from before the warm-up to the end of the soak after it
    d = run_bench("--case", "small", "--steps", "20", "--warmup", "3", "--latency-samples", "20",
                  "--no-serving", "--no-learned", "--no-large", "--no-packed")
    assert d["metric"] and d["unit"] == "Gpixel-frames/s" and d["higher_is_better"] is True
    assert d["n_gpus"] == 1 and d["steps"] == 20 and d["warmup"] == 3
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
    assert d["clocks"]["samples"] >= 3
    assert d["gpu_launches"] >= 20  # at least one library launch per timed step
    c1 = d["plain_c1"]
    assert c1["eager"]["us_per_call"] > 0 and c1["graph"]["us_per_call"] > 0
    assert c1["latency_us"]["p99"] >= c1["latency_us"]["p50"] > 0


def test_reference_arm_prints_its_line():
    d = run_bench("--impl", "reference", "--steps", "1", "--warmup", "3")
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "Gpixel-frames/s"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    # ms_per_step is the measured time of one timed step (a band of rows), so
    # steps x ms_per_step is time the run really spent
    assert d["steps"] >= 1 and 0 < d["ms_per_step"] < d["full_frame_ms_per_step_extrapolated"]


def test_row_split_arm_prints_a_strong_scaling_line():
    # one rank: the band is the whole 4096x4096 frame (N = 64 in the small case)
    d = run_bench("--split", "rows", "--case", "small", "--steps", "20", "--warmup", "3", "--no-cpu-baseline")
    assert d["scaling"] == "strong" and d["n_gpus"] == 1 and d["steps"] == 20
    assert d["config"]["band_rank0"] == [0, 4096] and d["value"] > 0
    r = d["roofline"]
    assert r["bound"] == "hbm" and abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-9
    assert d["e2e"]["h2d_bytes_per_step"] == 4096 * 4096 * 2 and d["gpu_launches"] >= 20
    assert d["clocks"] and d["clocks"]["samples"] >= 3
