"""bench.py's JSON line on a GPU: every key of the contract, with values of the right kind."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_bench(*args):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True, text=True,
                         check=True, cwd=ROOT, timeout=600)
    return json.loads(out.stdout.strip().splitlines()[-1])


def test_quick_line_has_the_contract_keys():
    d = run_bench("--quick", "--L", "16", "--steps", "3", "--warmup", "3")
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "roofline", "gpu_launches", "clocks", "launch_ms"):
        assert k in d, k
    assert d["n_gpus"] == 1 and d["steps"] == 3 and d["warmup"] == 3 and d["higher_is_better"] is True
    assert d["value"] > 0 and d["unit"] == "GB/s" and d["dtype"] == "f64" and d["gpu_launches"] == 3
    r = d["roofline"]
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert k in r, k
    assert r["bound"] == "alu" and 0 < r["frac"] < 1.2 and "hbm" in r
    # the FP64 pipe's rate measured on the device, beside the derived peak
    assert 0.3 < r["peak_measured"] < 3.0 and 0 < r["frac_of_measured"] < 1.3
    assert "workload" in d["config"] and d["config"]["lattice"] == "16^4"
    assert set(d["clocks"]) >= {"sm_mhz", "sm_max_mhz", "reasons"}


def test_launch_override_and_reduced_dtype():
    d = run_bench("--quick", "--L", "16", "--steps", "3", "--warmup", "3", "--dtype", "f16",
                  "--launch", "block=128,tile_sites=32,stages=3,ctas_per_sm=2,threads_per_link=3")
    assert d["roofline"]["bound"] == "hbm" and d["config"]["tuned"] is False
    assert d["config"]["launch_cfg"]["threads_per_link"] == 3 and d["config"]["launch_cfg"]["tile_sites"] == 32


def test_shard_mode_line():
    """--shard at N = 1: the one slab is the whole lattice; the line says strong scaling."""
    d = run_bench("--quick", "--shard", "--L", "16", "--steps", "3", "--warmup", "3")
    assert d["scaling"] == "strong" and d["value"] > 0 and d["config"]["parallelism"] == "single GPU"


def test_form_and_stride_lines():
    """--form times any tuner-named form alone (bytes, flops and the kernel's template from its
    repr pair); --stride times padded sites through the padded kernel."""
    d = run_bench("--quick", "--L", "16", "--steps", "3", "--warmup", "3", "--form", "f64-2to18-aos-f32pair")
    assert d["config"]["form"] == "f64-2to18-aos-f32pair" and "384 B read + 576 B written" in d["config"]["workload"]
    assert d["roofline"]["bound"] == "hbm" and "PairF64Op<6,3>" in d["roofline"]["kernel"]
    assert d["dtype"].startswith("f32x2") and d["gpu_launches"] == 3
    d = run_bench("--quick", "--L", "16", "--steps", "3", "--warmup", "3", "--form", "f64-2to18-aos")
    assert d["roofline"]["bound"] == "alu" and "NativeOp<F64,6,3>" in d["roofline"]["kernel"]
    assert abs(d["gflops"] / (d["site_updates_per_s"] / 1e9) - 1056) < 0.5
    d = run_bench("--quick", "--L", "16", "--steps", "3", "--warmup", "3", "--arith", "f32pair", "--stride", "640")
    assert d["config"]["form"].endswith("-p640") and d["roofline"]["kernel"].endswith("AOS, true>")
    assert "576 B read + 576 B written" in d["config"]["workload"] and d["value"] > 0
