"""Host side of bench.py (no GPU): the fixed algorithmic work counts, the peak
arithmetic and the reference arm's JSON line."""

import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_flop_counts_follow_the_counting_convention():
    # per-update flops of predictor, volume, local and neighbour flux at N = 5,
    # and the totals at N = 3, 4, 5, as tabulated for the element update
    f5 = bench.flops_per_update(5)
    assert (f5["pred"], f5["vol"], f5["loc"], f5["nb"]) == (193104, 133056, 182952, 214704)
    assert f5["total"] == 723816
    assert bench.flops_per_update(4)["total"] == 310896
    assert bench.flops_per_update(3)["total"] == 119376
    # kernel split and the tensor-core share of the local kernel
    assert f5["local_kernel"] + f5["neighbour_kernel"] == f5["total"]
    gemm_pred = sum(54 * a * b for a, b in ((35, 56), (20, 35), (10, 20)))
    assert f5["local_tensor"] == gemm_pred + 54 * 56 * 35 + 72 * 21 * 56


def test_byte_counts_are_the_arrays_moved():
    b = bench.bytes_per_update(5, 4)
    dofs, traces = 2 * 9 * 56 * 4, 4 * 9 * 21 * 4
    assert b["local_kernel"] == dofs + traces
    assert b["neighbour_kernel"] == dofs + 2 * traces
    padded = 4 * 192 * 4  # face blocks padded to a multiple of 4 floats
    assert b["local_tc_kernel"] == dofs + padded + 16 * 4
    assert b["neighbour_tc_kernel"] == dofs + 2 * padded + 4 * 32 + 16 * 4


def test_peak_arithmetic():
    units = {"tf32_tensor_tflops": 1200.0, "fp32_fma_tflops": 76.0, "fp64_fma_tflops": 1.2}
    # measured rates: a 3xTF32 product costs three TF32 MMAs
    assert bench.tf32x3_peak_tflops({"bf16_tflops": 1.0}, units)[0] == pytest.approx(400.0)
    assert bench.alu_peak_tflops(False, 2070.0, units)[0] == pytest.approx(76.0)
    assert bench.alu_peak_tflops(True, 2070.0, units)[0] == pytest.approx(1.2)
    # without them: the burst bf16 rate times the nominal tf32 ratio; lanes x clock; nominal FP64
    assert bench.tf32x3_peak_tflops({"bf16_tflops": 2250.0})[0] == pytest.approx(2250.0 * 1.1 / 2.25 / 3.0)
    assert bench.alu_peak_tflops(False, 2070.0, None, 148)[0] == pytest.approx(148 * 128 * 2 * 2.07e9 / 1e12)
    assert bench.alu_peak_tflops(True, 2070.0)[0] == pytest.approx(1.25)


def test_measured_peaks_file_is_read():
    u = bench.unit_peaks()
    assert u is not None and u["tf32_tensor_tflops"] > 0 and u["fp32_fma_tflops"] > 0 and u["fp64_fma_tflops"] > 0


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "1"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
