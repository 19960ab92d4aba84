"""bench.py's roofline arithmetic (CPU only): algorithmic work per family call, the peaks it is
divided by, and the whole-job rate of replicas, checked against numbers worked out by hand."""
import json
import os
from types import SimpleNamespace

import pytest

import bench

W = SimpleNamespace(n_traj=1024, nx=1024, nR=512)
PEAKS = {"hbm_gbs": 6700.0, "bf16_tflops_sustained": 1700.0}


def test_double_float_ceiling():
    # 152 SMs x 128 FP32 lanes x 2.07 GHz, 8 flops per 39 operations
    assert bench.DF64_TFLOPS == pytest.approx(152 * 128 * 2.07e9 * 8 / 39 / 1e12)
    assert bench.DF64_TFLOPS == pytest.approx(8.2613, rel=1e-4)


def test_cholesky_two_matrices_per_call():
    # 2 x (4/3) N^3 = 2.863e9 flop in 1.3 ms -> 2.202 TFLOP/s
    r = bench.roofline({"cholesky": (130.0, 100)}, W, 15, "tf32x3", PEAKS)
    assert r["kernel"] == "cholesky" and r["bound"] == "alu"
    assert r["achieved"] == pytest.approx(2 * 4 / 3 * 1024 ** 3 / 1.3e-3 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / bench.DF64_TFLOPS)
    assert r["traffic"] == pytest.approx(193.6e6)
    frozen = bench.roofline({"cholesky": (130.0, 100)}, W, 15, "tf32x3", PEAKS, "df64", 1)
    assert frozen["achieved"] == pytest.approx(r["achieved"] / 2)


def test_fp64_peaks_for_fp64_work():
    r = bench.roofline({"cholesky": (130.0, 100)}, W, 15, "tf32x3", PEAKS, "fp64")
    assert r["peak"] == bench.NOMINAL_FP64_TFLOPS and r["traffic"] is None
    r = bench.roofline({"assemble": (100.0, 100)}, W, 21, "fp64", PEAKS)
    assert r["bound"] == "alu" and r["peak"] == bench.NOMINAL_FP64_TFLOPS


def test_split_tensor_ceiling():
    # 4 N^2 (k+1)(nx+nR) flop; TF32 peak = BF16 sustained x 1.1/2.25, three products
    r = bench.roofline({"assemble": (92.0, 100)}, W, 15, "tf32x3", PEAKS)
    work = 4.0 * 1024 ** 2 * 16 * 1536
    assert r["achieved"] == pytest.approx(work / 0.92e-3 / 1e12)
    assert r["peak"] == pytest.approx(1700.0 * 1.1 / 2.25 / 3)
    b = bench.roofline({"assemble": (92.0, 100)}, W, 15, "bf16x3", PEAKS)
    assert b["peak"] == pytest.approx(1700.0 / 3)


def test_dominant_family_and_rate():
    r = bench.roofline({"cholesky": (130.0, 100), "assemble": (92.0, 100)}, W, 15, "tf32x3",
                       PEAKS)
    assert r["kernel"] == "cholesky"
    assert bench.whole_job_rate(4, 1024 * 100, 0.31) == pytest.approx(4 * 102400 / 0.31)


def test_measured_peaks_file_has_the_keys_bench_reads():
    path = os.path.join(bench.ROOT, "MEASURED_PEAKS.json")
    if not os.path.exists(path):
        pytest.skip("MEASURED_PEAKS.json is written per pool")
    p = json.load(open(path))
    assert p["hbm_gbs"] > 0 and p["bf16_tflops_sustained"] > 0


def test_a_failing_extra_record_keeps_the_line():
    """An extra record that raises is reported in the line as an error; the others still run."""
    out = {"value": 1.0}

    def boom():
        raise RuntimeError("no device")

    assert not bench.record(out, "serving", boom)
    assert bench.record(out, "exact2d", lambda a, b: {"value": a + b}, 2, 3)
    assert out["serving"] == {"error": "RuntimeError: no device"}
    assert out["exact2d"] == {"value": 5} and out["value"] == 1.0
    json.dumps(out)
