"""Host logic of bench.py's report, on CPU: the roofline block of the
dominant kernel class (achieved = algorithmic work per launch / average
launch time, frac = achieved / peak, the peak taken from the measured
numbers, the DRAM traffic scaled from the stored ncu captures), and the
clock summary parsed from nvidia-smi samples."""
import sys
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]
sys.path.insert(0, str(ROOT))

import bench  # noqa: E402

PEAKS = {"hbm_gbs": 6482.7, "bf16_tflops": 1810.3, "bf16_tflops_sustained": 1408.1}


def _kst(**classes):
    names = ("trsv32", "trsv64", "trmv64", "trmv_ds", "recysing", "lanczos", "trsv_ds", "rect_qr")
    k = {nm: {"launches": 0, "ms": 0.0, "flops": 0.0, "bytes": 0.0} for nm in names}
    k.update(classes)
    return k


def test_tensor_core_solve_roofline():
    n, cols, launches, ms_each = 8000, 2048, 140, 9.5
    flops = 4.0 * n * n * cols
    kst = _kst(trsv32={"launches": launches, "ms": launches * ms_each, "flops": launches * flops, "bytes": 0.0},
               trsv64={"launches": 12, "ms": 700.0, "flops": 1e12, "bytes": 0.0})
    rf = bench.roofline(kst, PEAKS, n, tensor_solve=True)
    assert rf["bound"] == "tensor" and rf["unit"] == "TFLOP/s"
    assert rf["peak"] == pytest.approx(1408.1 * 1.1 / 2.25 / 3.0)
    assert rf["achieved"] == pytest.approx(flops / (ms_each * 1e-3) / 1e12)
    assert rf["frac"] == pytest.approx(rf["achieved"] / rf["peak"])
    # traffic: the n = 8000 entry (wide-form capture at n = 4000, scaled by n^2) times the columns of a launch
    per_col = (8.017367296e9 + 0.663716864e9) / 4096 * 4.0
    assert rf["traffic"] == pytest.approx(per_col * cols)
    assert rf["launches"] == launches and rf["avg_launch_ms"] == pytest.approx(ms_each)


def test_traffic_is_null_without_a_capture_for_that_order():
    kst = _kst(trsv32={"launches": 10, "ms": 10.0, "flops": 10 * 4.0 * 3000 ** 2 * 64, "bytes": 0.0})
    assert bench.roofline(kst, PEAKS, 3000, tensor_solve=True)["traffic"] is None


def test_cuda_core_and_fp64_and_hbm_bounds():
    kst = _kst(trsv32={"launches": 10, "ms": 100.0, "flops": 10 * 1e11, "bytes": 0.0})
    rf = bench.roofline(kst, PEAKS, 2000, tensor_solve=False)
    assert rf["bound"] == "alu" and rf["peak"] == pytest.approx(bench.FP32_MEASURED_TFLOPS)
    kst = _kst(trsv64={"launches": 4, "ms": 400.0, "flops": 4 * 5e10, "bytes": 0.0})
    rf = bench.roofline(kst, PEAKS, 2000)
    assert rf["peak"] == pytest.approx(bench.FP64_MEASURED_TFLOPS)
    assert rf["achieved"] == pytest.approx(5e10 / 0.1 / 1e12)
    kst = _kst(lanczos={"launches": 100, "ms": 500.0, "flops": 0.0, "bytes": 100 * 2e9})
    rf = bench.roofline(kst, PEAKS, 2000)
    assert rf["bound"] == "hbm" and rf["unit"] == "GB/s" and rf["peak"] == PEAKS["hbm_gbs"]
    assert rf["frac"] == pytest.approx((2e9 / 5e-3 / 1e9) / PEAKS["hbm_gbs"])


def test_nothing_launched_gives_no_roofline():
    assert bench.roofline(_kst(), PEAKS, 2000) is None


def test_clock_summary(tmp_path):
    f = tmp_path / "clocks.csv"
    rows = ["0, 2032, 2032, 800.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"] * 3
    rows.append("0, 1900, 2032, 1100.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active")
    f.write_text("\n".join(rows) + "\n")
    c = bench.Clocks(str(f)).summary()
    assert c["sm_mhz"] == 2032.0 and c["sm_max_mhz"] == 2032.0 and c["samples"] == 4
    assert c["reasons"] == ["sw_power_cap"]


def test_compare_with_fp64_rule():
    """The bench's mixed-against-FP64 check: relative target with the n eps
    ||T||_F floor above 1e-8 ||T||_F, the relative target alone above 1e-6
    ||T||_F, nothing below 1e-8 ||T||_F, and membership compared outside the
    levels' bands."""
    import numpy as np

    fro, n = 100.0, 1000
    s64 = np.array([1.0, 1e-3, 5e-5, 2e-6, 1e-12])
    ok = s64 * (1 + 5e-9)
    rep = bench.compare_with_fp64(ok, s64, fro, n)
    assert rep["n_bad"] == 0 and rep["n_included"] == 4 and rep["n_rel_only"] == 2
    bad = s64.copy()
    bad[1] *= 1 + 2e-8            # above 1e-6 ||T||_F: the relative target alone fails it
    bad[4] = 1.0                  # below 1e-8 ||T||_F: not compared
    rep = bench.compare_with_fp64(bad, s64, fro, n)
    assert rep["n_bad"] == 1
    # a value between 1e-8 and 1e-6 ||T||_F may use the absolute floor 4 n eps ||T||_F
    floor = 4 * n * 2.220446049250313e-16 * fro
    near = s64.copy()
    near[3] = s64[3] + 0.9 * floor
    assert bench.compare_with_fp64(near, s64, fro, n)["n_bad"] == 0
    eps_levels = (1e-2, 1e-4)
    mem64 = np.array([0, 1, 3, 3, 3], dtype=np.uint32)
    mem = mem64.copy()
    mem[0] = 1                    # sigma = 1 against level 1e-2: far outside the band
    rep = bench.compare_with_fp64(s64, s64, fro, n, member=mem, member64=mem64, eps_levels=eps_levels)
    assert rep["member_mismatch"] == 1
