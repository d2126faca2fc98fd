"""Host logic of bench.py's roofline rows (no GPU): achieved work per CUDA-event second against the
bounding unit's peak, the share of the step, and the DRAM traffic attached from the ncu captures."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def test_roofline_rows():
    import bench
    peaks = {"hbm_gbs": 6000.0, "bf16_tflops": 2000.0}
    prof = {
        "dgemm": {"ms": 100.0, "flops": 1.0e11, "bytes": 4.0e9, "launches": 10},
        "spectral32": {"ms": 50.0, "flops": 1.0e10, "bytes": 1.5e11, "launches": 100},
        "tc_gemm": {"ms": 10.0, "flops": 1.0e12, "bytes": 1.0e9, "launches": 20},
        "qrcp": {"ms": 0.0, "flops": 0.0, "bytes": 0.0, "launches": 0},
    }
    rows = {r["kernel"].split()[0]: r for r in bench.roofline_rows(prof, 400.0, peaks, "measured")}
    assert "qr_persistent_kernel" not in rows  # a family that did not run has no row
    d = rows["dgemm_kernel"]
    assert d["bound"] == "alu" and d["unit"] == "TFLOP/s"
    assert d["achieved"] == pytest.approx(1.0, rel=1e-6)                    # 1e11 flop in 0.1 s
    assert d["frac"] == pytest.approx(1.0 / bench.FP64_PEAK_TFLOPS, rel=1e-3)
    assert d["share_of_step"] == pytest.approx(0.25)
    assert d["algorithmic_bytes_per_launch"] == 4e8
    assert d["traffic"] == bench.TRAFFIC["dgemm"][0]
    s = rows["spectral32_kernel"]
    assert s["bound"] == "hbm" and s["achieved"] == pytest.approx(3000.0) and s["frac"] == pytest.approx(0.5)
    t = rows["tc3_gemm_kernel"]
    assert t["bound"] == "tensor" and t["peak"] == pytest.approx(2000.0 * 1.1 / 2.25, rel=1e-4)
    assert t["achieved"] == pytest.approx(100.0)
