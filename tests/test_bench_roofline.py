"""bench.py's roofline records from a synthetic library profile (CPU): the SVD record counts the
textbook R-SVD flops and scales the committed capture's DRAM/algorithmic-bytes ratio by the run's
own algorithmic bytes per launch; the matvec record has no traffic while its capture is stale; the
record with more device time leads."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _prof(**kw):
    p = dict(mv_gemm_ms=400.0, mv_gemm_flops=1.2e14, mv_gemm_launches=4000, f64_gemm_ms=50.0,
             f64_gemm_flops=2e12, f64_gemm_launches=100, svd_block_calls=90, svd_block_ms=9000.0,
             svd_block_flops=7.2e13, svd_block_alg_flops=1.8e13, svd_block_alg_bytes=9e9)
    p.update(kw)
    return p


RATES = {"fp64_fma": 1.25, "fp32_fma": 78.0, "bf16_tc_gemm_8192": 1500.0, "tf32_tc_gemm_8192": 800.0}
PK = {"hbm_gbs": 7000.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}


def test_svd_leads_and_counts_textbook_flops():
    roof, other = bench.rooflines("bf16", True, _prof(), RATES, PK, "measured")
    assert roof["kernel"].startswith("k_bjacobi_queue")
    assert abs(roof["achieved"] - 1.8e13 / 9.0 / 1e12) < 1e-12            # 2.0 TFLOP/s
    assert abs(roof["frac"] - roof["achieved"] / 78.0) < 1e-15
    assert abs(roof["executed_tflops"] - 7.2e13 / 9.0 / 1e12) < 1e-12
    ratio = bench.ncu_traffic("bjacobi_queue_traffic")["dram_over_algorithmic_bytes"]
    assert abs(roof["traffic"] - ratio * 9e9 / 90) < 1e-3
    assert 2.0 < ratio < 4.0
    assert other["kernel"].startswith("k_tc_gemm") and other["traffic"] is None
    assert abs(other["achieved"] - 1.2e14 / 0.4 / 1e12) < 1e-9 and other["peak"] == 1700.0


def test_matvec_leads_without_splits_and_fp64_path():
    roof, other = bench.rooflines("bf16", False, _prof(svd_block_calls=0), RATES, PK, "measured")
    assert roof["kernel"].startswith("k_tc_gemm") and other is None
    roof, other = bench.rooflines("fp64", True, _prof(svd_block_calls=0), RATES, PK, "measured")
    assert roof["bound"] == "alu" and roof["peak"] == 1.25 and "emulated" in roof["kernel"]
    assert abs(roof["achieved"] - 2e12 / 0.05 / 1e12) < 1e-9


def test_tf32_peak_is_scaled_bf16_sustained():
    roof, _ = bench.rooflines("tf32", False, _prof(svd_block_calls=0), RATES, PK, "measured")
    assert abs(roof["peak"] - 1700.0 * bench.NOMINAL_TF32_OVER_BF16) < 1e-9
