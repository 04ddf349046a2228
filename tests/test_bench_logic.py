"""Host logic of bench.py on CPU: the per-phase rooflines and the oracle sample."""

import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

PEAKS = {"fp32": 80.0, "fp64": 1.0, "tf32_mma": 300.0, "bf16_mma": 600.0, "fp64_mma": 1.1, "hbm_gbs": 6000.0}
STATS = {"flops_gemm": 2e12, "flops_qr": 1e12, "flops_svd": 5e11, "flops_inv": 2e10, "flops_lu": 1e10,
         "solve_matrix_bytes": 3e9}


def test_phase_rooflines_work_over_time_against_the_bounding_unit():
    prof = {"gemm_fp32": (100, 200.0), "qr_fp32": (50, 500.0), "svd_fp32": (20, 100.0), "gauss_jordan": (10, 40.0),
            "solve_graph": (3, 3.0), "matvec": (3, 150.0)}
    ph = {e["kernel"]: e for e in bench.phase_rooflines(prof, STATS, PEAKS, "fp32", 131072, 2)}
    g = ph["gemm_fp32"]
    assert g["bound"] == "tensor" and abs(g["achieved"] - 2e12 / 0.2 / 1e12) < 1e-9
    assert abs(g["peak"] - 100.0) < 1e-9 and abs(g["frac"] - 0.1) < 1e-12  # 3xTF32: a third of the MMA rate
    q = ph["qr_fp32"]
    assert q["bound"] == "alu" and q["peak"] == 80.0 and abs(q["achieved"] - 2.0) < 1e-12
    assert ph["gauss_jordan"]["peak"] == 1.0 and abs(ph["gauss_jordan"]["achieved"] - 0.5) < 1e-12
    s = ph["solve_graph"]  # three applications (two iterations + the final one) of 3 GB in 3 ms
    assert s["bound"] == "hbm" and s["unit"] == "GB/s" and abs(s["achieved"] - 3 * 3e9 / 3e-3 / 1e9) < 1e-6
    m = ph["matvec"]
    assert m["unit"] == "Gpairs/s" and abs(m["achieved"] - 131072.0 ** 2 * 3 / 0.15 / 1e9) < 1e-3
    assert abs(m["peak"] - 80e12 / 2 / bench.MATVEC_DF_OPS_PER_PAIR / 1e9) < 1e-6


def test_phase_rooflines_fp64_and_bf16_peaks():
    prof = {"gemm_fp64": (10, 100.0), "gemm_fp32": (10, 100.0)}
    e64 = bench.phase_rooflines(prof, STATS, PEAKS, "fp64", 1000, 1)
    assert e64[0]["kernel"] == "gemm_fp64" and e64[0]["peak"] == 1.0 and e64[0]["bound"] == "alu"
    e16 = bench.phase_rooflines(prof, STATS, PEAKS, "bf16", 1000, 1)
    assert e16[0]["kernel"] == "gemm_fp32" and e16[0]["peak"] == 600.0


def test_sample_keeps_points_per_leaf():
    w, n, d = bench.sample_of("bumpy131k", 64)
    assert (n, d) == (2048, 3) and w.n == 131072 and w.depth == 6
    w, n, d = bench.sample_of("sphere32k", 16)
    assert (n, d) == (2048, 3)


def test_symmetric_matvec_counts_unordered_pairs():
    # the symmetric kernel evaluates each unordered pair once, at its own
    # operation count per pair; the plain one every ordered pair
    prof = {"matvec": (3, 90.0)}
    n = 131072
    sym = bench.phase_rooflines(prof, STATS, PEAKS, "fp32", n, 2, symmetric=True)[0]
    pairs = n * (n - 1) / 2.0 * 3
    assert abs(sym["achieved"] - pairs / 0.09 / 1e9) < 1e-6
    assert abs(sym["peak"] - 80e12 / 2 / bench.MATVEC_SYM_OPS_PER_PAIR / 1e9) < 1e-9
    assert abs(sym["frac"] - sym["achieved"] / sym["peak"]) < 1e-12 and "unordered" in sym["peak_note"]
    plain = bench.phase_rooflines(prof, STATS, PEAKS, "fp32", n, 2)[0]
    assert abs(plain["achieved"] - float(n) * n * 3 / 0.09 / 1e9) < 1e-6
    assert "unordered" not in plain["peak_note"]


def test_ncu_traffic_table_covers_the_timed_classes():
    # the per-class DRAM bytes of the 32k capture are scaled by N on the
    # default line; each key must be a class the profiler reports
    kinds = {"copy", "gemm_fp64", "gemm_fp32", "gauss_jordan", "qr_fp64", "qr_fp32", "svd_fp64", "svd_fp32", "gemv",
             "gemv_sum", "p2p", "interp", "tables", "matvec", "permute", "gauss_jordan_big", "solve_graph"}
    assert set(bench.NCU_DRAM_BYTES_BUMPY32K) <= kinds
    assert bench.NCU_CAPTURE_N == 32768
    assert all(v > 0 for v in bench.NCU_DRAM_BYTES_BUMPY32K.values())
