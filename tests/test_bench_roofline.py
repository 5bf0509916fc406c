"""The benchmark's roofline arithmetic on synthetic kernel timings (no GPU): the dominant kernel
is the one with the largest total device time; HBM-bound kernels report algorithmic bytes per
launch over the launch time against the measured copy peak; FP64 kernels whose FP64 pipe use
exceeds their HBM fraction report FP64 thread-instructions per second against the pipe's
304 per clock at the sampled SM clock."""
import bench


def test_fp64_lean_cells_reports_the_fp64_pipe():
    n = 511 ** 3
    # 240 launches of 24.8 ms and a smaller faces kernel: cells dominate
    k = {"k_lean_cells": (240, 240 * 24.8), "k_lean_faces": (240, 240 * 8.5), "k_lean_picard": (16, 16 * 29.3)}
    r = bench.roofline(k, n, sm_mhz=2070.0)
    assert r["kernel"] == "k_lean_cells" and r["bound"] == "alu" and r["unit"] == "G FP64 inst/s"
    peak = 304.0 * 2070e6 / 1e9
    assert abs(r["peak"] - peak) < 1e-9
    achieved = bench.KERNEL_FP64_INST_PER_CELL["k_lean_cells"] * n / 24.8e-3 / 1e9
    assert abs(r["achieved"] - achieved) < 1e-6 * achieved
    assert abs(r["frac"] - achieved / peak) < 1e-12
    # the algorithmic HBM rate stays in the line for reference
    hbm = bench.KERNEL_BYTES_PER_CELL["k_lean_cells"] * n / 24.8e-3 / 1e9
    assert abs(r["hbm_gbs"] - hbm) < 1e-6 * hbm
    assert r["traffic"] == bench.KERNEL_TRAFFIC_PER_CELL["k_lean_cells"] * n


def test_fp32_correction_reports_hbm():
    n = 511 ** 3
    k = {"k_corr_cells": (300, 300 * 4.0), "k_corr_faces": (300, 300 * 3.9), "k_mix_prepare": (2, 2 * 20.0)}
    r = bench.roofline(k, n)
    hbm, _ = bench.peaks()
    assert r["kernel"] == "k_corr_cells" and r["bound"] == "hbm" and r["unit"] == "GB/s"
    gbs = bench.KERNEL_BYTES_PER_CELL["k_corr_cells"] * n / 4.0e-3 / 1e9
    assert abs(r["achieved"] - gbs) < 1e-6 * gbs
    assert abs(r["peak"] - hbm) < 1e-9 and abs(r["frac"] - gbs / hbm) < 1e-12
