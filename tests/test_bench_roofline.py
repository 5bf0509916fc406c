"""The benchmark's roofline arithmetic on synthetic kernel timings (no GPU): the dominant kernel
is the one with the largest total device time; HBM-bound kernels report algorithmic bytes per
launch over the launch time against the measured copy peak; FP64 kernels whose FP64 pipe use
exceeds their HBM fraction report FP64 thread-instructions per second against the library's own
measured FP64 issue rate (else the pipe's nominal 304 per clock at the sampled SM clock); ncu
figures are used only while the kernel's sources are the ones they were captured from."""
import bench


def _with_profile(monkeypatch, name, **fig):
    monkeypatch.setitem(bench.PROFILED, name, dict(src=bench.source_hash(name), **fig))


def test_fp64_lean_cells_reports_the_fp64_pipe(monkeypatch):
    _with_profile(monkeypatch, "k_lean_cells", fp64_inst=99.9, fp64_flops=147.9, traffic=311.0)
    n = 511 ** 3
    # 240 launches of 24.8 ms and a smaller faces kernel: cells dominate
    k = {"k_lean_cells": (240, 240 * 24.8), "k_lean_faces": (240, 240 * 8.5), "k_lean_picard": (16, 16 * 29.3)}
    r = bench.roofline(k, n, sm_mhz=2070.0)
    assert r["kernel"] == "k_lean_cells" and r["bound"] == "alu" and r["unit"] == "G FP64 inst/s"
    peak = 304.0 * 2070e6 / 1e9
    assert abs(r["peak"] - peak) < 1e-9
    achieved = 99.9 * n / 24.8e-3 / 1e9
    assert abs(r["achieved"] - achieved) < 1e-6 * achieved
    assert abs(r["frac"] - achieved / peak) < 1e-12
    # the algorithmic HBM rate stays in the line for reference
    hbm = bench.KERNEL_BYTES_PER_CELL["k_lean_cells"] * n / 24.8e-3 / 1e9
    assert abs(r["hbm_gbs"] - hbm) < 1e-6 * hbm
    assert r["traffic"] == 311.0 * n and r["ncu_figures"] == "current"
    # with the library's own FP64 issue-rate measurement, that is the peak
    own = {"fp64_ginst": 500.0, "copy_gbs": 6800.0}
    r2 = bench.roofline(k, n, sm_mhz=2070.0, own=own)
    assert r2["bound"] == "alu" and r2["peak"] == 500.0 and abs(r2["frac"] - achieved / 500.0) < 1e-12
    assert abs(r2["frac_of_nominal_pipe"] - achieved / peak) < 1e-12
    assert abs(r2["own_copy_gbs"] - 6800.0) < 1e-12


def test_stale_ncu_figures_are_not_reported(monkeypatch):
    monkeypatch.setitem(bench.PROFILED, "k_lean_cells",
                        dict(src="0000000000000000", fp64_inst=99.9, traffic=311.0))
    n = 255 ** 3
    r = bench.roofline({"k_lean_cells": (10, 10 * 3.0)}, n, sm_mhz=2070.0)
    assert r["bound"] == "hbm" and r["traffic"] is None and "fp64_inst_per_cell" not in r
    assert r["ncu_figures"].startswith("stale")


def test_source_hash_tracks_the_kernel_files(tmp_path, monkeypatch):
    h = bench.source_hash("k_lean_cells_df64")
    assert h is not None and len(h) == 16
    assert bench.source_hash("k_lean_cells") == h          # same translation unit and headers
    assert bench.source_hash("no_such_kernel") is None
    # identical copies give the same hash; one changed byte changes it
    before = bench.source_hash("k_corr_iteration")
    for f in bench.KERNEL_SOURCES["k_corr_iteration"]:
        with open(bench.os.path.join(bench.CSRC, f), "rb") as fh:
            (tmp_path / f).write_bytes(fh.read())
    monkeypatch.setattr(bench, "CSRC", str(tmp_path))
    assert bench.source_hash("k_corr_iteration") == before
    f0 = bench.KERNEL_SOURCES["k_corr_iteration"][0]
    (tmp_path / f0).write_bytes((tmp_path / f0).read_bytes() + b" ")
    assert bench.source_hash("k_corr_iteration") != before


def test_fp32_correction_reports_hbm():
    n = 511 ** 3
    k = {"k_corr_iteration": (300, 300 * 4.0), "k_mix_prepare": (2, 2 * 20.0)}
    r = bench.roofline(k, n)
    hbm, _ = bench.peaks()
    assert r["kernel"] == "k_corr_iteration" and r["bound"] == "hbm" and r["unit"] == "GB/s"
    gbs = bench.KERNEL_BYTES_PER_CELL["k_corr_iteration"] * n / 4.0e-3 / 1e9
    assert abs(r["achieved"] - gbs) < 1e-6 * gbs
    assert abs(r["peak"] - hbm) < 1e-9 and abs(r["frac"] - gbs / hbm) < 1e-12


def test_double_float_cells_report_hbm_with_their_own_bytes():
    n = 511 ** 3
    k = {"k_lean_cells_df64": (93, 93 * 11.2), "k_lean_faces_df64": (90, 90 * 4.7)}
    r = bench.roofline(k, n, own={"copy_gbs": 6900.0})
    gbs = bench.KERNEL_BYTES_PER_CELL["k_lean_cells_df64"] * n / 11.2e-3 / 1e9
    assert r["kernel"] == "k_lean_cells_df64" and r["bound"] == "hbm"
    assert abs(r["achieved"] - gbs) < 1e-6 * gbs
    assert abs(r["frac_of_own_copy"] - gbs / 6900.0) < 1e-12


def test_fp32_correction_reports_ncu_traffic_while_current(monkeypatch):
    _with_profile(monkeypatch, "k_corr_iteration", traffic=106.6, thread_inst=720.8)
    n = 511 ** 3
    r = bench.roofline({"k_corr_iteration": (300, 300 * 4.85)}, n)
    assert r["ncu_figures"] == "current" and r["traffic"] is not None
    assert abs(r["traffic"] - 106.6 * n) < 1e-6 * r["traffic"]


def test_precision_check_size_list():
    assert bench._parse_sizes("512:1, 128:2,64", 50) == [(512, 1), (128, 2), (64, 50)]
    assert bench._parse_sizes("", 3) == []
