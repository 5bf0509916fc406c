#!/usr/bin/env python3
"""Benchmark: effective memory throughput T_eff (thesis Art. 1, Eqs. 28-29, 35-38) and PT
iterations per second of the porosity-wave PT solver on one GB300, 511^3 cells.

One benchmark step = one physical time step of the whole hot path: the old-state snapshot and
stress sub-step, `--iters` PT iterations (coefficients, pressures, stresses, momentum, Darcy,
porosity, velocities; Picard update and residual norms every 15th), and the end-of-step
stresses. T_eff = A_eff / t_it with A_eff = 25 N p bytes and t_it = timed time / PT iterations.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] ...
Multi-GPU (torchrun, one rank per GPU) runs independent replicas (seed = rank): weak scaling,
no data-path collective; only the timing max over ranks and a barrier are collective.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import pt_inputs as I  # noqa: E402
from paper_2207_08716_gb300 import measure as M  # noqa: E402

METRIC = "T_eff GB/s (% of HBM peak) and PT iter/s at 511^3: FP64 vs FP32 vs batched"
PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
HBM_FALLBACK_GBS = 6800.0

# Algorithmic bytes per cell and launch of each kernel of the step-by-step FP64 path: the
# arrays it must read and write once (8 B each), counted from its arguments.
KERNEL_BYTES_PER_CELL = {
    "k_perm": 3 * 8, "k_centres": 19 * 8, "k_edges": 10 * 8, "k_porosity": 11 * 8,
    "k_faces": 21 * 8, "k_picard": 13 * 8, "k_begin_step": 6 * 8,
    # FP64-lean form: cells reads 28 arrays (V, Pt, Pf, phi, w, k, Pto, Pfo, phio, Eo, iEo, ieta,
    # idtp, cm2, 3 toa_ii, 6 pre-multiplied edge moduli, 3 toa_e) and writes 11 (Pt, Pf, phi, w, k,
    # 6 stresses); faces reads 17 (6 stresses, Pt, phi, 3 dtv, 3 R, 3 V) and writes 6 (3 R, 3 V)
    "k_lean_cells": 39 * 8, "k_lean_faces": 23 * 8, "k_lean_picard": 11 * 8, "k_lean_coef": 23 * 8,
    "k_lean_begin": 11 * 8,
    # mixed precision, one fused FP32 correction iteration: reads 18 arrays (3 dV, dPt, dPf, cc, k,
    # 1/dtau_Pt, r_Pt, r_Pf, mu, centre dtau_V, 3 r_F, 3 R) and writes 8 (3 dV', dPt', dPf', 3 R)
    "k_corr_iteration": 26 * 4,
    # adjoint PT iteration: cells reads 26 arrays and writes 10, faces reads 17 and writes 6
    "k_adj_cells": 36 * 8, "k_adj_faces": 23 * 8,
    # with the power law (Eq. 24): edges read 10 arrays and write 6; cells read 50 (23
    # multiplier, right-hand-side and row-factor arrays, V, phi, mu, 17 power-law coefficients,
    # lambda_mu, g_mu, 3 edge Z) and write 8; faces read 20
    # (the per-face pseudo-steps added) and write 6
    "k_adj_edges_pl": 16 * 8, "k_adj_cells_pl": 58 * 8, "k_adj_faces_pl": 26 * 8,
    # double-float form (8 B per value): cells reads 22 arrays (V, Pt, Pf, phi, k, Pto, Pfo, phio,
    # ieta, idtp, cm2, 3 toa_ii, 3 edge moduli, 3 toa_e) and writes 10 (Pt, Pf, phi, k, 6 stresses); faces
    # reads 15 (6 stresses, Pt, phi, centre dtau_V, 3 R, 3 V) and writes 6; Picard reads 11 and
    # writes 2; coefficients read 8 (mu, eta, 6 old stresses) and write 13; step start 4 + 3
    "k_lean_cells_df64": 32 * 8, "k_lean_faces_df64": 21 * 8, "k_lean_picard_df64": 13 * 8,
    "k_lean_coef_df64": 21 * 8, "k_lean_begin_df64": 8 * 8,
}
PRECISIONS = {"fp64": 0, "fp32": 1, "fp64-stepwise": 2, "df64": 3}
# arithmetic each form computes in: df64 = double-float (an FP32 pair, 48-bit significand), the
# form whose fields match the FP64 oracle within 1e-10 after the same iterations (tests)
DTYPES = {"fp64": "f64", "fp32": "f32", "fp64-stepwise": "f64", "df64": "df64"}
# Per-kernel figures from one ncu capture each (profiles/*.md): FP64 thread-instructions
# (DADD + DFMA + DMUL) and flops (DFMA x 2 + DADD + DMUL) per cell, DRAM bytes per cell
# (dram__bytes_read.sum + dram__bytes_write.sum; the capture's per-cell figure scales with the
# cells of a launch). Each entry records the sha256 (16 hex digits) of the kernel's source files
# at the capture; when the sources have changed since, the figures are stale and the bench
# reports them as null (`python bench.py --source-hashes` prints the current hashes).
KERNEL_SOURCES = {
    **{k: ("pt_lean_kernels.cu", "pt_lean_body.cuh", "pt_lean.cuh", "df64.cuh", "pt_common.cuh")
       for k in ("k_lean_cells", "k_lean_faces", "k_lean_picard", "k_lean_coef", "k_lean_cells_df64",
                 "k_lean_faces_df64", "k_lean_picard_df64", "k_lean_coef_df64")},
    "k_centres": ("pt_ref_kernels.cu", "pt_kernels.cuh", "pt_common.cuh"),
    **{k: ("pt_adjoint_kernels.cu", "pt_adjoint.cuh", "pt_common.cuh")
       for k in ("k_adj_cells", "k_adj_faces", "k_adj_edges_pl", "k_adj_cells_pl", "k_adj_faces_pl")},
    "k_corr_iteration": ("pt_mixed_kernels.cu", "pt_mixed.cuh", "pt_common.cuh"),
    "k_mg_smooth_fp32": ("rx_mg_kernels.cu", "rx.cuh"),
}
PROFILED = {
    # profiles/kernels_191_ncu_metrics.md (191^3, every launch of one step of each form)
    "k_lean_cells": {"src": "847b74c5871329ee", "fp64_inst": 100.2, "fp64_flops": 148.4, "traffic": 310.9},
    "k_lean_faces": {"src": "847b74c5871329ee", "fp64_inst": 33.1, "fp64_flops": 50.0, "traffic": 180.3},
    "k_lean_cells_df64": {"src": "847b74c5871329ee", "traffic": 260.0, "thread_inst": 1929.0},
    "k_lean_faces_df64": {"src": "847b74c5871329ee", "traffic": 164.3, "thread_inst": 724.9},
    # profiles/k_corr_iteration_fp32_255.md (255^3, one launch)
    "k_corr_iteration": {"src": "642041b57f4bbbcc", "traffic": 106.3, "thread_inst": 720.8},
}
# The FP64 pipe's nominal issue capacity: 304 thread-instructions per GPU clock (2 per SM; ncu's
# sm__inst_executed_pipe_fp64 peak on this machine's GB300), 629 G/s at 2.07 GHz.
FP64_PIPE_INST_PER_CLK = 304.0
CSRC = os.path.join(ROOT, "paper_2207_08716_gb300", "csrc")


def source_hash(kernel: str) -> str | None:
    import hashlib
    files = KERNEL_SOURCES.get(kernel)
    if not files:
        return None
    h = hashlib.sha256()
    for f in sorted(files):
        with open(os.path.join(CSRC, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled(kernel: str) -> dict:
    """The kernel's ncu figures if they were captured from its current sources, else {}."""
    e = PROFILED.get(kernel)
    if not e or e.get("src") != source_hash(kernel):
        return {}
    return e

def parse():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--source-hashes", action="store_true",
                    help="print the current source hash of every kernel with ncu figures and exit")
    ap.add_argument("--steps", type=int, default=8)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("native", "reference"), default="native")
    ap.add_argument("--n", type=int, default=511, help="cells per direction (511 = benchmark grid)")
    ap.add_argument("--iters", type=int, default=30, help="PT iterations per physical step")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--seeds", default="0,1,2",
                    help="anomaly-position seeds of the headline form at N = 1 (value = median over them); "
                         "under torchrun each rank uses seed = rank")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-n", type=int, default=255, help="sub-block edge of the CPU sample")
    ap.add_argument("--cpu-iters", type=int, default=60)
    ap.add_argument("--cpu-timings", action="store_true",
                    help="time the oracle at 127^3 and 511^3 (PT iterations) and one full c1 step, on all host "
                         "cores and on one core, each in its own process, and exit")
    ap.add_argument("--cpu-timing-iters", type=int, default=20)
    ap.add_argument("--precision", choices=tuple(PRECISIONS), default="df64",
                    help="df64: the FP64-lean iteration in double-float arithmetic (FP64 oracle parity 1e-10); "
                         "fp64: FP64-lean kernels; fp64-stepwise: one kernel per step; fp32: FP32 PT")
    ap.add_argument("--forms", default="fp64,fp32,batched,batched32,fp32mg",
                    help="extra forms measured after the headline one (comma list of fp64, df64, fp32, "
                         "fp64-stepwise, batched (FP64 ensemble), batched32 (FP32 ensemble), fp32mg (one converged "
                         "step of the FP32 form with multigrid correction solves); '' for none)")
    ap.add_argument("--mg-form-levels", type=int, default=6, help="grids of the fp32mg form's V-cycles")
    ap.add_argument("--no-own-peaks", action="store_true",
                    help="skip the library's own copy / FP64 / FP32 peak measurements")
    ap.add_argument("--fp32-iters", type=int, default=300, help="FP32 iterations per step of the fp32 form")
    ap.add_argument("--batch-n", type=int, default=64, help="instances of the batched form")
    ap.add_argument("--batch-iters", type=int, default=60, help="PT iterations per step of the batched form")
    ap.add_argument("--workload", choices=("porosity", "shear"), default="porosity",
                    help="porosity: n^3 box, Gaussian anomaly (the benchmark); shear: the background-shear "
                         "setup of Table 2 on n x n x 2n cells (30 x 30 x 60 box, ellipsoidal anomaly)")
    ap.add_argument("--adjoint", action="store_true",
                    help="measure the adjoint instead (127^3, 20 steps, checkpoint every 5): forward and "
                         "backward wall time, cost multiple, optional finite-difference check")
    ap.add_argument("--adjoint-n", type=int, default=127)
    ap.add_argument("--adjoint-steps", type=int, default=20)
    ap.add_argument("--adjoint-ckpt", default="5,1", help="checkpoint spacings to measure (comma list)")
    ap.add_argument("--adjoint-fd", type=int, default=0, help="finite-difference directions to check")
    ap.add_argument("--reactive", action="store_true",
                    help="measure the reactive porosity-wave solver (Art. 3) instead: T_eff with A_eff = 7 N p")
    ap.add_argument("--rx-n", type=int, default=255, help="reactive grid n x n x 4n")
    ap.add_argument("--rx-iters", type=int, default=100, help="PT iterations per physical step (reactive)")
    ap.add_argument("--reactive-mg", action="store_true",
                    help="measure the multigrid-accelerated reactive step instead: time to a converged "
                         "physical step, FAS V-cycles against the plain PT iteration, n x n x 4n cells")
    ap.add_argument("--mg-n", type=int, default=256, help="multigrid reactive grid n x n x 4n (n divisible by 2^(levels-1))")
    ap.add_argument("--mg-levels", type=int, default=7)
    ap.add_argument("--mg-precisions", default="fp32,fp64", help="forms of the multigrid measurement")
    ap.add_argument("--mg-sweeps", default="", help="nu_pre,nu_post,nu_coarse of the V-cycle (default 2,2,30)")
    ap.add_argument("--mg-plain-steps", type=int, default=2,
                    help="timed converged steps of the plain PT solver (after one warm-up step)")
    ap.add_argument("--batch-precision", choices=("fp64", "fp32"), default="fp64",
                    help="precision of the batched ensemble (fp32: the defect-correction form in the "
                         "persistent FP32 engine)")
    ap.add_argument("--precision-check", action="store_true",
                    help="porosity of the FP32 form against an FP64-class form (and the oracle at the "
                         "--pc-oracle-n sizes) after converged physical steps of the c1 workload at each --pc-n")
    ap.add_argument("--pc-n", default="32,64", help="grid sizes of the precision check, n[:steps] each")
    ap.add_argument("--pc-steps", type=int, default=50, help="converged steps where --pc-n gives none")
    ap.add_argument("--pc-ref", choices=("fp64", "df64", "none"), default="fp64",
                    help="the FP64-class form the FP32 form is compared with (none: run the multigrid form "
                         "alone, no comparison)")
    ap.add_argument("--pc-oracle", type=int, default=1, help="also run the oracle (1) or not (0)")
    ap.add_argument("--pc-oracle-n", default="32", help="grid sizes at which the oracle runs too")
    ap.add_argument("--pc-plain-max", type=int, default=100000,
                    help="run the FP32 form with plain PT correction solves only up to this grid size")
    ap.add_argument("--pc-mg", type=int, default=0,
                    help="also the FP32 form with multigrid correction solves over this many levels (>= 2; "
                         "each level ceil(n / 2) cells per direction, the coarsest at least 2)")
    ap.add_argument("--batch-inner-rtol", type=float, default=0.0,
                    help="FP32 ensembles: relative residual drop of each FP32 correction solve (0: library default)")
    ap.add_argument("--batched-converge", action="store_true",
                    help="run one step of the batched ensemble to convergence and report p50/p99 "
                         "time-to-converge (minutes of GPU time) instead of the throughput bench")
    return ap.parse_args()


def peaks():
    try:
        with open(PEAKS_PATH) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


def workload_params(n: int, iters: int, precision: str = "fp64", workload: str = "porosity") -> dict:
    p = I.shear_params(n) if workload == "shear" else I.large_params(n)
    p["max_iter"] = iters
    p["precision"] = PRECISIONS[precision]
    return p


def workload_phi(p: dict, seed: int, workload: str = "porosity"):
    if workload == "shear":
        return I.ellipsoid_porosity(p)
    return I.gaussian_porosity(p, centres=(I.perturbed_centre(seed),))


def workload_name(n: int, iters: int, precision: str = "fp64", workload: str = "porosity") -> str:
    if workload == "shear":
        return (f"two-phase porosity-wave PT solver ({precision}) under background shear (Table 2 setup), "
                f"{n}x{n}x{2 * n} cells, 30x30x60 box, ellipsoidal anomaly, {iters} PT iterations per step")
    return (f"two-phase porosity-wave PT solver ({precision}), {n}^3 cells, one seed-perturbed "
            f"centred Gaussian anomaly, {iters} PT iterations per physical step")


def native_config(args, iters: int, world: int) -> dict:
    """The benchmark's `config` (the same for the native arm and the reference arm, which times
    the oracle on a bounded sample of this workload, described in its cpu_baseline)."""
    return {"workload": workload_name(args.n, iters, args.precision, args.workload),
            "n": args.n, "iters_per_step": iters, "precision": args.precision,
            "parallelism": "replicas" if world > 1 else "single",
            "l2": "inputs larger than L2 (every field >= 0.5 GB), no flush",
            "seeds": "value = median over the anomaly seeds run (N = 1) or seed = rank"}


# ------------------------------------------------------------------------ CPU (oracle) leg
def cpu_sample(n_sub: int, iters: int) -> dict:
    """Oracle (as it stands) on a bounded sample of the benchmark workload: an n_sub^3 block of
    the 511^3 grid around the anomaly (same spacing and parameters), `iters` PT iterations of
    the first physical step. Returns T_eff over that sample."""
    import oracle as O
    p = workload_params(511, iters)
    h = p["lx"] / p["nx"]
    sub = dict(p, nx=n_sub, ny=n_sub, nz=n_sub, lx=n_sub * h, ly=n_sub * h, lz=n_sub * h)
    sub["dtpt_scale"] = p["dtpt_scale"] * n_sub / p["nz"]
    phi = I.gaussian_porosity(sub, centres=((0.5, 0.5, 0.5),), width=0.1)
    st = O.make_state(sub, phi)
    O.begin_step(st)
    t0 = time.perf_counter()
    rc, _ = O.iterate_n(st, 0, iters)
    dt = time.perf_counter() - t0
    if rc != 0:
        raise RuntimeError(f"oracle rc {rc}")
    ncell = n_sub ** 3
    return {"value": M.t_eff_gbs(ncell, 8, dt / iters), "unit": "GB/s", "cores": O.max_threads(),
            "kind": "oracle", "t_it_s": dt / iters, "seconds": dt,
            "sample": (f"{n_sub}^3-cell block of the 511^3 workload (same spacing, parameters and "
                       f"anomaly width), {iters} PT iterations of the first step, FP64 C oracle "
                       f"with OpenMP; T_eff with A_eff = 25 N 8 B over the block")}


def _cpu_job(kind: str, n: int, iters: int, warm: int) -> dict:
    """One oracle timing in this process (its OpenMP thread count set by the caller's
    OMP_NUM_THREADS): `iters` PT iterations after `warm` warm-up ones of the first step of the n^3
    benchmark workload (kind "iter"), or one full step of the 32^3 c1 workload to its tolerance
    (kind "c1")."""
    import oracle as O
    if kind == "c1":
        p = I.c1_params(32)
        st = O.make_state(p, I.gaussian_porosity(p))
        t0 = time.perf_counter()
        rc, it, _ = O.step(st)
        dt = time.perf_counter() - t0
        return {"kind": "c1 step to tol 1e-8", "n": 32, "rc": rc, "iters": it, "seconds": dt,
                "t_it_s": dt / max(it, 1), "cores": O.max_threads()}
    p = workload_params(n, iters)
    st = O.make_state(p, I.gaussian_porosity(p, centres=(I.perturbed_centre(0),)))
    O.begin_step(st)
    O.iterate_n(st, 0, warm)
    t0 = time.perf_counter()
    rc, _ = O.iterate_n(st, warm, iters)
    dt = time.perf_counter() - t0
    return {"kind": "PT iterations", "n": n, "rc": rc, "iters": iters, "seconds": dt, "t_it_s": dt / iters,
            "t_eff_gbs": M.t_eff_gbs(n ** 3, 8, dt / iters), "cores": O.max_threads()}


def cpu_timings(args) -> dict:
    """The oracle timed as the measurement plan asks, each case in a fresh process with its
    thread count: t_it over 20 PT iterations (after 2 warm-up) at 127^3 and 511^3, with all
    host cores and with one; one full c1 step (32^3 to tol) likewise. A baseline, not a target."""
    import subprocess
    out = []
    ncores = os.cpu_count() or 1
    cases = [("iter", 127), ("iter", 511), ("c1", 32)]
    # the 511^3 oracle state and scratch take ~60 GB of host memory: run it only with room to spare
    avail_gb = None
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    avail_gb = int(line.split()[1]) / 2 ** 20
    except OSError:
        pass
    if avail_gb is None or avail_gb < 120:
        cases = [c for c in cases if c[1] != 511]
        out.append({"skipped": "511^3", "reason": f"host memory available {avail_gb} GB < 120 GB"})
    for kind, n in cases:
        for threads in (ncores, 1):
            env = dict(os.environ, OMP_NUM_THREADS=str(threads))
            code = (f"import json, bench; print('CPUJOB ' + json.dumps(bench._cpu_job({kind!r}, {n}, "
                    f"{args.cpu_timing_iters}, 2)))")
            r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True)
            line = [l for l in r.stdout.splitlines() if l.startswith("CPUJOB ")]
            rec = json.loads(line[-1][7:]) if line else {"error": (r.stderr or "")[-300:]}
            rec["threads_requested"] = threads
            out.append(rec)
            print(json.dumps(rec), flush=True)
    return {"host_cores": ncores, "host_mem_available_gb": avail_gb, "cases": out}


def run_reference(args):
    rank, _, world = M.rank_env()
    if rank != 0:
        return 0
    vals = []
    for s in range(args.warmup + args.steps):
        r = cpu_sample(args.cpu_n, args.cpu_iters)
        if s >= args.warmup:
            vals.append(r)
    v = float(np.median([r["value"] for r in vals]))
    t_step = float(np.median([r["seconds"] for r in vals]))
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "GB/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": native_config(args, args.iters, world),
        "cpu_baseline": {k: vals[-1][k] for k in ("kind", "cores", "sample")} | {"value": v, "unit": "GB/s"},
        "e2e": {"value": v, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- GPU leg
def roofline(kernels: dict, ncell: int, sm_mhz: float | None = None, own: dict | None = None) -> dict:
    """Roofline of the dominant kernel (largest device time) from the live per-kernel events.
    HBM: algorithmic bytes per launch over the launch time against the measured copy peak
    (MEASURED_PEAKS.json; the library's own 16-byte copy kernel in `own_copy_gbs` beside it).
    FP64 kernels issue-bound on the FP64 pipe (when their ncu counts are current) report FP64
    thread-instructions per second against the library's own FP64 issue-rate measurement
    (DFMA/DADD/DMUL mix) when given, else the pipe's nominal 304 per clock at the sampled clock."""
    hbm, hbm_kind = peaks()
    name, (nl, ms) = max(kernels.items(), key=lambda kv: kv[1][1])
    per_launch_s = ms / 1e3 / nl
    bytes_launch = KERNEL_BYTES_PER_CELL.get(name, 0) * ncell
    prof = profiled(name)
    inst_cell = prof.get("fp64_inst")
    flops_cell = prof.get("fp64_flops")
    traffic_cell = prof.get("traffic")
    gbs = bytes_launch / per_launch_s / 1e9
    roof = {"kernel": name, "bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s",
            "frac": gbs / hbm, "peak_source": f"{hbm_kind} HBM copy (MEASURED_PEAKS.json hbm_gbs)",
            "traffic": traffic_cell * ncell if traffic_cell else None,
            "algorithmic_bytes_per_launch": bytes_launch, "launch_ms": per_launch_s * 1e3,
            "ncu_figures": "current" if prof else ("stale (sources changed since the capture)"
                                                     if name in PROFILED else "none")}
    if own and own.get("copy_gbs"):
        roof["own_copy_gbs"] = own["copy_gbs"]
        roof["frac_of_own_copy"] = gbs / own["copy_gbs"]
    if inst_cell:
        clk = (sm_mhz or 2070.0) * 1e6
        nominal = FP64_PIPE_INST_PER_CLK * clk / 1e9
        peak, src = nominal, (f"FP64 pipe nominal capacity, {FP64_PIPE_INST_PER_CLK:.0f} thread-instructions "
                              f"per clock at the measured {clk / 1e6:.0f} MHz (ncu pipe peak)")
        if own and own.get("fp64_ginst"):
            peak, src = own["fp64_ginst"], ("measured FP64 issue rate, DFMA/DADD/DMUL mix "
                                            "(pt_peak_arith, this run)")
        ginst = inst_cell * ncell / per_launch_s / 1e9
        if ginst / peak > roof["frac"]:
            roof.update(bound="alu", achieved=ginst, peak=peak, unit="G FP64 inst/s", frac=ginst / peak,
                        peak_source=src, frac_of_nominal_pipe=ginst / nominal)
        roof["fp64_inst_per_cell"] = inst_cell
        if flops_cell:
            roof["fp64_tflops"] = flops_cell * ncell / per_launch_s / 1e12
        roof["hbm_gbs"] = gbs
    return roof


def measure_own_peaks(dev, copy_gib: float = 4.0) -> dict:
    """The library's own peak measurements on this GPU: 16-byte vector copy over copy_gib GiB
    (read + write bytes, best of 10), FP64 DFMA/DADD/DMUL mix and FP32 FMA issue rates."""
    import ctypes as C
    import torch
    from paper_2207_08716_gb300 import native as N
    lib = N.load()
    stream = torch.cuda.current_stream(dev)
    out = {}
    nbytes = int(copy_gib * (1 << 30))
    src = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    dst = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    src.fill_(1)
    ms, g = C.c_double(), C.c_double()
    torch.cuda.synchronize(dev)
    if lib.pt_peak_copy(src.data_ptr(), dst.data_ptr(), nbytes, 10, stream.cuda_stream, C.byref(ms), C.byref(g)) == 0:
        out["copy_gbs"] = g.value
        out["copy_bytes"] = nbytes
    del src, dst
    sink = torch.zeros(1 << 16, dtype=torch.float64, device=dev)
    if lib.pt_peak_arith(0, sink.data_ptr(), 2000, 5, stream.cuda_stream, C.byref(ms), C.byref(g)) == 0:
        out["fp64_ginst"] = g.value
        out["fp64_tflops_mix"] = g.value * 4.0 / 3.0 / 1e3     # DFMA counts 2 flops, DADD and DMUL 1
    if lib.pt_peak_arith(1, sink.data_ptr(), 100000, 5, stream.cuda_stream, C.byref(ms), C.byref(g)) == 0:
        out["fp32_ginst"] = g.value
        out["fp32_tflops"] = 2.0 * g.value / 1e3
    out["how"] = ("pt_peak_copy (16-byte vector copy, best of 10), pt_peak_arith (8 independent chains per "
                  "thread, 2048 threads per SM, best of 5)")
    del sink
    torch.cuda.empty_cache()
    return out


def measure_form(args, precision: str, iters: int, steps: int, warmup: int, e2e_steps: int,
                 dev, world: int, rank: int, local_rank: int, seed: int | None = None,
                 own: dict | None = None) -> dict:
    """Time `steps` physical steps (after `warmup`) of one form of the solver on this rank
    (anomaly seed = rank unless given)."""
    import torch
    import torch.distributed as dist
    from paper_2207_08716_gb300.solver import PTSolver

    n = args.n
    p = workload_params(n, iters, precision, args.workload)
    seed = M.replica_seed(rank) if seed is None else seed
    phi = workload_phi(p, seed, args.workload)
    stream = torch.cuda.current_stream(dev)
    s = PTSolver(p, phi, device=dev, stream=stream)
    del phi

    def one_step():
        s.step_begin()
        s.iterate(0, iters, report=False)
        s.step_end()

    def barrier():
        if world > 1:
            dist.barrier()

    for _ in range(warmup):
        one_step()
    torch.cuda.synchronize(dev)
    clocks = M.ClockSampler(local_rank)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = s.launch_count()
    barrier()
    torch.cuda.synchronize(dev)
    clocks.start()
    s.profile_begin()
    e0.record(stream)
    for _ in range(steps):
        one_step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    kernels = s.profile_end()
    clk = clocks.stop()
    barrier()
    t = M.max_over_ranks(e0.elapsed_time(e1) / 1e3, dev)
    launches = s.launch_count() - launches0
    ncell = p["nx"] * p["ny"] * p["nz"]
    pbytes = 4 if precision == "fp32" else 8
    total_iters = steps * iters
    value = world * M.a_eff_bytes(ncell, pbytes) * total_iters / t / 1e9
    out = {"precision": precision, "value": value, "unit": "GB/s", "p_bytes": pbytes,
           "ms_per_step": t / steps * 1e3, "iters_per_step": iters, "it_per_s": world * total_iters / t,
           "t_it_ms": t / total_iters * 1e3, "teff_frac_of_hbm": value / world / peaks()[0],
           "roofline": roofline(kernels, ncell, clk.get("sm_mhz") if clk else None, own),
           "gpu_launches": launches, "clocks": clk,
           "kernels": {k: {"launches": v[0], "ms": v[1]} for k, v in kernels.items()}}
    if e2e_steps > 0:
        host = s.host_mirror()
        s.download(host)
        s.upload(host)                       # one untimed round trip through the fresh buffers
        one_step()
        s.download(host)
        torch.cuda.synchronize(dev)
        barrier()
        h2d = d2h = 0
        per_step = []
        for _ in range(e2e_steps):
            t0 = time.perf_counter()
            h2d = s.upload(host)
            one_step()
            d2h = s.download(host)
            torch.cuda.synchronize(dev)
            per_step.append(M.max_over_ranks(time.perf_counter() - t0, dev))
        # the median step: the host copies share the host's memory bandwidth with whatever else
        # runs on the machine, which the device-side timing never sees
        t_med = sorted(per_step)[len(per_step) // 2]
        out["e2e"] = {"value": world * M.a_eff_bytes(ncell, pbytes) * iters / t_med / 1e9,
                      "unit": "GB/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                      "steps": e2e_steps, "step_seconds": per_step}
        del host
    s.close()
    del s
    torch.cuda.empty_cache()
    return out


def measure_batched(args, steps: int, warmup: int, dev, world: int, rank: int, converge: bool = False,
                    fp32: bool | None = None) -> dict:
    """The batched ensemble (64 instances, sizes {32,48,64,96,127}^3, seeded parameters and
    anomalies; seed = rank): aggregate cell updates per second over `steps` physical steps of
    `--batch-iters` PT iterations each, or one step to convergence with time-to-converge."""
    import torch
    from paper_2207_08716_gb300.solver import PTBatch

    if fp32 is None:
        fp32 = getattr(args, "batch_precision", "fp64") == "fp32"
    # the FP32 form counts its inner FP32 iterations, 2-4x the FP64 form's iterations (at least
    # nup of them per outer Picard update)
    mem = I.ensemble(seed=M.replica_seed(rank), n_inst=args.batch_n, max_iter=160000 if fp32 else 40000)
    if fp32 and getattr(args, "batch_inner_rtol", 0.0) > 0:
        for p, _ in mem:
            p["inner_rtol"] = args.batch_inner_rtol
    if not converge:
        for p, _ in mem:
            p["tol"] = 0.0
            p["max_iter"] = args.batch_iters
    cells = [p["nx"] * p["ny"] * p["nz"] for p, _ in mem]
    from paper_2207_08716_gb300 import native as N
    b = PTBatch(mem, device=dev, precision=N.PT_FP32 if fp32 else N.PT_FP64)
    del mem
    for _ in range(warmup):
        b.step()
    torch.cuda.synchronize(dev)
    clocks = M.ClockSampler(dev.index or 0)
    clocks.start()
    t0 = time.perf_counter()
    iters = [0] * len(cells)
    ttc_all = []
    for _ in range(1 if converge else steps):
        reps, ttc = b.step()
        for m, r in enumerate(reps):
            iters[m] += r["iters"]
        ttc_all = ttc
    torch.cuda.synchronize(dev)
    t = M.max_over_ranks(time.perf_counter() - t0, dev)
    clk = clocks.stop()
    upd = M.sum_over_ranks(float(sum(c * it for c, it in zip(cells, iters))), dev)
    bx, by, ipg = b.config()
    pbytes = 4 if fp32 else 8
    out = {"value": M.a_eff_bytes(1, pbytes) * upd / t / 1e9, "unit": "GB/s",
           "cell_updates_per_s": upd / t, "instances": len(cells), "total_cells": sum(cells),
           "iters_per_step": None if converge else args.batch_iters, "seconds": t,
           "tile": [bx, by], "iters_per_graph": ipg, "clocks": clk,
           "precision": "fp32" if fp32 else "fp64",
           "value_definition": f"T_eff-equivalent: 25 x {pbytes} B x aggregate cell updates per second"
                               + (" (FP32: inner FP32 PT iterations)" if fp32 else "")}
    if fp32:
        out["corr_tile_z"], out["corr_blocks_per_sm"], out["member_groups"] = b.config_fp32()
    if converge:
        st = sorted(ttc_all)
        out.update(statuses=[r["status"] for r in reps], iters=[r["iters"] for r in reps],
                   p50_time_to_converge_ms=st[len(st) // 2],
                   p99_time_to_converge_ms=st[min(len(st) - 1, int(0.99 * len(st)))],
                   converged=sum(1 for r in reps if r["status"] == 0))
    b.close()
    del b
    torch.cuda.empty_cache()
    return out


def measure_mg_step(args, dev, rank: int) -> dict:
    """The FP32 form with multigrid correction solves (`--mg-form-levels` grids) on the benchmark
    workload: one converged physical step (tol 1e-8) after one untimed converged step, timed with
    CUDA events on the solver's stream; the step's iteration count is in finest-grid sweeps."""
    import torch
    from paper_2207_08716_gb300.solver import PTSolver

    n = args.n
    p = workload_params(n, 400000, "fp32", args.workload)
    p["tol"] = I.large_params(n)["tol"]
    p["mg_levels"] = args.mg_form_levels
    phi = workload_phi(p, M.replica_seed(rank), args.workload)
    stream = torch.cuda.current_stream(dev)
    s = PTSolver(p, phi, device=dev, stream=stream)
    del phi
    warm = s.step()
    torch.cuda.synchronize(dev)
    clocks = M.ClockSampler(dev.index or 0)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = s.launch_count()
    e0.record(stream)
    rep = s.step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    out = {"value": e0.elapsed_time(e1) / 1e3, "unit": "s per converged step", "higher_is_better": False,
           "mg_levels": args.mg_form_levels, "fine_sweeps": rep["iters"], "status": rep["status"],
           "warmup_step_fine_sweeps": warm["iters"], "gpu_launches": s.launch_count() - l0, "clocks": clk,
           "definition": f"{n}^3 c1-parameter step to tol {p['tol']:g} (FP32 correction solves by V-cycles, "
                         "FP64 outer loop); the double-float form needs ~37,700 PT iterations for such a step"}
    s.close()
    torch.cuda.empty_cache()
    return out


# the kernels of one adjoint PT iteration (without and with the power law)
ADJ_ITER_KERNELS = ("k_adj_cells", "k_adj_faces", "k_adj_edges_pl", "k_adj_cells_pl", "k_adj_faces_pl")


def measure_adjoint(args, dev) -> dict:
    """Gradient of J = sum (phi^N - phi_target)^2 w.r.t. the log-permeability field: N converged
    steps recorded with checkpoints, then the checkpointed reverse sweep (recompute + adjoint PT
    per step), once per checkpoint spacing. theta and the target's theta are Gaussian random
    fields (corr. length 0.1, std 0.5, seeds 1 and 2); finite-difference directions use seeds
    10, 11, ..."""
    import torch
    from paper_2207_08716_gb300.adjoint import adjoint_scope
    from paper_2207_08716_gb300.solver import PTSolver

    n, N = args.adjoint_n, args.adjoint_steps
    spacings = [int(x) for x in str(args.adjoint_ckpt).split(",") if x]
    p = adjoint_scope(I.c1_params(n))
    p["precision"] = PRECISIONS["fp64"]
    p["max_iter"] = 200000
    phi = I.gaussian_porosity(p, centres=(I.perturbed_centre(0),))
    theta = I.gaussian_random_field(phi.shape, seed=1, corr_len=0.1, std=0.5)
    theta_t = I.gaussian_random_field(phi.shape, seed=2, corr_len=0.1, std=0.5)

    def run_forward(th):
        s = PTSolver(p, phi, logk=th, device=dev)
        its = 0
        for _ in range(N):
            its += s.step()["iters"]
        out = s.get("phi")
        s.close()
        return out, its

    clocks = M.ClockSampler(dev.index or 0)
    t0 = time.perf_counter()
    target, _ = run_forward(theta_t)
    t_target = time.perf_counter() - t0
    ncell = n ** 3
    runs, grad = [], None
    clocks.start()
    for every in spacings:
        s = PTSolver(p, phi, logk=theta, device=dev)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        reps = s.adjoint_forward(N, every)
        t_fwd = time.perf_counter() - t0
        phiN = s.get("phi")
        launches0 = s.launch_count()
        s.profile_begin()
        t0 = time.perf_counter()
        g, rep = s.adjoint(2.0 * (phiN - target))
        torch.cuda.synchronize(dev)
        t_bwd = time.perf_counter() - t0
        kernels = s.profile_end()
        launches = s.launch_count() - launches0
        g = g.cpu().numpy()
        adj_ms = sum(kernels.get(k, (0, 0.0))[1] for k in ADJ_ITER_KERNELS)
        r = {"ckpt_every": every, "forward_s": t_fwd, "backward_s": t_bwd, "cost_multiple": t_bwd / t_fwd,
             "forward_pt_iters": sum(x["iters"] for x in reps), "adjoint_pt_iters": rep["iters"],
             "adjoint_ms_per_iter": adj_ms / max(rep["iters"], 1),
             "forward_statuses": sorted({x["status"] for x in reps}), "adjoint_status": rep["status"],
             "J": float(np.sum((phiN - target) ** 2)), "grad_max": float(np.abs(g).max()),
             "gpu_launches": launches,
             "kernels": {k: {"launches": v[0], "ms": v[1]} for k, v in kernels.items()}}
        # algorithmic bytes of one adjoint PT iteration: cells reads 26 arrays (3 lambda_V, 4 centre
        # multipliers, 3 right-hand sides, phi, 1/(1-phi), 6 Darcy face factors, 5 row factors, V (3))
        # and writes 10 (6 adjoint stresses, 4 multipliers); faces reads 17 (6 stresses, lambda_P,
        # lambda_L/(1-phi), 3 advection factors, 3 lambda_V, 3 R) and writes 6 (3 R, 3 lambda_V).
        # With the power law: edges 10 read + 6 written, cells 50 + 8, faces 20 + 6 (100 arrays).
        arrays = 100 if p.get("powerlaw_on") else 36 + 23
        if adj_ms > 0:
            r["adjoint_gbs"] = arrays * 8 * ncell * rep["iters"] / (adj_ms / 1e3) / 1e9
        if grad is not None:
            r["max_rel_diff_vs_first"] = float(np.abs(g - grad).max() / np.abs(grad).max())
        grad = g if grad is None else grad
        runs.append(r)
        s.close()
        print(json.dumps({"adjoint_run": {k: v for k, v in r.items() if k != "kernels"}}), file=sys.stderr,
              flush=True)
    clk = clocks.stop()
    for r in runs:
        adj = {k: (v["launches"], v["ms"]) for k, v in r["kernels"].items() if k in ADJ_ITER_KERNELS}
        if adj:
            r["roofline"] = roofline(adj, ncell, clk.get("sm_mhz") if clk else None)
    out = {"n": n, "steps": N, "target_forward_s": t_target, "runs": runs, "clocks": clk,
           "model": {"powerlaw_on": int(p.get("powerlaw_on", 0)), "R_weak": p["R_weak"], "beta_n": p["beta_n"],
                     "tau0": p["tau0"], "n_pow": p["n_pow"]}}
    if args.adjoint_fd > 0:
        eps = 1e-6 * float(np.abs(theta).max())
        checks = []
        for d in range(args.adjoint_fd):
            v = I.gaussian_random_field(phi.shape, seed=10 + d, corr_len=0.1, std=1.0)
            Jp = float(np.sum((run_forward(theta + eps * v)[0] - target) ** 2))
            Jm = float(np.sum((run_forward(theta - eps * v)[0] - target) ** 2))
            fd = (Jp - Jm) / (2 * eps)
            ad = float(np.sum(grad * v))
            checks.append({"seed": 10 + d, "adjoint": ad, "fd": fd, "rel": abs(ad - fd) / abs(fd)})
            print(json.dumps({"fd_check": checks[-1]}), file=sys.stderr, flush=True)
        out["fd_checks"] = checks
        out["fd_eps"] = eps
    torch.cuda.empty_cache()
    return out


def measure_reactive(args, dev) -> dict:
    """Reactive porosity-wave solver (thesis Art. 3; appendix A.6 parameters, Da = 100,
    dt = 1e-6) on n x n x 4n cells: `--steps` physical steps of `--rx-iters` PT iterations after
    `--warmup` steps, FP32 (the thesis's precision for this solver) and FP64; T_eff = 7 N p / t_it
    (3 unknowns read and written, 1 known field read, Art. 3); the fused iteration kernel moves
    10 arrays per cell (Pf, phi with neighbours, Xs, 3 old-step fields read; Pf, phi, Xs written)."""
    import torch
    from paper_2207_08716_gb300 import native as N
    from paper_2207_08716_gb300.solver import RXSolver

    n = args.rx_n
    out = {}
    for prec, pbytes in (("fp32", 4), ("fp64", 8)):
        p = I.rx_params(n)
        p["precision"] = N.PT_FP32 if prec == "fp32" else N.PT_FP64
        Pf, phi, Xs = I.rx_initial(p)
        s = RXSolver(p, Pf, phi, Xs, device=dev)
        del Pf, phi, Xs
        for _ in range(args.warmup):
            s.iterate(args.rx_iters)
        torch.cuda.synchronize(dev)
        clocks = M.ClockSampler(dev.index or 0)
        clocks.start()
        l0 = s.launch_count()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s.stream)
        for _ in range(args.steps):
            s.iterate(args.rx_iters)
        e1.record(s.stream)
        torch.cuda.synchronize(dev)
        clk = clocks.stop()
        t = e0.elapsed_time(e1) / 1e3
        ncell = p["nx"] * p["ny"] * p["nz"]
        iters = args.steps * args.rx_iters
        t_it = t / iters
        hbm, hbm_kind = peaks()
        kern_gbs = 10 * pbytes * ncell / t_it / 1e9
        out[prec] = {"value": 7 * pbytes * ncell / t_it / 1e9, "unit": "GB/s", "t_it_ms": t_it * 1e3,
                     "it_per_s": 1.0 / t_it, "cells": ncell, "grid": [p["nx"], p["ny"], p["nz"]],
                     "gpu_launches": s.launch_count() - l0, "clocks": clk,
                     "roofline": {"kernel": "k_rx_iter (whole step, begin/end and checks included)",
                                  "bound": "hbm", "achieved": kern_gbs, "peak": hbm, "unit": "GB/s",
                                  "frac": kern_gbs / hbm, "traffic": None,
                                  "algorithmic_bytes_per_cell": 10 * pbytes}}
        s.close()
        del s
        torch.cuda.empty_cache()
    return out


def _oracle_steps_job(n: int, nsteps: int, out_path: str) -> dict:
    """The oracle's `nsteps` converged physical steps of the c1 workload at n^3 (run in a child
    process by the precision check); the final porosity goes to `out_path` (.npy)."""
    import oracle as O
    p = I.c1_params(n)
    p["max_iter"] = 400000
    st = O.make_state(p, I.gaussian_porosity(p))
    iters, t0 = [], time.perf_counter()
    for _ in range(nsteps):
        rc, it, _ = O.step(st)
        if rc != 0:
            raise RuntimeError(f"oracle rc {rc}")
        iters.append(it)
    dt = time.perf_counter() - t0
    np.save(out_path, st["phi"])
    return {"n": n, "steps": nsteps, "iters": iters, "seconds": dt, "cores": O.max_threads()}


def _parse_sizes(spec: str, default_steps: int) -> list:
    """'127:3,511:1,32' -> [(127, 3), (511, 1), (32, default_steps)]."""
    out = []
    for tok in spec.split(","):
        tok = tok.strip()
        if tok:
            n, _, k = tok.partition(":")
            out.append((int(n), int(k) if k else default_steps))
    return out


def measure_precision(args, dev) -> dict:
    """The FP32 + FP64 defect-correction form against an FP64-class form (--pc-ref: the FP64-lean
    or the double-float form, which matches the FP64 oracle to 1e-10) after converged physical
    steps of the c1 workload (one centred anomaly), both on the GPU from the same state; at the
    sizes of --pc-oracle-n also against the FP64 oracle's converged steps, which run on the host
    cores in a child process started before the first GPU call. --pc-n lists n[:steps] entries.
    Porosity error = max |phi - phi_ref| / max |phi_ref| and, more telling, relative to the
    porosity change over the run, max |phi - phi_ref| / max |phi_ref - phi_initial|."""
    import subprocess
    import tempfile
    import torch
    from paper_2207_08716_gb300 import native as N
    from paper_2207_08716_gb300.solver import PTSolver

    sizes = _parse_sizes(args.pc_n, args.pc_steps)
    oracle_n = {int(v) for v in str(args.pc_oracle_n).split(",") if v.strip()} if args.pc_oracle else set()
    ref_prec = {"fp64": N.PT_FP64, "df64": N.PT_DF64, "none": None}[args.pc_ref]
    tmp = tempfile.mkdtemp(prefix="pc_oracle_")
    children = {}
    ncores = os.cpu_count() or 1
    for n, k in sizes:
        if n in oracle_n:
            path = os.path.join(tmp, f"phi_{n}.npy")
            code = f"import json, bench; print('ORACLE ' + json.dumps(bench._oracle_steps_job({n}, {k}, {path!r})))"
            env = dict(os.environ, OMP_NUM_THREADS=str(max(1, ncores - 1)))
            children[n] = (subprocess.Popen([sys.executable, "-c", code], cwd=ROOT, env=env, stdout=subprocess.PIPE,
                                            stderr=subprocess.PIPE, text=True), path)

    def run(p, phi0, nsteps):
        s = PTSolver(p, phi0, device=dev)
        iters, t0 = [], time.perf_counter()
        for _ in range(nsteps):
            r = s.step(raise_on_notconv=False)
            iters.append(r["iters"])
            if r["status"] != 0:
                print(json.dumps({"not_converged": {"n": p["nx"], "precision": p["precision"],
                                                    "mg_levels": p.get("mg_levels", 0), "report": r}}),
                      file=sys.stderr, flush=True)
        torch.cuda.synchronize(dev)
        t = time.perf_counter() - t0
        phi = s.get("phi")
        s.close()
        return phi, iters, t

    def errs(a, ref, phi0):
        d = float(np.abs(a - ref).max())
        return {"max_rel": d / float(np.abs(ref).max()), "rel_to_change": d / float(np.abs(ref - phi0).max())}

    out = {"reference_form": args.pc_ref}
    for n, k in sizes:
        p = I.c1_params(n)
        p["max_iter"] = 400000
        phi0 = I.gaussian_porosity(p)
        if ref_prec is None:   # the multigrid form alone (launch lists)
            phimg, itmg, tmg = run(dict(p, precision=N.PT_FP32, mg_levels=args.pc_mg), phi0, k)
            out[str(n)] = {"steps": k, "fp32mg_levels": args.pc_mg, "fp32mg_iters": sum(itmg), "fp32mg_s": tmg}
            continue
        phi64, it64, t64 = run(dict(p, precision=ref_prec), phi0, k)
        r = {"steps": k, "ref_iters": sum(it64), "ref_s": t64, "porosity_change_max": float(np.abs(phi64 - phi0).max())}
        phi32 = None
        if n <= args.pc_plain_max:
            phi32, it32, t32 = run(dict(p, precision=N.PT_FP32), phi0, k)
            r.update(fp32_iters=sum(it32), fp32_s=t32, fp32_vs_ref=errs(phi32, phi64, phi0))
        L = args.pc_mg
        nc = n
        for _ in range(max(L - 1, 0)):
            nc = (nc + 1) // 2                     # each level ceil(n / 2) cells per direction
        if L >= 2 and nc >= 2:
            phimg, itmg, tmg = run(dict(p, precision=N.PT_FP32, mg_levels=L), phi0, k)
            r.update(fp32mg_levels=L, fp32mg_iters=sum(itmg), fp32mg_s=tmg, fp32mg_vs_ref=errs(phimg, phi64, phi0))
            if phi32 is not None:
                r["fp32mg_vs_fp32"] = errs(phimg, phi32, phi0)
        print(json.dumps({"precision_check": {str(n): r}}), file=sys.stderr, flush=True)
        if n in children:
            proc, path = children.pop(n)
            so, se = proc.communicate()
            line = [l for l in so.splitlines() if l.startswith("ORACLE ")]
            if proc.returncode != 0 or not line:
                r["oracle_error"] = (se or "")[-300:]
            else:
                rec = json.loads(line[-1][7:])
                phio = np.load(path)
                r["oracle_s"], r["oracle_iters"], r["oracle_cores"] = rec["seconds"], sum(rec["iters"]), rec["cores"]
                r["ref_vs_oracle"] = errs(phi64, phio, phi0)
                if phi32 is not None:
                    r["fp32_vs_oracle"] = errs(phi32, phio, phi0)
                if "fp32mg_levels" in r:
                    r["fp32mg_vs_oracle"] = errs(phimg, phio, phi0)
                os.remove(path)
        out[str(n)] = r
        torch.cuda.empty_cache()
    for proc, _ in children.values():
        proc.kill()
    if not os.listdir(tmp):
        os.rmdir(tmp)
    return out


MG_DEFAULT = dict(nu_pre=2, nu_post=2, nu_coarse=30, max_cycles=100, omega=6.0 / 7.0)


def measure_reactive_mg(args, dev) -> dict:
    """Multigrid-accelerated reactive step (FAS V-cycles smoothed by the PT iteration with local
    pseudo steps) against the plain PT iteration, on the reactive workload of Art. 3 (Da = 100,
    dt = 1e-6, tol 2e-8) on n x n x 4n cells: both solvers advance the same physical steps from
    the same state; time to a converged step with CUDA events (host reads of the change norm
    included: they decide when to stop). FP32 (the thesis's precision for this solver) for both;
    FP64 for the multigrid form. The fine-grid sweep (k_mg_smooth, the dominant kernel) is timed
    alone for its roofline: 6 arrays read (Pf, phi with neighbours, Xs, 3 old-step fields) and
    3 written per cell."""
    import torch
    from paper_2207_08716_gb300 import native as N
    from paper_2207_08716_gb300.solver import RXSolver

    n = args.mg_n
    mg = dict(MG_DEFAULT, levels=args.mg_levels)
    if args.mg_sweeps:
        mg.update(zip(("nu_pre", "nu_post", "nu_coarse"), (int(v) for v in args.mg_sweeps.split(","))))
    hbm, hbm_kind = peaks()
    out = {"mg": mg}

    def timed(s, fn, nsteps):
        torch.cuda.synchronize(dev)
        l0 = s.launch_count()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = []
        e0.record(s.stream)
        for _ in range(nsteps):
            reps.append(fn())
        e1.record(s.stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / nsteps, reps, s.launch_count() - l0

    for prec, pbytes in (("fp32", 4), ("fp64", 8)):
        if prec not in args.mg_precisions.split(","):
            continue
        p = I.rx_params(n)
        p["precision"] = N.PT_FP32 if prec == "fp32" else N.PT_FP64
        Pf, phi, Xs = I.rx_initial(p)
        ncell = p["nx"] * p["ny"] * p["nz"]
        r = {"grid": [p["nx"], p["ny"], p["nz"]], "cells": ncell}
        s = RXSolver(p, Pf, phi, Xs, device=dev, mg=mg)
        for _ in range(args.warmup):
            s.mg_step(raise_on_notconv=True)
        clocks = M.ClockSampler(dev.index or 0)
        clocks.start()
        ms, reps, launches = timed(s, lambda: s.mg_step(raise_on_notconv=True), args.steps)
        r["multigrid"] = {"ms_per_step": ms, "cycles": [q["iters"] for q in reps],
                          "change": [q["r_v"] for q in reps], "gpu_launches": launches}
        r["clocks"] = clocks.stop()
        s.close()
        # the fine-grid sweep alone: a one-level hierarchy of nu_coarse sweeps per cycle
        one = RXSolver(p, Pf, phi, Xs, device=dev, mg=dict(mg, levels=1, nu_coarse=50))
        one.mg_cycles(1)
        t_cyc, _, _ = timed(one, lambda: one.mg_cycles(1), 3)
        one.close()
        t_sweep = t_cyc / 50 / 1e3
        gbs = 9 * pbytes * ncell / t_sweep / 1e9
        traffic_cell = profiled(f"k_mg_smooth_{prec}").get("traffic")
        r["roofline"] = {"kernel": "k_mg_smooth (finest grid)", "bound": "hbm", "achieved": gbs, "peak": hbm,
                         "unit": "GB/s", "frac": gbs / hbm,
                         "traffic": traffic_cell * ncell if traffic_cell else None,
                         "algorithmic_bytes_per_cell": 9 * pbytes, "peak_kind": hbm_kind, "sweep_ms": t_sweep * 1e3}
        if prec == "fp32" and args.mg_plain_steps > 0:
            b = RXSolver(dict(p, max_iter=200000), Pf, phi, Xs, device=dev)
            for _ in range(args.warmup):
                b.step(raise_on_notconv=True)
            ms_b, reps_b, launches_b = timed(b, lambda: b.step(raise_on_notconv=True), args.mg_plain_steps)
            r["plain"] = {"ms_per_step": ms_b, "iters": [q["iters"] for q in reps_b], "gpu_launches": launches_b,
                          "steps": args.mg_plain_steps}
            r["speedup"] = ms_b / ms
            b.close()
        out[prec] = r
        del Pf, phi, Xs
        torch.cuda.empty_cache()
    return out


def run_native(args):
    import torch
    import torch.distributed as dist

    rank, local_rank, world = M.rank_env()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if world > 1 and not dist.is_initialized():
        dist.init_process_group("nccl", device_id=dev)

    if args.reactive:
        if rank == 0:
            r = measure_reactive(args, dev)
            print(json.dumps({"metric": "reactive porosity-wave solver T_eff (A_eff = 7 N p)",
                              "value": r["fp32"]["value"], "unit": "GB/s", "dtype": "f32",
                              "config": {"workload": f"reactive porosity waves (Art. 3, Da = 100), "
                                                     f"{args.rx_n}x{args.rx_n}x{4 * args.rx_n} cells, "
                                                     f"{args.rx_iters} PT iterations per step"},
                              "forms": r}), flush=True)
        return 0
    if args.precision_check:
        if rank == 0:
            r = measure_precision(args, dev)
            print(json.dumps({"metric": "porosity error of the FP32 form after converged steps", "unit": "max rel",
                              "config": {"workload": "c1 workload (one centred anomaly), converged physical "
                                                     f"steps per grid (n:steps) {args.pc_n}",
                                         "reference_form": args.pc_ref}, "grids": r}), flush=True)
        return 0
    if args.reactive_mg:
        if rank == 0:
            r = measure_reactive_mg(args, dev)
            f32 = r["fp32"] if "fp32" in r else r["fp64"]
            print(json.dumps({"metric": "reactive step time-to-solution (multigrid-accelerated PT)",
                              "value": f32["multigrid"]["ms_per_step"], "unit": "ms per converged step",
                              "higher_is_better": False, "dtype": "f32" if "fp32" in r else "f64",
                              "steps": args.steps,
                              "warmup": args.warmup,
                              "config": {"workload": f"reactive porosity waves (Art. 3, Da = 100, dt = 1e-6, "
                                                     f"tol 2e-8), {args.mg_n}x{args.mg_n}x{4 * args.mg_n} cells, "
                                                     f"FAS V({r['mg']['nu_pre']},{r['mg']['nu_post']}) "
                                                     f"cycles on {args.mg_levels} levels"},
                              "gpu_launches": f32["multigrid"]["gpu_launches"], "roofline": f32["roofline"],
                              "forms": r}), flush=True)
        return 0
    if args.adjoint:
        if rank == 0:
            r = measure_adjoint(args, dev)
            print(json.dumps({"metric": "adjoint gradient dJ/dlogk: cost multiple of the forward", **r}),
                  flush=True)
        return 0
    if args.batched_converge:
        r = measure_batched(args, 1, 0, dev, world, rank, converge=True)
        if rank == 0:
            print(json.dumps({"metric": "batched ensemble time-to-converge", **r}), flush=True)
        return 0
    head_iters = args.fp32_iters if args.precision == "fp32" else args.iters
    own = None if args.no_own_peaks else measure_own_peaks(dev)
    seeds = [int(v) for v in args.seeds.split(",") if v.strip()] if world == 1 else [None]
    runs = []
    for m, sd in enumerate(seeds or [None]):
        r = measure_form(args, args.precision, head_iters, args.steps, args.warmup,
                         args.e2e_steps if m == 0 else 0, dev, world, rank, local_rank, seed=sd, own=own)
        r["seed"] = sd if sd is not None else M.replica_seed(rank)
        runs.append(r)
    head = sorted(runs, key=lambda r: r["value"])[len(runs) // 2]      # the median seed's run
    if "e2e" in runs[0]:
        head["e2e"] = runs[0]["e2e"]
    forms = {}
    for f in [x for x in args.forms.split(",") if x and x != args.precision]:
        if f in ("batched", "batched32"):
            forms[f] = measure_batched(args, max(2, args.steps // 2), 1, dev, world, rank, fp32=f == "batched32")
        elif f == "fp32mg":
            forms[f] = measure_mg_step(args, dev, rank)
        elif f in PRECISIONS:
            it = args.fp32_iters if f == "fp32" else args.iters
            forms[f] = measure_form(args, f, it, max(2, args.steps // 2), 2, 0, dev, world, rank, local_rank,
                                    own=own)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_sample(args.cpu_n, args.cpu_iters)

    if rank == 0:
        line = {
            "metric": METRIC, "value": head["value"], "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPES[args.precision], "data": "synthetic",
            "config": native_config(args, head["iters_per_step"], world),
            "it_per_s": head["it_per_s"], "t_it_ms": head["t_it_ms"],
            "seeds": {str(r["seed"]): r["value"] for r in runs}, "median_seed": head["seed"],
            "teff_frac_of_hbm": head["teff_frac_of_hbm"], "roofline": head["roofline"],
            "cpu_baseline": cpu, "e2e": head.get("e2e"), "gpu_launches": head["gpu_launches"],
            "clocks": head["clocks"], "kernels": head["kernels"], "own_peaks": own,
            "forms": {k: ({kk: v[kk] for kk in ("value", "unit", "p_bytes", "it_per_s", "t_it_ms",
                                                  "teff_frac_of_hbm", "iters_per_step", "roofline",
                                                  "gpu_launches", "clocks")}
                          if not (k.startswith("batched") or k == "fp32mg") else v)
                      for k, v in forms.items()},
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.source_hashes:
        print(json.dumps({k: source_hash(k) for k in KERNEL_SOURCES}, indent=1))
        return 0
    if args.cpu_timings:
        print(json.dumps({"metric": "oracle t_it and T_eff on the host cores (baseline)", **cpu_timings(args)}),
              flush=True)
        return 0
    if args.impl == "reference":
        return run_reference(args)
    return run_native(args)


if __name__ == "__main__":
    sys.exit(main())
