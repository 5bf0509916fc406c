"""Build and load the CUDA library (libpt_gb300.so) and declare its C ABI for ctypes.

The library is compiled in-tree with nvcc for sm_103a (``build_library``). Loading never falls
back to anything: if the shared object is missing or fails to load, ``load`` raises.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

_PKG = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_PKG)
_CSRC = os.path.join(_PKG, "csrc")
_INC = os.path.join(_ROOT, "include")
_BUILD = os.path.join(_PKG, "_build")
LIB_PATH = os.path.join(_BUILD, "libpt_gb300.so")
SOURCES = ("pt_api.cu", "pt_ref_kernels.cu", "pt_lean_kernels.cu", "pt_mixed_kernels.cu",
           "pt_batch_kernels.cu", "pt_adjoint_kernels.cu", "pt_dd_kernels.cu", "pt_static.cu", "pt_peaks.cu",
           "rx_api.cu", "rx_kernels.cu", "rx_mg_kernels.cu")
HEADERS = ("pt_common.cuh", "pt_host.h", "pt_kernels.cuh", "pt_ref_points.cuh", "pt_lean.cuh", "pt_lean_body.cuh", "df64.cuh", "pt_mixed.cuh", "pt_batch.cuh", "pt_adjoint.cuh", "pt_dd.cuh", "rx.cuh")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"

_lock = threading.Lock()
_lib = None

PT_OK, PT_EINVAL, PT_ENOTCONV, PT_ENAN, PT_ETIMEOUT, PT_ECUDA, PT_ESPACE = 0, -1, -2, -3, -4, -5, -6
PT_FP64, PT_FP32, PT_FP64_STEPWISE, PT_DF64 = 0, 1, 2, 3


def _inputs():
    files = [os.path.join(_CSRC, s) for s in SOURCES + HEADERS]
    files.append(os.path.join(_INC, "porowave_pt.h"))
    files.append(os.path.join(_INC, "porowave_rx.h"))
    return files


def build_library(force: bool = False, verbose: bool = False) -> str:
    """Compile every .cu of the library into _build/libpt_gb300.so (objects in parallel)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(f) for f in _inputs())
    if not force and os.path.exists(LIB_PATH) and os.path.getmtime(LIB_PATH) >= newest:
        return LIB_PATH
    flags = [ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", f"-I{_INC}"]
    procs, objs = [], []
    for s in SOURCES:
        obj = os.path.join(_BUILD, s.replace(".cu", f".{os.getpid()}.o"))
        objs.append(obj)
        procs.append(subprocess.Popen(["nvcc", *flags, "-c", os.path.join(_CSRC, s), "-o", obj],
                                      stdout=None if verbose else subprocess.PIPE,
                                      stderr=subprocess.STDOUT))
    for p, s in zip(procs, SOURCES):
        out, _ = p.communicate()
        if p.returncode != 0:
            raise RuntimeError(f"nvcc failed on {s}:\n{(out or b'').decode(errors='replace')}")
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    subprocess.run(["nvcc", ARCH, "-shared", "-o", tmp, *objs], check=True)
    os.replace(tmp, LIB_PATH)
    for o in objs:
        os.remove(o)
    return LIB_PATH


class Grid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("lx", C.c_double), ("ly", C.c_double), ("lz", C.c_double)]


class Phys(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("phi0", "k0", "mu0", "eta0", "R_weak", "n_pow", "tau0",
                                          "alpha", "B", "beta_d", "beta_phi", "G", "rhof_g",
                                          "rhos_g")] + \
               [("powerlaw_on", C.c_int32), ("compaction_on", C.c_int32), ("tau_bg", C.c_double)]


class Num(C.Structure):
    _fields_ = [("dt", C.c_double), ("tol", C.c_double), ("max_iter", C.c_int32),
                ("nup", C.c_int32), ("damp", C.c_double * 3), ("rho_i", C.c_double),
                ("beta_n", C.c_double), ("rel_mu", C.c_double), ("rel_eta", C.c_double),
                ("cfl_v", C.c_double), ("cfl_pf", C.c_double), ("dtpt_scale", C.c_double),
                ("xsi_w", C.c_double), ("precision", C.c_int32), ("iters_per_graph", C.c_int32),
                ("inner_rtol", C.c_double), ("mg_levels", C.c_int32), ("mg_reserved", C.c_int32)]


FIELD_NAMES = ("Vx", "Vy", "Vz", "Pt", "Pf", "phi", "txx", "tyy", "tzz", "txy", "txz", "tyz",
               "mu", "eta")


class Fields(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in FIELD_NAMES] + [("logk", C.c_void_p)]


class Report(C.Structure):
    _fields_ = [("iters", C.c_int32), ("status", C.c_int32), ("res_v", C.c_double),
                ("res_pt", C.c_double), ("res_pf", C.c_double), ("res_pic", C.c_double)]

    def as_dict(self) -> dict:
        return dict(iters=self.iters, status=self.status, r_v=self.res_v, r_pt=self.res_pt,
                    r_pf=self.res_pf, r_pic=self.res_pic)


def grid_from(p: dict) -> Grid:
    return Grid(p["nx"], p["ny"], p["nz"], p["lx"], p["ly"], p["lz"])


def phys_from(p: dict) -> Phys:
    ph = Phys()
    for n, _ in Phys._fields_:
        setattr(ph, n, p.get(n, 0.0) if n == "tau_bg" else p[n])
    return ph


def num_from(p: dict, precision: int = PT_FP64, iters_per_graph: int = 0) -> Num:
    nm = Num()
    for n, _ in Num._fields_:
        if n == "damp":
            nm.damp[0], nm.damp[1], nm.damp[2] = p["damp_x"], p["damp_y"], p["damp_z"]
        elif n == "precision":
            nm.precision = p.get("precision", precision)
        elif n == "iters_per_graph":
            nm.iters_per_graph = p.get("iters_per_graph", iters_per_graph)
        elif n == "inner_rtol":
            nm.inner_rtol = p.get("inner_rtol", 0.0)
        elif n == "mg_levels":
            nm.mg_levels = p.get("mg_levels", 0)
        elif n == "mg_reserved":
            nm.mg_reserved = 0
        else:
            setattr(nm, n, p[n])
    return nm


class OldFields(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("Pto", "Pfo", "txxo", "tyyo", "tzzo", "txyo", "txzo", "tyzo")]


class RxPhys(C.Structure):
    _fields_ = [(k, C.c_double) for k in ("phi0", "k0", "eta", "rhof", "rhos", "g", "beta_d", "beta_s", "beta_f",
                                          "beta_x", "dX", "xs_max", "tau")]


class RxNum(C.Structure):
    _fields_ = [("dt", C.c_double), ("tol", C.c_double), ("cfl_div", C.c_double), ("pf_scale", C.c_double),
                ("max_iter", C.c_int32), ("nup", C.c_int32), ("precision", C.c_int32)]


class RxMg(C.Structure):
    _fields_ = [(k, C.c_int32) for k in ("levels", "nu_pre", "nu_post", "nu_coarse", "max_cycles")] + \
               [("omega", C.c_double)]


class RxFields(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in ("Pf", "phi", "Xs", "R")]


class AdjVec(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("Vx", "Vy", "Vz", "Pt", "Pf", "phi", "mu")]


class KernelTime(C.Structure):
    _fields_ = [("name", C.c_char * 24), ("launches", C.c_int64), ("total_ms", C.c_double)]


# Every exported symbol of include/porowave_pt.h with its ctypes signature.
SIGNATURES = {
    "pt_field_elems": (C.c_size_t, [C.POINTER(Grid)]),
    "pt_pitch_x": (C.c_int32, [C.POINTER(Grid)]),
    "pt_workspace_size": (C.c_size_t, [C.POINTER(Grid), C.POINTER(Num)]),
    "pt_init": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(Grid), C.POINTER(Phys), C.POINTER(Num),
                          C.POINTER(Fields), C.c_void_p, C.c_size_t, C.c_void_p, C.c_int32]),
    "pt_step": (C.c_int, [C.c_void_p, C.POINTER(Report)]),
    "pt_step_begin": (C.c_int, [C.c_void_p]),
    "pt_iterate": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.POINTER(Report)]),
    "pt_step_end": (C.c_int, [C.c_void_p]),
    "pt_residual": (C.c_int, [C.c_void_p, C.POINTER(Report)]),
    "pt_profile_begin": (C.c_int, [C.c_void_p]),
    "pt_profile_end": (C.c_int, [C.c_void_p, C.POINTER(KernelTime), C.c_int32, C.POINTER(C.c_int32)]),
    "pt_launch_count": (C.c_int64, [C.c_void_p]),
    "pt_peak_copy": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t, C.c_int32, C.c_void_p,
                               C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "pt_peak_arith": (C.c_int, [C.c_int32, C.c_void_p, C.c_int32, C.c_int32, C.c_void_p,
                                C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "pt_math_check": (C.c_int, [C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]),
    "pt_residual_static": (C.c_int, [C.POINTER(Grid), C.POINTER(Phys), C.POINTER(Num), C.POINTER(Fields),
                                     C.POINTER(OldFields), C.c_double, C.c_void_p, C.POINTER(Report)]),
    "pt_adjoint_workspace_size": (C.c_size_t, [C.POINTER(Grid), C.c_int32, C.c_int32]),
    "pt_adjoint_forward": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_size_t, C.POINTER(Report)]),
    "pt_adjoint": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(Report)]),
    "pt_adjoint_apply": (C.c_int, [C.c_void_p, C.POINTER(AdjVec), C.POINTER(AdjVec), C.c_void_p, C.c_size_t]),
    "rx_workspace_size": (C.c_size_t, [C.POINTER(Grid), C.POINTER(RxNum)]),
    "rx_init": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(Grid), C.POINTER(RxPhys), C.POINTER(RxNum),
                          C.POINTER(RxFields), C.c_void_p, C.c_size_t, C.c_void_p]),
    "rx_step": (C.c_int, [C.c_void_p, C.POINTER(Report)]),
    "rx_iterate": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(Report)]),
    "rx_mg_workspace_size": (C.c_size_t, [C.POINTER(Grid), C.POINTER(RxNum), C.POINTER(RxMg)]),
    "rx_mg_init": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(Grid), C.POINTER(RxPhys), C.POINTER(RxNum),
                             C.POINTER(RxMg), C.POINTER(RxFields), C.c_void_p, C.c_size_t, C.c_void_p]),
    "rx_mg_step": (C.c_int, [C.c_void_p, C.POINTER(Report)]),
    "rx_mg_cycles": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(Report)]),
    "rx_launch_count": (C.c_longlong, [C.c_void_p]),
    "rx_destroy": (None, [C.c_void_p]),
    "pt_dd_workspace_size": (C.c_size_t, [C.POINTER(Grid), C.POINTER(Num), C.POINTER(C.c_int32)]),
    "pt_dd_init": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(Grid), C.POINTER(Phys), C.POINTER(Num),
                             C.POINTER(Fields), C.POINTER(C.c_int32), C.c_void_p, C.c_size_t, C.c_void_p]),
    "pt_dd_step": (C.c_int, [C.c_void_p, C.POINTER(Report)]),
    "pt_dd_gather": (C.c_int, [C.c_void_p]),
    "pt_dd_config": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                               C.POINTER(C.c_int32)]),
    "pt_dd_destroy": (None, [C.c_void_p]),
    "pt_batch_workspace_size": (C.c_size_t, [C.c_int32, C.POINTER(Grid), C.POINTER(Num)]),
    "pt_batch_init": (C.c_int, [C.POINTER(C.c_void_p), C.c_int32, C.POINTER(Grid), C.POINTER(Phys),
                                C.POINTER(Num), C.POINTER(Fields), C.c_void_p, C.c_size_t, C.c_void_p]),
    "pt_batch_step": (C.c_int, [C.c_void_p, C.POINTER(Report), C.POINTER(C.c_double)]),
    "pt_batch_config": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "pt_batch_config_fp32": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                       C.POINTER(C.c_int32)]),
    "pt_mg_axis_words": (C.c_size_t, [C.c_int32]),
    "pt_mg_axis_tables": (C.c_int, [C.c_int32, C.c_void_p, C.c_size_t]),
    "pt_batch_destroy": (None, [C.c_void_p]),
    "pt_destroy": (None, [C.c_void_p]),
    "pt_strerror": (C.c_char_p, [C.c_int]),
}


def load(build: bool = True) -> C.CDLL:
    """Load libpt_gb300.so (building it first if `build`); raises if it cannot be loaded."""
    global _lib
    with _lock:
        if _lib is None:
            if build:
                build_library()
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"CUDA library {LIB_PATH} is missing; run "
                                   "paper_2207_08716_gb300.native.build_library() on a machine with nvcc")
            lib = C.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def strerror(code: int) -> str:
    return load().pt_strerror(code).decode()
