"""Reactive porosity-wave oracle (thesis Art. 3, Eqs. 8-10; appendix A.6) — TEST
INFRASTRUCTURE ONLY. ctypes front end of rx_oracle.c on numpy arrays of shape (nz, ny, nx)."""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import binding as B

RX_KEYS = ("nx", "ny", "nz", "lx", "ly", "lz", "phi0", "k0", "eta", "rhof", "rhos", "g", "beta_d",
           "beta_s", "beta_f", "beta_x", "dX", "xs_max", "tau", "dt", "tol", "cfl_div", "pf_scale",
           "max_iter", "nup")
_INT = ("nx", "ny", "nz", "max_iter", "nup")


class RxParams(C.Structure):
    _fields_ = ([(k, C.c_int) for k in ("nx", "ny", "nz")] +
                [(k, C.c_double) for k in ("lx", "ly", "lz", "phi0", "k0", "eta", "rhof", "rhos", "g",
                                          "beta_d", "beta_s", "beta_f", "beta_x", "dX", "xs_max", "tau",
                                          "dt", "tol", "cfl_div", "pf_scale")] +
                [(k, C.c_int) for k in ("max_iter", "nup")])

    @classmethod
    def from_dict(cls, d: dict) -> "RxParams":
        p = cls()
        for name, _ in cls._fields_:
            setattr(p, name, int(d[name]) if name in _INT else float(d[name]))
        return p


_FIELDS = ("Pf", "phi", "Xs", "R", "Pf_o", "phi_o", "Xs_o")


class RxMgParams(C.Structure):
    _fields_ = [(k, C.c_int) for k in ("levels", "nu_pre", "nu_post", "nu_coarse", "max_cycles")] + \
               [("omega", C.c_double)]

    @classmethod
    def from_dict(cls, d: dict) -> "RxMgParams":
        m = cls()
        for name, _ in cls._fields_:
            setattr(m, name, float(d[name]) if name == "omega" else int(d[name]))
        return m


class RxStateC(C.Structure):
    _fields_ = [(k, C.POINTER(C.c_double)) for k in _FIELDS] + [("dtau", C.c_double)]


_lib = None


def _L():
    global _lib
    if _lib is None:
        B.build()
        lib = C.CDLL(B.lib_path())
        P, S, D = C.POINTER(RxParams), C.POINTER(RxStateC), C.POINTER(C.c_double)
        lib.rx_begin_step.argtypes = [P, S]
        lib.rx_iteration.argtypes = [P, S, C.c_int, D]
        lib.rx_step.argtypes = [P, S, C.POINTER(C.c_int), D]
        lib.rx_iterate_n.argtypes = [P, S, C.c_int, D]
        lib.rx_div_qd.argtypes = [P, D, D, D]
        lib.rx_pseudo_step.argtypes = [P, D]
        lib.rx_pseudo_step.restype = C.c_double
        lib.rx_xseq.argtypes = [P, C.c_double]
        lib.rx_xseq.restype = C.c_double
        M = C.POINTER(RxMgParams)
        lib.rx_mg_step.argtypes = [P, M, S, C.POINTER(C.c_int), D]
        lib.rx_mg_cycles_n.argtypes = [P, M, S, C.c_int, D]
        lib.rx_mg_restrict.argtypes = [C.c_int, C.c_int, C.c_int, D, D]
        lib.rx_mg_prolong_add.argtypes = [C.c_int, C.c_int, C.c_int, D, D]
        lib.rx_mg_equations.argtypes = [P] + [D] * 9 + [C.c_double] + [D] * 5
        for f in ("rx_begin_step", "rx_iteration", "rx_step", "rx_iterate_n", "rx_mg_step", "rx_mg_cycles_n"):
            getattr(lib, f).restype = C.c_int
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


class RxState:
    """Oracle state: numpy arrays (nz, ny, nx) and the C struct pointing at them."""

    def __init__(self, p: dict, Pf, phi, Xs, R=None):
        self.p = dict(p)
        self.cp = RxParams.from_dict(self.p)
        shape = (p["nz"], p["ny"], p["nx"])
        self.a = {k: np.zeros(shape) for k in _FIELDS}
        self.a["Pf"][...] = Pf
        self.a["phi"][...] = phi
        self.a["Xs"][...] = Xs
        if R is not None:
            self.a["R"][...] = R
        self.c = RxStateC(*[_ptr(self.a[k]) for k in _FIELDS], 0.0)

    def __getitem__(self, k):
        return self.a[k]

    @property
    def dtau(self):
        return self.c.dtau


def step(st: RxState):
    it, ch = C.c_int(0), C.c_double(0.0)
    rc = _L().rx_step(C.byref(st.cp), C.byref(st.c), C.byref(it), C.byref(ch))
    return rc, it.value, ch.value


def iterate_n(st: RxState, niter: int):
    ch = C.c_double(0.0)
    rc = _L().rx_iterate_n(C.byref(st.cp), C.byref(st.c), niter, C.byref(ch))
    return rc, ch.value


def div_qd(p: dict, Pf, phi) -> np.ndarray:
    cp = RxParams.from_dict(p)
    Pf = np.ascontiguousarray(Pf, dtype=float)
    phi = np.ascontiguousarray(phi, dtype=float)
    out = np.zeros_like(Pf)
    _L().rx_div_qd(C.byref(cp), _ptr(Pf), _ptr(phi), _ptr(out))
    return out


def pseudo_step(p: dict, phi) -> float:
    phi = np.ascontiguousarray(phi, dtype=float)
    return _L().rx_pseudo_step(C.byref(RxParams.from_dict(p)), _ptr(phi))


def xseq(p: dict, Pf: float) -> float:
    return _L().rx_xseq(C.byref(RxParams.from_dict(p)), float(Pf))


def mg_step(st: RxState, mg: dict):
    """One physical step by FAS V-cycles to the change tolerance: (rc, cycles, change)."""
    it, ch = C.c_int(0), C.c_double(0.0)
    rc = _L().rx_mg_step(C.byref(st.cp), C.byref(RxMgParams.from_dict(mg)), C.byref(st.c), C.byref(it),
                         C.byref(ch))
    return rc, it.value, ch.value


def mg_cycles(st: RxState, mg: dict, ncycles: int):
    """Begin a step and run exactly ncycles V-cycles: (rc, change of the last)."""
    ch = C.c_double(0.0)
    rc = _L().rx_mg_cycles_n(C.byref(st.cp), C.byref(RxMgParams.from_dict(mg)), C.byref(st.c), ncycles,
                             C.byref(ch))
    return rc, ch.value


def mg_restrict(fine) -> np.ndarray:
    fine = np.ascontiguousarray(fine, dtype=float)
    nz, ny, nx = fine.shape
    out = np.zeros((nz // 2, ny // 2, nx // 2))
    _L().rx_mg_restrict(nx, ny, nz, _ptr(fine), _ptr(out))
    return out


def mg_prolong_add(coarse_e, fine) -> np.ndarray:
    """fine + the trilinear interpolation of the coarse correction (a new array)."""
    e = np.ascontiguousarray(coarse_e, dtype=float)
    out = np.array(fine, dtype=float, copy=True, order="C")
    nz, ny, nx = out.shape
    assert e.shape == (nz // 2, ny // 2, nx // 2)
    _L().rx_mg_prolong_add(nx, ny, nz, _ptr(e), _ptr(out))
    return out


def mg_equations(p: dict, u, old, f=None, omega: float = 6.0 / 7.0):
    """(gP, gphi, gX, den, R) of the step equations at the state u = (Pf, phi, Xs) with old-step
    fields old and FAS sources f (None: zero)."""
    cp = RxParams.from_dict(p)
    arr = [np.ascontiguousarray(a, dtype=float) for a in (*u, *old)]
    fs = [None] * 3 if f is None else [np.ascontiguousarray(a, dtype=float) for a in f]
    outs = [np.zeros_like(arr[0]) for _ in range(5)]
    fp = [None if a is None else _ptr(a) for a in fs]
    _L().rx_mg_equations(C.byref(cp), *[_ptr(a) for a in arr], *fp, float(omega), *[_ptr(a) for a in outs])
    return tuple(outs)
