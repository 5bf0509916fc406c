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
        for f in ("rx_begin_step", "rx_iteration", "rx_step", "rx_iterate_n"):
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
