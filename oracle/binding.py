"""ctypes binding and build step of the C oracle (test infrastructure only)."""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pt_oracle.c")
_HDR = os.path.join(_HERE, "pt_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

ORACLE_OK, ORACLE_EINVAL, ORACLE_ENOTCONV, ORACLE_ENAN = 0, -1, -2, -3


def lib_path() -> str:
    return _LIB


_RX_SRC = os.path.join(_HERE, "rx_oracle.c")
_RX_HDR = os.path.join(_HERE, "rx_oracle.h")
_MG_SRC = os.path.join(_HERE, "rx_mg_oracle.c")
_MG_HDR = os.path.join(_HERE, "rx_mg_oracle.h")


def build(force: bool = False) -> str:
    """Compile pt_oracle.c, rx_oracle.c and rx_mg_oracle.c into oracle/_build/liboracle.so (gcc,
    -O2, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(f) for f in (_SRC, _HDR, _RX_SRC, _RX_HDR, _MG_SRC, _MG_HDR))
    stale = not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-Wall",
               "-o", tmp, _SRC, _RX_SRC, _MG_SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class OracleParams(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("lx", C.c_double), ("ly", C.c_double), ("lz", C.c_double),
        ("phi0", C.c_double), ("k0", C.c_double), ("mu0", C.c_double), ("eta0", C.c_double),
        ("R_weak", C.c_double), ("n_pow", C.c_double), ("tau0", C.c_double),
        ("alpha", C.c_double), ("B", C.c_double), ("beta_d", C.c_double),
        ("beta_phi", C.c_double), ("G", C.c_double), ("rhof_g", C.c_double),
        ("rhos_g", C.c_double), ("powerlaw_on", C.c_int), ("compaction_on", C.c_int),
        ("dt", C.c_double), ("tol", C.c_double), ("max_iter", C.c_int), ("nup", C.c_int),
        ("damp_x", C.c_double), ("damp_y", C.c_double), ("damp_z", C.c_double),
        ("rho_i", C.c_double), ("beta_n", C.c_double), ("rel_mu", C.c_double),
        ("rel_eta", C.c_double), ("cfl_v", C.c_double), ("cfl_pf", C.c_double),
        ("dtpt_scale", C.c_double), ("xsi_w", C.c_double), ("mech_on", C.c_int),
        ("tau_bg", C.c_double),
    ]

    @classmethod
    def from_dict(cls, d: dict, mech_on: int = 1) -> "OracleParams":
        p = cls()
        for name, _ in cls._fields_:
            if name in ("mech_on", "tau_bg"):
                continue
            setattr(p, name, d[name])
        p.mech_on = int(d.get("mech_on", mech_on))
        p.tau_bg = float(d.get("tau_bg", 0.0))
        return p


class OracleRes(C.Structure):
    _fields_ = [("r_v", C.c_double), ("r_pt", C.c_double), ("r_pf", C.c_double),
                ("r_pic", C.c_double)]

    def as_dict(self) -> dict:
        return dict(r_v=self.r_v, r_pt=self.r_pt, r_pf=self.r_pf, r_pic=self.r_pic)


_STATE_FIELDS = ("Vx", "Vy", "Vz", "Pt", "Pf", "phi", "txx", "tyy", "tzz", "txy", "txz", "tyz",
                 "mu", "eta", "Rx", "Ry", "Rz", "Pto", "Pfo", "Lo",
                 "txxo", "tyyo", "tzzo", "txyo", "txzo", "tyzo")


class _CState(C.Structure):
    _fields_ = ([(n, C.POINTER(C.c_double)) for n in _STATE_FIELDS] +
                [("logk", C.POINTER(C.c_double)), ("dtS", C.c_double), ("dt_cum", C.c_double),
                 ("nsteps", C.c_int)])


_DP = C.POINTER(C.c_double)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = C.CDLL(_LIB)
            P, S, R = C.POINTER(OracleParams), C.POINTER(_CState), C.POINTER(OracleRes)
            for fn, args in [
                ("or_init_viscosities", [P, S]), ("or_begin_step", [P, S]),
                ("or_iteration", [P, S, C.c_int, R, C.POINTER(C.c_int)]),
                ("or_end_step", [P, S]), ("or_step", [P, S, C.POINTER(C.c_int), R]),
                ("or_iterate_n", [P, S, C.c_int, C.c_int, R]),
                ("or_system_residual", [P, S] + [_DP] * 8),
            ]:
                f = getattr(lib, fn)
                f.argtypes = args
                f.restype = C.c_int
            for fn, n in [("or_coefficients", 5), ("or_darcy", 7), ("or_divergence", 12),
                          ("or_stress", 19), ("or_momentum", 12), ("or_advection", 6),
                          ("or_tau_II", 8)]:
                f = getattr(lib, fn)
                f.argtypes = [P] + [_DP] * (n - 1)
                f.restype = None
            lib.or_stress.argtypes = [P, C.c_double] + [_DP] * 18
            lib.or_max_threads.argtypes = []
            lib.or_max_threads.restype = C.c_int
            _lib = lib
    return _lib


def max_threads() -> int:
    """OpenMP threads the oracle uses."""
    return int(_load().or_max_threads())


def _shapes(p: dict) -> dict:
    nx, ny, nz = p["nx"], p["ny"], p["nz"]
    c = (nz, ny, nx)
    return dict(Vx=(nz, ny, nx + 1), Vy=(nz, ny + 1, nx), Vz=(nz + 1, ny, nx),
                Rx=(nz, ny, nx + 1), Ry=(nz, ny + 1, nx), Rz=(nz + 1, ny, nx),
                txy=(nz, ny + 1, nx + 1), txz=(nz + 1, ny, nx + 1), tyz=(nz + 1, ny + 1, nx),
                txyo=(nz, ny + 1, nx + 1), txzo=(nz + 1, ny, nx + 1), tyzo=(nz + 1, ny + 1, nx),
                **{n: c for n in ("Pt", "Pf", "phi", "txx", "tyy", "tzz", "mu", "eta", "Pto",
                                  "Pfo", "Lo", "txxo", "tyyo", "tzzo")})


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_DP)


class State(dict):
    """All oracle state arrays (numpy float64, natural staggered shapes) plus the params and
    the stress sub-stepping scalars (dtS, dt_cum, nsteps)."""

    def __init__(self, params: dict, arrays: dict, logk, dtS=0.0, dt_cum=0.0, nsteps=0):
        super().__init__(arrays)
        self.params = dict(params)
        self.logk = logk
        self.dtS, self.dt_cum, self.nsteps = dtS, dt_cum, nsteps

    def cstruct(self) -> _CState:
        cs = _CState()
        for n in _STATE_FIELDS:
            setattr(cs, n, _ptr(self[n]))
        cs.logk = _ptr(self.logk) if self.logk is not None else None
        cs.dtS, cs.dt_cum, cs.nsteps = self.dtS, self.dt_cum, self.nsteps
        return cs

    def pull(self, cs: _CState) -> None:
        self.dtS, self.dt_cum, self.nsteps = cs.dtS, cs.dt_cum, cs.nsteps

    def cparams(self, **over) -> OracleParams:
        d = dict(self.params)
        d.update(over)
        return OracleParams.from_dict(d)

    def copy(self) -> "State":
        return State(self.params, {k: v.copy() for k, v in self.items()},
                     None if self.logk is None else self.logk.copy(),
                     self.dtS, self.dt_cum, self.nsteps)


def make_state(params: dict, phi: np.ndarray, logk: np.ndarray | None = None,
               fields: dict | None = None, init_visc: bool = True) -> State:
    """Zero state (V, P, tau, R = 0) with the given porosity; `fields` overrides entries."""
    sh = _shapes(params)
    arrays = {n: np.zeros(s, dtype=np.float64) for n, s in sh.items()}
    arrays["phi"][...] = phi
    for k, v in (fields or {}).items():
        arrays[k][...] = v
    lk = None if logk is None else np.ascontiguousarray(logk, dtype=np.float64)
    st = State(params, arrays, lk)
    if init_visc:
        init_viscosities(st)
    return st


def _call(fn, st: State, *args, **over):
    lib = _load()
    p = st.cparams(**over)
    cs = st.cstruct()
    rc = getattr(lib, fn)(C.byref(p), C.byref(cs), *args)
    st.pull(cs)
    return rc


def init_viscosities(st: State, **over) -> int:
    return _call("or_init_viscosities", st, **over)


def begin_step(st: State, **over) -> int:
    return _call("or_begin_step", st, **over)


def end_step(st: State, **over) -> int:
    return _call("or_end_step", st, **over)


def iteration(st: State, it: int, **over):
    """One PT iteration number `it` (1-based). Returns (rc, res dict or None)."""
    res, chk = OracleRes(), C.c_int(0)
    rc = _call("or_iteration", st, it, C.byref(res), C.byref(chk), **over)
    return rc, (res.as_dict() if chk.value else None)


def iterate_n(st: State, it0: int, niter: int, **over):
    res = OracleRes()
    rc = _call("or_iterate_n", st, it0, niter, C.byref(res), **over)
    return rc, res.as_dict()


def step(st: State, **over):
    """One physical time step to tol (or max_iter). Returns (rc, iters, res dict)."""
    res, iters = OracleRes(), C.c_int(0)
    rc = _call("or_step", st, C.byref(iters), C.byref(res), **over)
    return rc, iters.value, res.as_dict()


def system_residual(st: State, **over) -> dict:
    sh = _shapes(st.params)
    out = dict(Vx=np.zeros(sh["Vx"]), Vy=np.zeros(sh["Vy"]), Vz=np.zeros(sh["Vz"]),
               pt=np.zeros(sh["Pt"]), pf=np.zeros(sh["Pt"]), L=np.zeros(sh["Pt"]),
               mu=np.zeros(sh["Pt"]), eta=np.zeros(sh["Pt"]))
    rc = _call("or_system_residual", st, *[_ptr(out[k]) for k in
                                           ("Vx", "Vy", "Vz", "pt", "pf", "L", "mu", "eta")], **over)
    if rc != 0:
        raise RuntimeError(f"or_system_residual rc={rc}")
    return out


# ---- building blocks on raw arrays (unit pins) ----
def _p(params: dict, **over) -> OracleParams:
    d = dict(params)
    d.update(over)
    return OracleParams.from_dict(d)


def coefficients(params, phi, logk=None):
    sh = _shapes(params)
    perm, rog = np.zeros(sh["Pt"]), np.zeros(sh["Pt"])
    _load().or_coefficients(C.byref(_p(params)), _ptr(phi), _ptr(logk) if logk is not None else None,
                            _ptr(perm), _ptr(rog))
    return perm, rog


def darcy(params, Pf, perm):
    sh = _shapes(params)
    qx, qy, qz, dq = np.zeros(sh["Vx"]), np.zeros(sh["Vy"]), np.zeros(sh["Vz"]), np.zeros(sh["Pt"])
    _load().or_darcy(C.byref(_p(params)), _ptr(Pf), _ptr(perm), _ptr(qx), _ptr(qy), _ptr(qz), _ptr(dq))
    return qx, qy, qz, dq


def divergence(params, Vx, Vy, Vz, Pt, Pf, Pto, Pfo, phi, eta):
    sh = _shapes(params)
    dv, dvn = np.zeros(sh["Pt"]), np.zeros(sh["Pt"])
    _load().or_divergence(C.byref(_p(params)), *[_ptr(a) for a in (Vx, Vy, Vz, Pt, Pf, Pto, Pfo, phi, eta)],
                          _ptr(dv), _ptr(dvn))
    return dv, dvn


def stress(params, dtS, Vx, Vy, Vz, divV, divVn, mu, told):
    """told = (txxo, tyyo, tzzo, txyo, txzo, tyzo); returns the six new stresses."""
    sh = _shapes(params)
    out = [np.zeros(sh[k]) for k in ("Pt", "Pt", "Pt", "txy", "txz", "tyz")]
    _load().or_stress(C.byref(_p(params)), C.c_double(dtS),
                      *[_ptr(a) for a in (Vx, Vy, Vz, divV, divVn, mu)],
                      *[_ptr(a) for a in told], *[_ptr(a) for a in out])
    return tuple(out)


def momentum(params, tau, Pt, rog):
    sh = _shapes(params)
    F = [np.zeros(sh[k]) for k in ("Vx", "Vy", "Vz")]
    _load().or_momentum(C.byref(_p(params)), *[_ptr(a) for a in tau], _ptr(Pt), _ptr(rog),
                        *[_ptr(a) for a in F])
    return tuple(F)


def advection(params, Vx, Vy, Vz, phi):
    sh = _shapes(params)
    adv = np.zeros(sh["Pt"])
    _load().or_advection(C.byref(_p(params)), _ptr(Vx), _ptr(Vy), _ptr(Vz), _ptr(phi), _ptr(adv))
    return adv


def tau_II(params, tau):
    sh = _shapes(params)
    t = np.zeros(sh["Pt"])
    _load().or_tau_II(C.byref(_p(params)), *[_ptr(a) for a in tau], _ptr(t))
    return t
