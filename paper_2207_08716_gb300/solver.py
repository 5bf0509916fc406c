"""Thin Python front end of the C ABI: device memory and the stream come from PyTorch, every
step of the solve runs in the CUDA library (argument marshalling only here).

Arrays at this level are in the natural staggered shapes (see ``pt_inputs.field_shapes``):
numpy or torch, ``(nz_s, ny_s, nx_s)`` with x fastest. They are copied into the library's
padded box layout on the device (``box[:nz_s, :ny_s, :nx_s] = a``).
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import native as N

_SHAPE_OF = {"Vx": (0, 0, 1), "Vy": (0, 1, 0), "Vz": (1, 0, 0), "txy": (0, 1, 1),
             "txz": (1, 0, 1), "tyz": (1, 1, 0)}


def natural_shape(name: str, nx: int, ny: int, nz: int) -> tuple:
    dz, dy, dx = _SHAPE_OF.get(name, (0, 0, 0))
    return (nz + dz, ny + dy, nx + dx)


class PTError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {N.strerror(code)} ({code})")
        self.code = code


class PTSolver:
    """One solver context over device fields owned by this object (torch tensors).

    params: dict with the keys of ``pt_inputs.PARAM_KEYS``; phi: initial porosity at cell
    centres; logk: optional log-permeability prefactor field; fields: optional initial values of
    any other field (natural shapes); keep_visc: keep given mu / eta instead of initialising
    them from phi (Eq. 26).
    """

    def __init__(self, params: dict, phi, logk=None, fields: dict | None = None,
                 device: str | torch.device = "cuda", stream: torch.cuda.Stream | None = None,
                 keep_visc: bool = False):
        self.lib = N.load()
        self.params = dict(params)
        self.device = torch.device(device)
        if self.device.type != "cuda":
            raise ValueError("PTSolver runs on a CUDA device only")
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        p = self.params
        self.nx, self.ny, self.nz = p["nx"], p["ny"], p["nz"]
        self._grid = N.grid_from(p)
        self._phys = N.phys_from(p)
        self._num = N.num_from(p)
        n = self.lib.pt_field_elems(C.byref(self._grid))
        if n == 0:
            raise PTError(N.PT_EINVAL, "grid")
        self.px = self.lib.pt_pitch_x(C.byref(self._grid))
        self.box_shape = (self.nz + 1, self.ny + 1, self.px)
        with torch.cuda.device(self.device):
            self.f = {name: torch.zeros(self.box_shape, dtype=torch.float64, device=self.device)
                      for name in N.FIELD_NAMES}
            self.logk = None
            if logk is not None:
                self.logk = torch.zeros(self.box_shape, dtype=torch.float64, device=self.device)
                self._put(self.logk, "centre", logk)
            self._put(self.f["phi"], "phi", phi)
            for k, v in (fields or {}).items():
                self._put(self.f[k], k, v)
            ws = self.lib.pt_workspace_size(C.byref(self._grid), C.byref(self._num))
            self.workspace = torch.empty(ws, dtype=torch.uint8, device=self.device)
        fs = N.Fields(*[self.f[k].data_ptr() for k in N.FIELD_NAMES],
                      self.logk.data_ptr() if self.logk is not None else None)
        ctx = C.c_void_p()
        torch.cuda.synchronize(self.device)
        rc = self.lib.pt_init(C.byref(ctx), C.byref(self._grid), C.byref(self._phys),
                              C.byref(self._num), C.byref(fs), self.workspace.data_ptr(), ws,
                              self.stream.cuda_stream, int(keep_visc))
        if rc != N.PT_OK:
            raise PTError(rc, "pt_init")
        self.ctx = ctx

    # -------------------------------------------------------------- layout marshalling
    def _put(self, box: torch.Tensor, name: str, a) -> None:
        t = torch.as_tensor(a, dtype=torch.float64).to(self.device)
        sh = natural_shape(name, self.nx, self.ny, self.nz)
        if tuple(t.shape) != sh:
            raise ValueError(f"{name}: expected shape {sh}, got {tuple(t.shape)}")
        box[: sh[0], : sh[1], : sh[2]].copy_(t)

    def get(self, name: str) -> np.ndarray:
        """Current field in its natural staggered shape, as a numpy array."""
        torch.cuda.synchronize(self.device)
        sh = natural_shape(name, self.nx, self.ny, self.nz)
        return self.f[name][: sh[0], : sh[1], : sh[2]].cpu().numpy().copy()

    def set(self, name: str, a) -> None:
        self._put(self.f[name], name, a)
        torch.cuda.synchronize(self.device)

    # ------------------------------------------------------------------------ solve
    def _check(self, rc: int, what: str, allow=(N.PT_OK,)) -> None:
        if rc not in allow:
            raise PTError(rc, what)

    def step(self, raise_on_notconv: bool = False) -> dict:
        rep = N.Report()
        rc = self.lib.pt_step(self.ctx, C.byref(rep))
        allow = (N.PT_OK,) if raise_on_notconv else (N.PT_OK, N.PT_ENOTCONV)
        self._check(rc, "pt_step", allow)
        return rep.as_dict()

    def step_begin(self) -> None:
        self._check(self.lib.pt_step_begin(self.ctx), "pt_step_begin")

    def iterate(self, it0: int, niter: int, report: bool = True) -> dict | None:
        rep = N.Report()
        rc = self.lib.pt_iterate(self.ctx, it0, niter, C.byref(rep) if report else None)
        self._check(rc, "pt_iterate")
        return rep.as_dict() if report else None

    def step_end(self) -> None:
        self._check(self.lib.pt_step_end(self.ctx), "pt_step_end")

    def residual(self) -> dict:
        rep = N.Report()
        self._check(self.lib.pt_residual(self.ctx, C.byref(rep)), "pt_residual")
        return rep.as_dict()

    # ------------------------------------------------------------------- adjoint
    def adjoint_forward(self, nsteps: int, ckpt_every: int | None = None) -> list:
        """Run `nsteps` steps from the current (fresh) state keeping adjoint checkpoints."""
        every = int(ckpt_every or nsteps)
        need = self.lib.pt_adjoint_workspace_size(C.byref(self._grid), nsteps, every)
        if need == 0:
            raise PTError(N.PT_EINVAL, "pt_adjoint_workspace_size")
        with torch.cuda.device(self.device):
            self.adj_workspace = torch.empty(need, dtype=torch.uint8, device=self.device)
        reps = (N.Report * nsteps)()
        rc = self.lib.pt_adjoint_forward(self.ctx, nsteps, every, self.adj_workspace.data_ptr(), need, reps)
        self._check(rc, "pt_adjoint_forward")
        return [r.as_dict() for r in reps]

    def adjoint(self, dJ_dphi) -> tuple:
        """dJ/dlogk (cell-centred, natural shape, torch on the device) for dJ/dphi^N."""
        g = torch.zeros(self.box_shape, dtype=torch.float64, device=self.device)
        self._put(g, "phi", dJ_dphi)
        out = torch.empty_like(g)
        rep = N.Report()
        torch.cuda.current_stream(self.device).synchronize()
        self._check(self.lib.pt_adjoint(self.ctx, g.data_ptr(), out.data_ptr(), C.byref(rep)), "pt_adjoint")
        return out[: self.nz, : self.ny, : self.nx].clone(), rep.as_dict()

    def adjoint_apply(self, lam: dict) -> dict:
        """J_F(u)^T lam at the current fields (pt_adjoint_apply): lam and the result map
        Vx, Vy, Vz, Pt, Pf, phi and, with the power law on, mu (natural shapes; wall-normal
        faces of lam must be zero)."""
        keys = ("Vx", "Vy", "Vz", "Pt", "Pf", "phi") + (("mu",) if self.params.get("powerlaw_on") else ())
        need = self.lib.pt_adjoint_workspace_size(C.byref(self._grid), 0, 1)
        with torch.cuda.device(self.device):
            ws = torch.empty(need, dtype=torch.uint8, device=self.device)
            lb = {k: torch.zeros(self.box_shape, dtype=torch.float64, device=self.device) for k in keys}
            ob = {k: torch.empty(self.box_shape, dtype=torch.float64, device=self.device) for k in keys}
        for k in keys:
            self._put(lb[k], k, lam[k])
        torch.cuda.current_stream(self.device).synchronize()
        lv = N.AdjVec(*[lb[k].data_ptr() for k in keys] + [None] * (7 - len(keys)))
        ov = N.AdjVec(*[ob[k].data_ptr() for k in keys] + [None] * (7 - len(keys)))
        self._check(self.lib.pt_adjoint_apply(self.ctx, C.byref(lv), C.byref(ov), ws.data_ptr(), need),
                    "pt_adjoint_apply")
        out = {}
        for k in keys:
            sh = natural_shape(k, self.nx, self.ny, self.nz)
            out[k] = ob[k][: sh[0], : sh[1], : sh[2]].cpu().numpy().copy()
        return out

    # ------------------------------------------------------------- measurement aids
    def profile_begin(self) -> None:
        self._check(self.lib.pt_profile_begin(self.ctx), "pt_profile_begin")

    def profile_end(self) -> dict:
        """{kernel name: (launches, total ms)} measured with CUDA events on the solver stream."""
        out = (N.KernelTime * 32)()
        n = C.c_int32(0)
        self._check(self.lib.pt_profile_end(self.ctx, out, 32, C.byref(n)), "pt_profile_end")
        return {out[i].name.decode(): (int(out[i].launches), float(out[i].total_ms)) for i in range(n.value)}

    def launch_count(self) -> int:
        return int(self.lib.pt_launch_count(self.ctx))

    # ------------------------------------------------ host-resident state (end to end)
    def host_mirror(self) -> dict:
        """Pinned host tensors in the padded box layout, one per field."""
        return {k: torch.empty(self.box_shape, dtype=torch.float64, pin_memory=True)
                for k in N.FIELD_NAMES}

    def upload(self, host: dict) -> int:
        """Copy host (pinned, box layout) fields to the device on the solver stream; bytes."""
        nbytes = 0
        with torch.cuda.stream(self.stream):
            for k, h in host.items():
                self.f[k].copy_(h, non_blocking=True)
                nbytes += h.numel() * h.element_size()
        return nbytes

    def download(self, host: dict) -> int:
        nbytes = 0
        with torch.cuda.stream(self.stream):
            for k, h in host.items():
                h.copy_(self.f[k], non_blocking=True)
                nbytes += h.numel() * h.element_size()
        return nbytes

    def close(self) -> None:
        if getattr(self, "ctx", None):
            self.lib.pt_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class PTBatch:
    """An ensemble of independent instances advanced together (pt_batch_* of the C ABI).

    members: list of (params, phi) or (params, phi, logk); every instance uses the same nup and
    the same precision: PT_FP64 (the FP64-lean form) or PT_FP32 (the FP32 + FP64
    defect-correction form), either way in the library's persistent batched engine.
    """

    def __init__(self, members, device="cuda", stream=None, precision: int = N.PT_FP64):
        self.lib = N.load()
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.n = len(members)
        self.params = [dict(m[0]) for m in members]
        G, P, U, F = (N.Grid * self.n)(), (N.Phys * self.n)(), (N.Num * self.n)(), (N.Fields * self.n)()
        self.f, self.logk, self.shape = [], [], []
        with torch.cuda.device(self.device):
            for m, mem in enumerate(members):
                p = dict(mem[0])
                p["precision"] = precision
                G[m], P[m], U[m] = N.grid_from(p), N.phys_from(p), N.num_from(p)
                px = self.lib.pt_pitch_x(C.byref(G[m]))
                box = (p["nz"] + 1, p["ny"] + 1, px)
                f = {k: torch.zeros(box, dtype=torch.float64, device=self.device) for k in N.FIELD_NAMES}
                sh = natural_shape("phi", p["nx"], p["ny"], p["nz"])
                f["phi"][: sh[0], : sh[1], : sh[2]].copy_(torch.as_tensor(mem[1], dtype=torch.float64))
                lk = None
                if len(mem) > 2 and mem[2] is not None:
                    lk = torch.zeros(box, dtype=torch.float64, device=self.device)
                    lk[: sh[0], : sh[1], : sh[2]].copy_(torch.as_tensor(mem[2], dtype=torch.float64))
                self.f.append(f)
                self.logk.append(lk)
                self.shape.append((p["nx"], p["ny"], p["nz"]))
                F[m] = N.Fields(*[f[k].data_ptr() for k in N.FIELD_NAMES], lk.data_ptr() if lk is not None else None)
            ws = self.lib.pt_batch_workspace_size(self.n, G, U)
            if ws == 0:
                raise PTError(N.PT_EINVAL, "pt_batch_workspace_size")
            self.workspace = torch.empty(ws, dtype=torch.uint8, device=self.device)
        self._keep = (G, P, U, F)
        torch.cuda.synchronize(self.device)
        h = C.c_void_p()
        rc = self.lib.pt_batch_init(C.byref(h), self.n, G, P, U, F, self.workspace.data_ptr(), ws,
                                    self.stream.cuda_stream)
        if rc != N.PT_OK:
            raise PTError(rc, "pt_batch_init")
        self.h = h

    def step(self):
        """One physical step of every instance: (list of report dicts, time-to-converge ms)."""
        reps = (N.Report * self.n)()
        ttc = (C.c_double * self.n)()
        rc = self.lib.pt_batch_step(self.h, reps, ttc)
        if rc not in (N.PT_OK, N.PT_ENOTCONV):
            raise PTError(rc, "pt_batch_step")
        return [r.as_dict() for r in reps], [float(t) for t in ttc]

    def config(self) -> tuple:
        bx, by, ipg = C.c_int32(), C.c_int32(), C.c_int32()
        self.lib.pt_batch_config(self.h, C.byref(bx), C.byref(by), C.byref(ipg))
        return bx.value, by.value, ipg.value

    def config_fp32(self) -> tuple:
        """FP32 ensembles: (correction tile depth, CTAs per SM of the correction kernel, member groups)."""
        tz, mb, gr = C.c_int32(), C.c_int32(), C.c_int32()
        rc = self.lib.pt_batch_config_fp32(self.h, C.byref(tz), C.byref(mb), C.byref(gr))
        if rc != N.PT_OK:
            raise PTError(rc, "pt_batch_config_fp32")
        return tz.value, mb.value, gr.value

    def get(self, m: int, name: str) -> np.ndarray:
        torch.cuda.synchronize(self.device)
        sh = natural_shape(name, *self.shape[m])
        return self.f[m][name][: sh[0], : sh[1], : sh[2]].cpu().numpy().copy()

    def close(self):
        if getattr(self, "h", None):
            self.lib.pt_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class PTDomains:
    """The grid split into parts x parts x parts sub-domains with halo exchange (pt_dd_* of the
    C ABI): same arguments as PTSolver plus `parts` = (px, py, pz); FP64-lean form."""

    def __init__(self, params: dict, phi, parts=(2, 2, 2), logk=None, device="cuda", stream=None):
        self.lib = N.load()
        p = dict(params)
        p["precision"] = N.PT_FP64
        self.params = p
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.nx, self.ny, self.nz = p["nx"], p["ny"], p["nz"]
        self._grid, self._phys, self._num = N.grid_from(p), N.phys_from(p), N.num_from(p)
        self._parts = (C.c_int32 * 3)(*[int(x) for x in parts])
        px = self.lib.pt_pitch_x(C.byref(self._grid))
        if px == 0:
            raise PTError(N.PT_EINVAL, "grid")
        self.box_shape = (self.nz + 1, self.ny + 1, px)
        ws = self.lib.pt_dd_workspace_size(C.byref(self._grid), C.byref(self._num), self._parts)
        if ws == 0:
            raise PTError(N.PT_EINVAL, "pt_dd_workspace_size")
        with torch.cuda.device(self.device):
            self.f = {k: torch.zeros(self.box_shape, dtype=torch.float64, device=self.device) for k in N.FIELD_NAMES}
            self.logk = None
            if logk is not None:
                self.logk = torch.zeros(self.box_shape, dtype=torch.float64, device=self.device)
                self.logk[: self.nz, : self.ny, : self.nx].copy_(torch.as_tensor(logk, dtype=torch.float64))
            self.f["phi"][: self.nz, : self.ny, : self.nx].copy_(torch.as_tensor(phi, dtype=torch.float64))
            self.workspace = torch.empty(ws, dtype=torch.uint8, device=self.device)
        self._fields = N.Fields(*[self.f[k].data_ptr() for k in N.FIELD_NAMES],
                                self.logk.data_ptr() if self.logk is not None else None)
        torch.cuda.synchronize(self.device)
        h = C.c_void_p()
        rc = self.lib.pt_dd_init(C.byref(h), C.byref(self._grid), C.byref(self._phys), C.byref(self._num),
                                 C.byref(self._fields), self._parts, self.workspace.data_ptr(), ws,
                                 self.stream.cuda_stream)
        if rc != N.PT_OK:
            raise PTError(rc, "pt_dd_init")
        self.h = h

    def step(self) -> dict:
        rep = N.Report()
        rc = self.lib.pt_dd_step(self.h, C.byref(rep))
        if rc not in (N.PT_OK, N.PT_ENOTCONV):
            raise PTError(rc, "pt_dd_step")
        return rep.as_dict()

    def gather(self) -> None:
        rc = self.lib.pt_dd_gather(self.h)
        if rc != N.PT_OK:
            raise PTError(rc, "pt_dd_gather")

    def get(self, name: str) -> np.ndarray:
        """Field in its natural staggered shape (call gather() first)."""
        torch.cuda.synchronize(self.device)
        sh = natural_shape(name, self.nx, self.ny, self.nz)
        return self.f[name][: sh[0], : sh[1], : sh[2]].cpu().numpy().copy()

    def config(self) -> tuple:
        n, bx, by, ipg = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
        self.lib.pt_dd_config(self.h, C.byref(n), C.byref(bx), C.byref(by), C.byref(ipg))
        return n.value, bx.value, by.value, ipg.value

    def close(self):
        if getattr(self, "h", None):
            self.lib.pt_dd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class RXSolver:
    """Reactive porosity-wave solver (rx_* of the C ABI; thesis Art. 3, Eqs. 8-10).

    params: the keys of ``pt_inputs.rx_params`` plus optional ``precision`` (PT_FP64 default,
    PT_FP32); Pf, phi, Xs: initial cell fields (nz, ny, nx); mg: multigrid settings (keys of
    rx_mg: levels, nu_pre, nu_post, nu_coarse, max_cycles, omega) to enable ``mg_step`` and
    ``mg_cycles`` (FAS V-cycles) besides the plain PT ``step`` and ``iterate``."""

    _PHYS = ("phi0", "k0", "eta", "rhof", "rhos", "g", "beta_d", "beta_s", "beta_f", "beta_x", "dX",
             "xs_max", "tau")

    _MG = ("levels", "nu_pre", "nu_post", "nu_coarse", "max_cycles", "omega")

    def __init__(self, params: dict, Pf, phi, Xs, device="cuda", stream=None, mg: dict | None = None):
        self.lib = N.load()
        p = dict(params)
        self.params = p
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.nx, self.ny, self.nz = p["nx"], p["ny"], p["nz"]
        self._grid = N.Grid(p["nx"], p["ny"], p["nz"], p["lx"], p["ly"], p["lz"])
        self._phys = N.RxPhys(*[float(p[k]) for k in self._PHYS])
        self._num = N.RxNum(p["dt"], p["tol"], p["cfl_div"], p["pf_scale"], int(p["max_iter"]), int(p["nup"]),
                            int(p.get("precision", N.PT_FP64)))
        px = self.lib.pt_pitch_x(C.byref(self._grid))
        if px == 0:
            raise PTError(N.PT_EINVAL, "grid")
        self.box_shape = (self.nz + 1, self.ny + 1, px)
        self._mg = None
        if mg is not None:
            self._mg = N.RxMg(*[int(mg[k]) for k in self._MG[:-1]], float(mg["omega"]))
            ws = self.lib.rx_mg_workspace_size(C.byref(self._grid), C.byref(self._num), C.byref(self._mg))
        else:
            ws = self.lib.rx_workspace_size(C.byref(self._grid), C.byref(self._num))
        if ws == 0:
            raise PTError(N.PT_EINVAL, "rx_workspace_size")
        with torch.cuda.device(self.device):
            self.f = {k: torch.zeros(self.box_shape, dtype=torch.float64, device=self.device)
                      for k in ("Pf", "phi", "Xs", "R")}
            for k, v in (("Pf", Pf), ("phi", phi), ("Xs", Xs)):
                self.f[k][: self.nz, : self.ny, : self.nx].copy_(torch.as_tensor(v, dtype=torch.float64))
            self.workspace = torch.empty(ws, dtype=torch.uint8, device=self.device)
        fs = N.RxFields(*[self.f[k].data_ptr() for k in ("Pf", "phi", "Xs", "R")])
        torch.cuda.synchronize(self.device)
        h = C.c_void_p()
        if self._mg is not None:
            rc = self.lib.rx_mg_init(C.byref(h), C.byref(self._grid), C.byref(self._phys), C.byref(self._num),
                                     C.byref(self._mg), C.byref(fs), self.workspace.data_ptr(), ws,
                                     self.stream.cuda_stream)
        else:
            rc = self.lib.rx_init(C.byref(h), C.byref(self._grid), C.byref(self._phys), C.byref(self._num),
                                  C.byref(fs), self.workspace.data_ptr(), ws, self.stream.cuda_stream)
        if rc != N.PT_OK:
            raise PTError(rc, "rx_init")
        self.h = h

    def step(self, raise_on_notconv: bool = False) -> dict:
        rep = N.Report()
        rc = self.lib.rx_step(self.h, C.byref(rep))
        if rc not in ((N.PT_OK,) if raise_on_notconv else (N.PT_OK, N.PT_ENOTCONV)):
            raise PTError(rc, "rx_step")
        return rep.as_dict()

    def iterate(self, niter: int) -> dict:
        rep = N.Report()
        rc = self.lib.rx_iterate(self.h, niter, C.byref(rep))
        if rc != N.PT_OK:
            raise PTError(rc, "rx_iterate")
        return rep.as_dict()

    def mg_step(self, raise_on_notconv: bool = False) -> dict:
        """One physical step by FAS V-cycles to the tolerance (report iters = cycles)."""
        rep = N.Report()
        rc = self.lib.rx_mg_step(self.h, C.byref(rep))
        if rc not in ((N.PT_OK,) if raise_on_notconv else (N.PT_OK, N.PT_ENOTCONV)):
            raise PTError(rc, "rx_mg_step")
        return rep.as_dict()

    def mg_cycles(self, ncycles: int) -> dict:
        rep = N.Report()
        rc = self.lib.rx_mg_cycles(self.h, ncycles, C.byref(rep))
        if rc != N.PT_OK:
            raise PTError(rc, "rx_mg_cycles")
        return rep.as_dict()

    def get(self, name: str) -> np.ndarray:
        torch.cuda.synchronize(self.device)
        return self.f[name][: self.nz, : self.ny, : self.nx].cpu().numpy().copy()

    def launch_count(self) -> int:
        return int(self.lib.rx_launch_count(self.h))

    def close(self):
        if getattr(self, "h", None):
            self.lib.rx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
