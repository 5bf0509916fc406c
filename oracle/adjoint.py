"""CPU adjoint of the porosity-wave solver — TEST INFRASTRUCTURE ONLY (oracle side).

Differentiates the converged implicit time step (thesis Art. 1, Eqs. 17-27 as discretised by
pt_oracle.c), not the PT iterations: each step solves F(u^{n+1}; u^n, theta) = 0 for
u = (V, Pt, Pf, phi); for J = sum (phi^N - phi_target)^2 the adjoint recursion is
    J_F(u^{n+1})^T lambda^{n+1} = g^{n+1},
    g^N = dJ/du^N,   g^n = -(dF^{n+1}/du^n)^T lambda^{n+1}  (n < N),
    dJ/dtheta = -sum_n (dF^{n}/dtheta)^T lambda^{n}.
Scope: no weakening switch (R = 1; Eq. 25 is a step function), beta_n = 0, zero old-step
stresses over the window (no stress sub-step refresh). With the power law off the converged
Picard state is mu = mu0, eta = eta0 mu0 / phi and u = (V on interior faces, Pt, Pf, phi) is
the whole unknown. With the power law on (Eq. 24) mu joins the unknowns with the Picard
fixed-point row F_mu = log mu - log mu*(tau_II) (the Maxwell stresses of Eq. 21 with moduli
2 mu / (1 + xi), xi = mu / (G dtS), edge values from the mean of the four centres' mu),
eta = eta0 mu / phi (Eq. 26 at its fixed point), and the step's stress sub-step
dtS = max(mu_prev) / (G xsi_w) makes each step depend on the previous step's mu as well.

The residual is written with plain PyTorch CPU ops in FP64 (one expression per term of the
oracle's discretisation), so autograd gives exact Jacobian products; on tiny grids the adjoint
systems are solved with dense LU. It is pinned to the C oracle's own residual in the tests and
the gradient to finite differences of the C oracle's converged forward runs.
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding as B

_T = torch.float64


def _geom(p):
    return p["lx"] / p["nx"], p["ly"] / p["ny"], p["lz"] / p["nz"]


def residual(p: dict, u: dict, old: dict, theta: torch.Tensor) -> dict:
    """F(u; old, theta) of one implicit step (scope of the module docstring).

    u: Vx (nz, ny, nx+1), Vy (nz, ny+1, nx), Vz (nz+1, ny, nx) — boundary faces included and
    kept at zero —, Pt, Pf, phi (nz, ny, nx); old: Pto, Pfo, Lo (centres); theta: log-k field.
    Returns the residual fields: Fx/Fy/Fz on interior faces, Fpt, Fpf, FL at centres.
    """
    dx, dy, dz = _geom(p)
    Vx, Vy, Vz, Pt, Pf, phi = (u[k] for k in ("Vx", "Vy", "Vz", "Pt", "Pf", "phi"))
    Pto, Pfo, Lo = old["Pto"], old["Pfo"], old["Lo"]
    bd, al, B_, bphi, dt = p["beta_d"], p["alpha"], p["B"], p["beta_phi"], p["dt"]
    mu0, eta0, G = p["mu0"], p["eta0"], p["G"]
    pl = bool(p.get("powerlaw_on", 0))
    rho_bg = p["phi0"] * p["rhof_g"] + (1 - p["phi0"]) * p["rhos_g"]
    if pl:
        mu = u["mu"]
        Gdt = torch.max(old["mu_o"]) / p["xsi_w"]                   # G dtS, dtS = max mu_prev / (G xsi_w)
        eta = eta0 * mu / phi                                       # Eq. 26, R = 1
    else:
        eta = eta0 * mu0 / phi                                      # Eq. 26, R = 1
    cc = 1.0 / (eta * (1.0 - phi))                                  # compaction coefficient
    # div V and the total-pressure residual (Eq. 17)
    gx = (Vx[:, :, 1:] - Vx[:, :, :-1]) / dx
    gy = (Vy[:, 1:, :] - Vy[:, :-1, :]) / dy
    gz = (Vz[1:, :, :] - Vz[:-1, :, :]) / dz
    divV = gx + gy + gz
    Fpt = divV + bd * ((Pt - Pto) - al * (Pf - Pfo)) / dt + (Pt - Pf) * cc
    # Darcy flux with k = k0 e^theta (phi/phi0)^3 (Eqs. 20, 23), zero normal flux on the walls
    k = p["k0"] * torch.exp(theta) * (phi / p["phi0"]) ** 3
    qx = -0.5 * (k[:, :, 1:] + k[:, :, :-1]) * (Pf[:, :, 1:] - Pf[:, :, :-1]) / dx
    qy = -0.5 * (k[:, 1:, :] + k[:, :-1, :]) * (Pf[:, 1:, :] - Pf[:, :-1, :]) / dy
    qz = -0.5 * (k[1:] + k[:-1]) * ((Pf[1:] - Pf[:-1]) / dz + (p["rhof_g"] - rho_bg))
    z = lambda t, dim: torch.zeros_like(t.narrow(dim, 0, 1))
    qx = torch.cat([z(qx, 2), qx, z(qx, 2)], 2)
    qy = torch.cat([z(qy, 1), qy, z(qy, 1)], 1)
    qz = torch.cat([z(qz, 0), qz, z(qz, 0)], 0)
    divq = (qx[:, :, 1:] - qx[:, :, :-1]) / dx + (qy[:, 1:, :] - qy[:, :-1, :]) / dy + (qz[1:] - qz[:-1]) / dz
    Fpf = divq + bd * al * ((Pf - Pfo) / B_ - (Pt - Pto)) / dt + (Pf - Pt) * cc
    # Maxwell stresses with tau_o = 0 (Eq. 21): 2 mu / (1 + xi) times the deviatoric strain rate,
    # xi = mu / (G dtS); the power law off: mu = mu0 and dtS = mu0 / (G xsi_w), so xi = xsi_w
    exy = 0.5 * ((Vx[:, 1:, 1:-1] - Vx[:, :-1, 1:-1]) / dy + (Vy[:, 1:-1, 1:] - Vy[:, 1:-1, :-1]) / dx)
    exz = 0.5 * ((Vx[1:, :, 1:-1] - Vx[:-1, :, 1:-1]) / dz + (Vz[1:-1, :, 1:] - Vz[1:-1, :, :-1]) / dx)
    eyz = 0.5 * ((Vy[1:, 1:-1, :] - Vy[:-1, 1:-1, :]) / dz + (Vz[1:-1, 1:, :] - Vz[1:-1, :-1, :]) / dy)
    pad = lambda t, dims: torch.nn.functional.pad(t, dims)
    if pl:
        mod = lambda m: 2.0 * m / (1.0 + m / Gdt)
        mc = mod(mu)
        m_xy = mod(0.25 * (mu[:, 1:, 1:] + mu[:, :-1, 1:] + mu[:, 1:, :-1] + mu[:, :-1, :-1]))
        m_xz = mod(0.25 * (mu[1:, :, 1:] + mu[:-1, :, 1:] + mu[1:, :, :-1] + mu[:-1, :, :-1]))
        m_yz = mod(0.25 * (mu[1:, 1:, :] + mu[:-1, 1:, :] + mu[1:, :-1, :] + mu[:-1, :-1, :]))
    else:
        mc = m_xy = m_xz = m_yz = 2.0 * mu0 / (1.0 + p["xsi_w"])
    txx = mc * (gx - divV / 3.0)
    tyy = mc * (gy - divV / 3.0)
    tzz = mc * (gz - divV / 3.0)
    txy = pad(m_xy * exy, (1, 1, 1, 1))          # zero on boundary edges (free slip)
    txz = pad(m_xz * exz, (1, 1, 0, 0, 1, 1))
    tyz = pad(m_yz * eyz, (0, 0, 1, 1, 1, 1))
    rog = (phi - p["phi0"]) * (p["rhof_g"] - p["rhos_g"])
    Fx = ((txx[:, :, 1:] - txx[:, :, :-1]) / dx + (txy[:, 1:, 1:-1] - txy[:, :-1, 1:-1]) / dy +
          (txz[1:, :, 1:-1] - txz[:-1, :, 1:-1]) / dz - (Pt[:, :, 1:] - Pt[:, :, :-1]) / dx)
    Fy = ((txy[:, 1:-1, 1:] - txy[:, 1:-1, :-1]) / dx + (tyy[:, 1:, :] - tyy[:, :-1, :]) / dy +
          (tyz[1:, 1:-1, :] - tyz[:-1, 1:-1, :]) / dz - (Pt[:, 1:, :] - Pt[:, :-1, :]) / dy)
    Fz = ((txz[1:-1, :, 1:] - txz[1:-1, :, :-1]) / dx + (tyz[1:-1, 1:, :] - tyz[1:-1, :-1, :]) / dy +
          (tzz[1:] - tzz[:-1]) / dz - (Pt[1:] - Pt[:-1]) / dz - 0.5 * (rog[1:] + rog[:-1]))
    # porosity in log space (Eq. 22) with V.grad(1-phi)/(1-phi) advection
    om = 1.0 - phi
    ax = torch.zeros_like(phi)
    ax = ax + torch.nn.functional.pad(Vx[:, :, 1:-1] * (om[:, :, 1:] - om[:, :, :-1]) / dx, (1, 0))
    ax = ax + torch.nn.functional.pad(Vx[:, :, 1:-1] * (om[:, :, 1:] - om[:, :, :-1]) / dx, (0, 1))
    ay = torch.nn.functional.pad(Vy[:, 1:-1, :] * (om[:, 1:, :] - om[:, :-1, :]) / dy, (0, 0, 1, 0)) + \
        torch.nn.functional.pad(Vy[:, 1:-1, :] * (om[:, 1:, :] - om[:, :-1, :]) / dy, (0, 0, 0, 1))
    az = torch.nn.functional.pad(Vz[1:-1] * (om[1:] - om[:-1]) / dz, (0, 0, 0, 0, 1, 0)) + \
        torch.nn.functional.pad(Vz[1:-1] * (om[1:] - om[:-1]) / dz, (0, 0, 0, 0, 0, 1))
    adv = 0.5 * (ax + ay + az) / om
    FL = torch.log(1.0 - phi) - (Lo - dt * (bphi * ((Pf - Pfo) - (Pt - Pto)) / dt + (Pf - Pt) / eta + adv))
    out = dict(Fx=Fx, Fy=Fy, Fz=Fz, Fpt=Fpt, Fpf=Fpf, FL=FL)
    if pl:
        # Picard fixed point of Eq. 24: log mu - log(mu0 / (1 + (tau_II / tau0)^(n-1))), tau_II from
        # the centre stresses and the four edges' shear stresses averaged to the centre
        axy = 0.25 * (txy[:, :-1, :-1] + txy[:, :-1, 1:] + txy[:, 1:, :-1] + txy[:, 1:, 1:])
        axz = 0.25 * (txz[:-1, :, :-1] + txz[:-1, :, 1:] + txz[1:, :, :-1] + txz[1:, :, 1:])
        ayz = 0.25 * (tyz[:-1, :-1, :] + tyz[:-1, 1:, :] + tyz[1:, :-1, :] + tyz[1:, 1:, :])
        t2 = 0.5 * (txx * txx + tyy * tyy + tzz * tzz) + axy * axy + axz * axz + ayz * ayz
        x = (t2 / p["tau0"] ** 2) ** (0.5 * (p["n_pow"] - 1.0))
        out["Fmu"] = torch.log(mu) - np.log(mu0) + torch.log(1.0 + x)
    return out


# ---------------------------------------------------------------- packing of the unknowns
def _interior(u):
    d = dict(Vx=u["Vx"][:, :, 1:-1], Vy=u["Vy"][:, 1:-1, :], Vz=u["Vz"][1:-1], Pt=u["Pt"], Pf=u["Pf"],
             phi=u["phi"])
    if "mu" in u:
        d["mu"] = u["mu"]
    return d


def _pack(d, keys):
    return torch.cat([d[k].reshape(-1) for k in keys])


U_KEYS = ("Vx", "Vy", "Vz", "Pt", "Pf", "phi")
F_KEYS = ("Fx", "Fy", "Fz", "Fpt", "Fpf", "FL")
U_KEYS_PL = U_KEYS + ("mu",)
F_KEYS_PL = F_KEYS + ("Fmu",)


def _keys(p):
    return (U_KEYS_PL, F_KEYS_PL) if p.get("powerlaw_on", 0) else (U_KEYS, F_KEYS)


def _unpack_u(x, p):
    nx, ny, nz = p["nx"], p["ny"], p["nz"]
    shapes = dict(Vx=(nz, ny, nx - 1), Vy=(nz, ny - 1, nx), Vz=(nz - 1, ny, nx), Pt=(nz, ny, nx),
                  Pf=(nz, ny, nx), phi=(nz, ny, nx), mu=(nz, ny, nx))
    out, o = {}, 0
    for k in _keys(p)[0]:
        n = int(np.prod(shapes[k]))
        out[k] = x[o:o + n].reshape(shapes[k])
        o += n
    out["Vx"] = torch.nn.functional.pad(out["Vx"], (1, 1))
    out["Vy"] = torch.nn.functional.pad(out["Vy"], (0, 0, 1, 1))
    out["Vz"] = torch.nn.functional.pad(out["Vz"], (0, 0, 0, 0, 1, 1))
    return out


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=_T)


def state_u(st) -> dict:
    return {k: _t(st[k]) for k in U_KEYS_PL}


def old_from(st) -> dict:
    """Old-step fields a step starting from oracle state `st` uses (mu_o sets its dtS)."""
    return dict(Pto=_t(st["Pt"]), Pfo=_t(st["Pf"]), Lo=torch.log(1.0 - _t(st["phi"])), mu_o=_t(st["mu"]))


def adjoint_params(p: dict, powerlaw: bool = False) -> dict:
    """The scope of the adjoint: no weakening, beta_n = 0; the power law off unless asked for."""
    q = dict(p)
    q.update(powerlaw_on=int(bool(powerlaw)), R_weak=1.0, beta_n=0.0, tau_bg=0.0)
    return q


def forward(p: dict, phi0: np.ndarray, theta: np.ndarray, nsteps: int, tol: float = 1e-12):
    """Converged oracle steps; returns the list of states [u^0, ..., u^N] (oracle states)."""
    q = dict(adjoint_params(p, p.get("powerlaw_on", 0)), tol=tol, max_iter=max(p["max_iter"], 400000))
    st = B.make_state(q, phi0, logk=theta)
    states = [st.copy()]
    for _ in range(nsteps):
        rc, iters, res = B.step(st)
        if rc != 0:
            raise RuntimeError(f"oracle step rc={rc} after {iters} iterations: {res}")
        states.append(st.copy())
    return states


def misfit(phi: np.ndarray, target: np.ndarray) -> float:
    return float(np.sum((phi - target) ** 2))


def gradient(p: dict, states: list, theta: np.ndarray, target: np.ndarray) -> np.ndarray:
    """dJ/dtheta by the discrete adjoint (dense LU per step; tiny grids only)."""
    q = adjoint_params(p, p.get("powerlaw_on", 0))
    UK, FK = _keys(q)
    th = _t(theta)
    N = len(states) - 1
    u = [{k: v for k, v in _interior(state_u(s)).items() if k in UK} for s in states]
    g = {k: torch.zeros_like(v) for k, v in u[N].items()}
    g["phi"] = 2.0 * (_t(states[N]["phi"]) - _t(target))
    grad = torch.zeros_like(th)
    for n in range(N, 0, -1):
        old = old_from(states[n - 1])
        x0 = _pack(u[n], UK)

        def Fu(x):
            return _pack(residual(q, _unpack_u(x, q), old, th), FK)

        Jm = torch.autograd.functional.jacobian(Fu, x0)
        lam = torch.linalg.solve(Jm.T, _pack(g, UK))
        # dJ/dtheta -= (dF/dtheta)^T lambda
        thv = th.clone().requires_grad_(True)
        Fth = _pack(residual(q, _unpack_u(x0, q), old, thv), FK)
        (gth,) = torch.autograd.grad(Fth, thv, grad_outputs=lam)
        grad -= gth
        # carry into the previous step: g^{n-1} = -(dF^n/du^{n-1})^T lambda (through Pto, Pfo,
        # Lo and, with the power law, the previous mu's maximum in dtS)
        prev = {k: v.clone().requires_grad_(True) for k, v in u[n - 1].items()}
        oldv = dict(Pto=prev["Pt"], Pfo=prev["Pf"], Lo=torch.log(1.0 - prev["phi"]),
                    mu_o=prev["mu"] if "mu" in prev else old["mu_o"])
        Fo = _pack(residual(q, _unpack_u(x0, q), oldv, th), FK)
        keys = [k for k in ("Pt", "Pf", "phi", "mu") if k in prev]
        gs = torch.autograd.grad(Fo, [prev[k] for k in keys], grad_outputs=lam, allow_unused=True)
        g = {k: torch.zeros_like(v) for k, v in u[n - 1].items()}
        for k, gk in zip(keys, gs):
            if gk is not None:
                g[k] = -gk
    return grad.numpy()
