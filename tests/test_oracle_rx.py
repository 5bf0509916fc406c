"""Pins of the reactive porosity-wave oracle (thesis Art. 3, Eqs. 8-10; appendix A.6 form):

* 0-D: a uniform state without gravity is one scalar implicit step; the oracle's converged step
  equals the root of the four scalar step equations solved independently (scipy fsolve);
* linear limit: compaction and reaction off and beta_s = beta_d (1 - phi0) (porosity frozen),
  no gravity: the fluid pressure obeys backward-Euler diffusion with no-flux walls, whose exact
  discrete solution comes from the DCT-II eigenbasis of the Neumann Laplacian;
* fast reaction: with dt / tau = 10 the converged Xs keeps tau / (tau + dt) of the old
  disequilibrium from Xs_eq(Pf) (backward Euler of Eq. 10); a reaction time far below dt makes
  the iteration diverge, which the step reports (ENAN) instead of converging on NaN;
* the Darcy divergence telescopes to zero over the box (no-flux walls) and vanishes for the
  hydrostatic fluid pressure Pf = rho_f g z;
* two anomalies centred in x and y keep the x and y mirror symmetries.
"""
import numpy as np
import pytest
import scipy.fft
from scipy.optimize import fsolve

import pt_inputs as I
from oracle import rx as R


def _p(n=(6, 5, 8), **kw):
    p = I.rx_params(*n)
    p.update(kw)
    return p


def test_uniform_state_is_the_scalar_implicit_step():
    p = _p(g=0.0, tol=1e-15, max_iter=200000, dt=1e-3)
    shape = (p["nz"], p["ny"], p["nx"])
    Pf0, phi0, Xs0 = 0.1, 0.015, 0.01
    st = R.RxState(p, np.full(shape, Pf0), np.full(shape, phi0), np.full(shape, Xs0))
    rc, iters, ch = R.step(st)
    assert rc == 0, (iters, ch)
    dt, tau, eta, dX = p["dt"], p["tau"], p["eta"], p["dX"]
    Sr = 1.0 - p["rhos"] / (p["rhof"] * (1.0 + dX))

    def eqs(u):
        Pf, phi, Xs, Rt = u
        xseq = min(max(p["beta_x"] * Pf + 0.5 * p["xs_max"], 0.0), p["xs_max"])
        dXs = (xseq - Xs) / tau
        bphi = p["beta_d"] - p["beta_s"] / (1.0 - phi)
        bp = phi * p["beta_f"] + p["beta_d"] - (1.0 + phi) * p["beta_s"]
        return [Rt - (Pf - Pf0) / dt,
                Xs - (Xs0 + dt * dXs),
                phi - (phi0 + dt * (1.0 - phi) * (bphi * Rt + Pf / (eta * (1.0 - phi)) - (1.0 + dX) / (1.0 - Xs) * dXs)),
                Rt * bp - (-Pf / (eta * (1.0 - phi)) + Sr * (1.0 - phi) * (1.0 + dX) / (1.0 - Xs) * dXs)]

    sol = fsolve(eqs, [Pf0, phi0, Xs0, 0.0], xtol=1e-13)
    assert max(abs(v) for v in eqs(sol)) < 1e-10
    for k, v in zip(("Pf", "phi", "Xs", "R"), sol):
        np.testing.assert_allclose(st[k], v, rtol=1e-9, atol=1e-13, err_msg=k)
    assert abs(sol[0] - Pf0) > 1e-3 and abs(sol[2] - Xs0) > 1e-5     # the step does move


def test_linear_limit_is_backward_euler_diffusion():
    p = _p(n=(9, 7, 11), g=0.0, eta=1e30, tau=1e30, tol=1e-15, max_iter=400000, dt=2e-4)
    p["beta_s"] = p["beta_d"] * (1.0 - p["phi0"])           # Bphi = 0 at phi0: porosity frozen
    nx, ny, nz = p["nx"], p["ny"], p["nz"]
    rng = np.random.default_rng(3)
    Pf0 = rng.standard_normal((nz, ny, nx)) * 1e-2
    st = R.RxState(p, Pf0, np.full(Pf0.shape, p["phi0"]), np.full(Pf0.shape, 0.02))
    nsteps = 3
    for _ in range(nsteps):
        rc, iters, ch = R.step(st)
        assert rc == 0, (iters, ch)
    bp = p["phi0"] * p["beta_f"] + p["beta_d"] - (1.0 + p["phi0"]) * p["beta_s"]
    h = (p["lx"] / nx, p["ly"] / ny, p["lz"] / nz)
    lam = [(2.0 - 2.0 * np.cos(np.pi * np.arange(m) / m)) / hh ** 2 for m, hh in zip((nx, ny, nz), h)]
    L = lam[2][:, None, None] + lam[1][None, :, None] + lam[0][None, None, :]
    c = scipy.fft.dctn(Pf0, type=2, norm="ortho")
    c = c / (1.0 + p["dt"] * p["k0"] * L / bp) ** nsteps
    exact = scipy.fft.idctn(c, type=2, norm="ortho")
    np.testing.assert_allclose(st["Pf"], exact, rtol=0, atol=1e-10 * np.abs(Pf0).max())
    np.testing.assert_allclose(st["phi"], p["phi0"], rtol=1e-14)


def test_fast_reaction_relaxes_xs_towards_equilibrium():
    # backward Euler of dXs/dt = (Xs_eq - Xs) / tau leaves tau / (tau + dt) of the old
    # disequilibrium (Eq. 10); dt / tau = 10, from a state in equilibrium before the step
    p = _p(tau=1e-7, tol=1e-14, max_iter=400000)
    Pf, phi, _ = I.rx_initial(p)
    Pf = Pf + 0.05
    xs0 = np.clip(p["beta_x"] * Pf + 0.5 * p["xs_max"], 0.0, p["xs_max"])
    st = R.RxState(p, Pf, phi, xs0)
    rc, iters, ch = R.step(st)
    assert rc == 0, (iters, ch)
    xseq = np.clip(p["beta_x"] * st["Pf"] + 0.5 * p["xs_max"], 0.0, p["xs_max"])
    gap_old = np.abs(xs0 - xseq)
    assert gap_old.max() > 1e-8                                    # the fluid pressure did move
    shrink = p["tau"] / (p["tau"] + p["dt"])
    assert np.all(np.abs(st["Xs"] - xseq) <= gap_old * shrink * (1.0 + 1e-6) + 1e-15)


def test_diverging_step_reports_nan():
    # a reaction time far below dt makes the first Jacobi iterate's porosity rate explode
    p = _p(tau=1e-12, tol=1e-14, max_iter=1000)
    Pf, phi, Xs = I.rx_initial(p)
    st = R.RxState(p, Pf + 0.05, phi, Xs)
    rc, iters, ch = R.step(st)
    assert rc == -3 and not np.isfinite(ch), (rc, iters, ch)


def test_darcy_divergence_telescopes_and_hydrostatic_flux_vanishes():
    p = _p()
    rng = np.random.default_rng(1)
    shape = (p["nz"], p["ny"], p["nx"])
    phi = p["phi0"] * (1.0 + 0.5 * rng.random(shape))
    Pf = rng.standard_normal(shape)
    dq = R.div_qd(p, Pf, phi)
    vol = p["lx"] * p["ly"] * p["lz"] / np.prod(shape)
    assert abs(dq.sum() * vol) <= 1e-11 * np.abs(dq).max()
    z = (np.arange(p["nz"]) + 0.5) * p["lz"] / p["nz"]
    hyd = np.broadcast_to(p["rhof"] * p["g"] * z[:, None, None], shape).copy()
    assert np.abs(R.div_qd(p, hyd, phi)).max() <= 1e-11


def test_centred_anomalies_keep_mirror_symmetry():
    p = _p(n=(8, 8, 24))
    Pf, phi, Xs = I.rx_initial(p)
    st = R.RxState(p, Pf, phi, Xs)
    for _ in range(2):
        rc, iters, ch = R.step(st)
        assert rc == 0
    for k in ("Pf", "phi", "Xs", "R"):
        a = st[k]
        s = max(np.abs(a).max(), 1e-30)
        np.testing.assert_allclose(a, a[:, :, ::-1], rtol=0, atol=1e-12 * s, err_msg=k)
        np.testing.assert_allclose(a, a[:, ::-1, :], rtol=0, atol=1e-12 * s, err_msg=k)
    assert np.abs(st["Pf"]).max() > 1e-3
