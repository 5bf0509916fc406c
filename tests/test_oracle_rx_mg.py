"""Pins of the multigrid (FAS V-cycle) oracle of the reactive porosity-wave step (thesis Art. 3,
Eqs. 8-10; the thesis's future-work section: PT iterations with local pseudo steps are weighted
Jacobi iterations that geometric multigrid can accelerate):

* transfer operators: the 8-child mean restricts an affine field to its values at the coarse
  centres; trilinear prolongation reproduces an affine correction at every fine centre whose
  stencil stays off the walls, keeps constants everywhere and conserves the integral;
* the step equations: at the first iteration of a step their targets are the plain PT
  iteration's (porosity, Xs, rate), the Jacobi denominator holds the diagonal of the Darcy
  operator (probed from the pinned Darcy divergence) plus the implicit local terms;
* the linear limit converges to the exact backward-Euler diffusion step (DCT-II eigenbasis);
* the V-cycle contracts the error of the linear limit by at most the smoothing-factor bound
  (5/7)^4 of four omega = 6/7 Jacobi sweeps in 3-D, independently of the grid, where four sweeps
  of the smoother alone contract the smooth error that remains by no more than 0.9;
* the converged nonlinear step is the plain PT iteration's fixed point, keeps the x and y mirror
  symmetries, and a diverging step is reported (ENAN), not swallowed by the max norm.
"""
import numpy as np
import pytest
import scipy.fft

import pt_inputs as I
from oracle import rx as R

MG = dict(levels=3, nu_pre=2, nu_post=2, nu_coarse=30, max_cycles=200, omega=6.0 / 7.0)


def _affine(shape, d, coef):
    nz, ny, nx = shape
    z, y, x = [(np.arange(m) + 0.5) * h for m, h in zip((nz, ny, nx), d)]
    zz, yy, xx = np.meshgrid(z, y, x, indexing="ij")
    return coef[0] + coef[1] * xx + coef[2] * yy + coef[3] * zz


def test_transfer_operators():
    shape, d = (8, 6, 10), (1.0, 1.0, 1.0)
    coef = (0.3, -1.2, 0.7, 2.1)
    fine = _affine(shape, d, coef)
    coarse = R.mg_restrict(fine)
    np.testing.assert_allclose(coarse, _affine((4, 3, 5), (2.0, 2.0, 2.0), coef), rtol=0, atol=1e-13)
    # affine correction: exact at fine centres whose side neighbour is inside the coarse grid
    e = _affine((4, 3, 5), (2.0, 2.0, 2.0), coef)
    up = R.mg_prolong_add(e, np.zeros(shape))
    np.testing.assert_allclose(up[1:-1, 1:-1, 1:-1], fine[1:-1, 1:-1, 1:-1], rtol=0, atol=1e-13)
    # constants everywhere; integral conserved (each coarse cell spreads a total weight of 8)
    np.testing.assert_allclose(R.mg_prolong_add(np.full((4, 3, 5), 1.7), np.zeros(shape)), 1.7, rtol=1e-15)
    rng = np.random.default_rng(0)
    e = rng.standard_normal((4, 3, 5))
    assert abs(R.mg_prolong_add(e, np.zeros(shape)).sum() - 8.0 * e.sum()) < 1e-12
    base = rng.standard_normal(shape)
    np.testing.assert_allclose(R.mg_prolong_add(e, base) - base, R.mg_prolong_add(e, np.zeros(shape)), atol=1e-14)
    # a one-cell-thick coarse direction degenerates to piecewise-constant interpolation
    e1 = rng.standard_normal((1, 3, 5))
    up1 = R.mg_prolong_add(e1, np.zeros((2, 6, 10)))
    np.testing.assert_allclose(up1[0], up1[1], rtol=0, atol=0)


def test_step_equations_match_the_plain_iteration_and_the_darcy_diagonal():
    p = I.rx_params(6, 5, 9)
    Pf, phi, Xs = I.rx_initial(p)
    rng = np.random.default_rng(4)
    Pf = Pf + 0.05 * rng.standard_normal(Pf.shape)
    omega = 0.8
    gP, gphi, gX, den, Rr = R.mg_equations(p, (Pf, phi, Xs), (Pf, phi, Xs), omega=omega)
    st = R.RxState(p, Pf, phi, Xs)
    rc, _ = R.iterate_n(st, 1)
    assert rc == 0
    # first iteration of a step: Pf_o = Pf, so gP is the rate itself
    np.testing.assert_allclose(Rr, st["R"], rtol=1e-13, atol=0)
    np.testing.assert_allclose(gP, st["R"], rtol=1e-13, atol=0)
    np.testing.assert_allclose(phi + gphi, st["phi"], rtol=1e-14, atol=0)
    np.testing.assert_allclose(Xs + gX, st["Xs"], rtol=1e-14, atol=0)
    # the plain update Pf1 - Pf = dtau R / (1 + dtau (1/dt + a)) gives the implicit local terms
    dtau = R.pseudo_step(p, phi)
    local = (dtau * Rr / (st["Pf"] - Pf) - 1.0) / dtau            # = 1/dt + a
    bp = phi * p["beta_f"] + p["beta_d"] - (1.0 + phi) * p["beta_s"]
    Dk = (den - local) * omega * bp
    # the Darcy operator's diagonal probed from its (pinned) divergence: unit bumps 3 cells apart
    probe = np.zeros_like(Pf)
    base = R.div_qd(p, Pf, phi)
    for a in range(3):
        for b in range(3):
            for c in range(3):
                bump = np.zeros_like(Pf)
                bump[a::3, b::3, c::3] = 1.0
                probe += (R.div_qd(p, Pf + bump, phi) - base) * bump
    np.testing.assert_allclose(Dk, probe, rtol=1e-7)


def _linear(n, dt):
    p = I.rx_params(*n, dt=dt)
    p.update(g=0.0, eta=1e30, tau=1e30, tol=1e-14, max_iter=400000)
    p["beta_s"] = p["beta_d"] * (1.0 - p["phi0"])               # Bphi = 0 at phi0: porosity frozen
    rng = np.random.default_rng(3)
    Pf0 = rng.standard_normal((p["nz"], p["ny"], p["nx"])) * 1e-2
    return p, Pf0, np.full(Pf0.shape, p["phi0"]), np.full(Pf0.shape, 0.02)


def test_linear_limit_is_backward_euler_diffusion():
    p, Pf0, phi, Xs = _linear((16, 8, 24), 2e-4)
    st = R.RxState(p, Pf0, phi, Xs)
    nsteps = 2
    for _ in range(nsteps):
        rc, cycles, ch = R.mg_step(st, MG)
        assert rc == 0, (cycles, ch)
    nx, ny, nz = p["nx"], p["ny"], p["nz"]
    bp = p["phi0"] * p["beta_f"] + p["beta_d"] - (1.0 + p["phi0"]) * p["beta_s"]
    h = (p["lx"] / nx, p["ly"] / ny, p["lz"] / nz)
    lam = [(2.0 - 2.0 * np.cos(np.pi * np.arange(m) / m)) / hh ** 2 for m, hh in zip((nx, ny, nz), h)]
    L = lam[2][:, None, None] + lam[1][None, :, None] + lam[0][None, None, :]
    c = scipy.fft.dctn(Pf0, type=2, norm="ortho") / (1.0 + p["dt"] * p["k0"] * L / bp) ** nsteps
    exact = scipy.fft.idctn(c, type=2, norm="ortho")
    np.testing.assert_allclose(st["Pf"], exact, rtol=0, atol=1e-10 * np.abs(Pf0).max())
    np.testing.assert_allclose(st["phi"], p["phi0"], rtol=1e-14)


def _rates(p, u, mg, ncycles):
    ch = []
    for k in range(1, ncycles + 1):
        st = R.RxState(p, *u)
        rc, c = R.mg_cycles(st, mg, k)
        assert rc == 0
        ch.append(c)
    return [ch[i + 1] / ch[i] for i in range(len(ch) - 1)]


def test_vcycle_contraction_is_bounded_and_grid_independent():
    bound = (5.0 / 7.0) ** 4
    rho = {}
    for n, levels in ((8, 3), (16, 4)):
        p, Pf0, phi, Xs = _linear((n, n, 4 * n), 1e-2)
        r = _rates(p, (Pf0, phi, Xs), dict(MG, levels=levels), 7)
        rho[n] = max(r[3:])
        assert rho[n] <= bound, (n, r)
    assert abs(rho[8] - rho[16]) < 0.05, rho
    p, Pf0, phi, Xs = _linear((16, 16, 64), 1e-2)
    r = _rates(p, (Pf0, phi, Xs), dict(MG, levels=1, nu_coarse=50), 4)
    assert r[-1] ** (4.0 / 50.0) > 0.9, r                          # the smoother alone stalls


def test_converged_step_is_the_plain_fixed_point_and_far_cheaper():
    p = I.rx_params(16, dt=1e-4)
    p.update(tol=1e-14, max_iter=400000)
    u = I.rx_initial(p)
    mg_st, pl_st = R.RxState(p, *u), R.RxState(p, *u)
    rc, cycles, ch = R.mg_step(mg_st, dict(MG, levels=4))
    assert rc == 0, (cycles, ch)
    rc, iters, ch = R.step(pl_st)
    assert rc == 0, (iters, ch)
    assert 20 * cycles < iters, (cycles, iters)
    for k in ("Pf", "phi", "Xs", "R"):
        s = np.abs(pl_st[k]).max()
        np.testing.assert_allclose(mg_st[k], pl_st[k], rtol=0, atol=1e-9 * s, err_msg=k)
    a = mg_st["Pf"]
    np.testing.assert_allclose(a, a[:, :, ::-1], rtol=0, atol=1e-12 * np.abs(a).max())
    np.testing.assert_allclose(a, a[:, ::-1, :], rtol=0, atol=1e-12 * np.abs(a).max())


def test_diverging_step_is_reported():
    p = I.rx_params(8, dt=1e-2)
    u = I.rx_initial(p)
    assert R.mg_step(R.RxState(p, *u), MG)[0] == -3
    assert R.step(R.RxState(p, *u))[0] == -3


@pytest.mark.parametrize("bad", [dict(levels=4), dict(nu_post=0), dict(nu_coarse=0), dict(omega=1.5),
                                 dict(levels=0)])
def test_invalid_hierarchy_is_rejected(bad):
    p = I.rx_params(12, 12, 20)                                   # 20 is not divisible by 8
    u = I.rx_initial(p)
    assert R.mg_step(R.RxState(p, *u), dict(MG, **bad))[0] == -1
