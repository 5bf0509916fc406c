"""Solver-level pins of the oracle: what the thesis's equations fix independently of the code.

* linear diffusion limit vs the exact discrete (DCT) backward-Euler solution;
* uniform (0-D) compaction vs the continuum ODE of Eqs. 1, 2 and 6 (first-order in dt);
* hydrostatic rest states that must not move;
* telescoping (conservation) of div V and div qD with free-slip / no-flux boundaries;
* mirror symmetry of a centred anomaly;
* monotone reduction of the residual to tolerance within the cap (32^3 workload);
* the PT + Picard fixed point equals the root of the implicit-step residual found by a
  brute-force Newton solve with a finite-difference Jacobian and dense LU (tiny grid).
"""
import numpy as np
import pytest
import scipy.fft
from scipy.integrate import solve_ivp

import pt_inputs as I


def _base(nx, ny, nz, **kw):
    p = I.c1_params(nx, ny, nz)
    p.update(kw)
    return p


# ------------------------------------------------------------------ diffusion limit (DCT)
def _neumann_eigs(p):
    """Eigenvalues of the negative cell-centred Neumann Laplacian in the DCT-II basis."""
    lam = 0.0
    for n, L, ax in ((p["nx"], p["lx"], 2), (p["ny"], p["ly"], 1), (p["nz"], p["lz"], 0)):
        h = L / n
        m = np.arange(n)
        e = 4.0 / h ** 2 * np.sin(np.pi * m / (2 * n)) ** 2
        shape = [1, 1, 1]
        shape[ax] = n
        lam = lam + e.reshape(shape)
    return lam


@pytest.mark.parametrize("dims", [(12, 10, 8), (9, 11, 7)])
def test_diffusion_limit_matches_dct_backward_euler(oracle_lib, dims):
    """Solid frozen, no compaction, uniform porosity, no buoyancy: Eqs. 17-18 reduce to
    dPt = alpha dPf and S dPf/dt = k lap(Pf), S = beta_d alpha (1/B - alpha); with zero-flux
    walls backward Euler is diagonal in the cosine basis (exact discrete solution)."""
    O = oracle_lib
    nx, ny, nz = dims
    p = _base(nx, ny, nz, lx=1.0, ly=0.9, lz=1.1, compaction_on=0, beta_phi=0.0,
              rhos_g=1.0, rhof_g=1.0, tol=1e-12, max_iter=400000, dt=3e-5)
    S = p["beta_d"] * p["alpha"] * (1.0 / p["B"] - p["alpha"])
    k = p["k0"]
    phi = np.full((nz, ny, nx), p["phi0"])
    x = (np.arange(nx) + 0.5) / nx * p["lx"]
    y = (np.arange(ny) + 0.5) / ny * p["ly"]
    z = (np.arange(nz) + 0.5) / nz * p["lz"]
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    Pf0 = 0.01 * np.exp(-((X - 0.4) ** 2 + (Y - 0.5) ** 2 + (Z - 0.6) ** 2) / 0.15 ** 2)
    st = O.make_state(p, phi, fields=dict(Pf=Pf0))
    lam = _neumann_eigs(p)
    ref_f, ref_t = Pf0.copy(), np.zeros_like(Pf0)
    for step in range(4):
        rc, iters, res = O.step(st, mech_on=0)
        assert rc == 0, (rc, iters, res)
        new_f = scipy.fft.idctn(scipy.fft.dctn(ref_f, type=2, norm="ortho") /
                                (1.0 + p["dt"] * k * lam / S), type=2, norm="ortho")
        ref_t = ref_t + p["alpha"] * (new_f - ref_f)
        ref_f = new_f
        scale = np.abs(ref_f).max()
        np.testing.assert_allclose(st["Pf"], ref_f, rtol=0, atol=1e-8 * scale)
        np.testing.assert_allclose(st["Pt"], ref_t, rtol=0, atol=1e-8 * scale)
    # and the solution actually diffused (not a trivial pass)
    assert np.abs(st["Pf"] - Pf0).max() > 0.05 * np.abs(Pf0).max()
    np.testing.assert_allclose(st["phi"], phi, rtol=1e-13)   # porosity frozen in this limit


# --------------------------------------------------------------- 0-D compaction vs ODE
def _ode_rhs(p, R_weak):
    bd, al, B, bphi, eta0, mu0 = p["beta_d"], p["alpha"], p["B"], p["beta_phi"], p["eta0"], p["mu0"]
    M = np.array([[-bd, al * bd], [al * bd, -al * bd / B]])

    def rhs(t, u):
        Pt, Pf, phi = u
        R = R_weak if Pf > Pt else 1.0
        eta = eta0 * mu0 / phi * R                         # Eqs. 9-10 (Picard target)
        d = Pt - Pf
        c = d / ((1.0 - phi) * eta)
        # Eq. 1 with div V = 0:    -beta_d (Pt' - al Pf') - c = 0
        # Eq. 2 with no flux:       al beta_d (Pt' - Pf' / B) + c = 0
        dPt, dPf = np.linalg.solve(M, np.array([c, -c]))
        # Eq. 6: phi' / (1 - phi) = -beta_phi (Pt' - Pf') - d / eta
        dphi = (1.0 - phi) * (-bphi * (dPt - dPf) - d / eta)
        return [dPt, dPf, dphi]
    return rhs


@pytest.mark.parametrize("dP0, R_weak", [(-0.4, 0.1), (0.4, 0.1)])
def test_uniform_compaction_matches_continuum_ode_first_order(oracle_lib, dP0, R_weak):
    """Uniform fields: the backward-Euler + PT + Picard solution converges to the continuum
    ODE of Eqs. 1, 2, 6 (with Eqs. 9-10) at first order in dt. The run stops well before
    Pt - Pf decays to round-off, where the sign switch of Eq. 9 would be decided by noise."""
    O = oracle_lib
    T = 0.6
    errs = []
    for nt in (10, 20, 40):
        p = _base(2, 2, 2, lx=10.0, ly=10.0, lz=10.0, rhos_g=1.0, rhof_g=1.0, dt=T / nt,
                  tol=1e-13, max_iter=500000, eta0=5.0, beta_phi=0.02)
        phi = np.full((2, 2, 2), 0.02)
        st = O.make_state(p, phi, fields=dict(Pf=np.full((2, 2, 2), -dP0 / 2),
                                              Pt=np.full((2, 2, 2), dP0 / 2)))
        # start from the converged Picard state eta = eta*(phi, R) of the initial pressures
        R0 = R_weak if -dP0 / 2 > dP0 / 2 else 1.0
        st["eta"][...] = p["eta0"] * p["mu0"] / phi * R0
        for _ in range(nt):
            rc, iters, res = O.step(st, R_weak=R_weak)
            assert rc == 0, (rc, iters, res)
        sol = solve_ivp(_ode_rhs(dict(p, R_weak=R_weak), R_weak), (0, T),
                        [dP0 / 2, -dP0 / 2, 0.02], rtol=1e-11, atol=1e-13, method="Radau")
        exact = sol.y[:, -1]
        got = np.array([st["Pt"][0, 0, 0], st["Pf"][0, 0, 0], st["phi"][0, 0, 0]])
        for a in ("Pt", "Pf", "phi"):
            assert np.ptp(st[a]) == 0.0                    # stays uniform
        errs.append(np.abs(got - exact) / np.array([abs(dP0), abs(dP0), 0.02]))
    errs = np.array(errs)
    # the solution moved by O(1) of its scale, and the error halves with dt (first order)
    assert abs(exact[0] - exact[1] - dP0) > 0.1 * abs(dP0)
    ratio = errs[:-1].max(axis=1) / errs[1:].max(axis=1)
    assert np.all(ratio > 1.7) and np.all(ratio < 2.3), (errs, ratio)
    assert errs[-1].max() < 0.05


# ----------------------------------------------------------------------- rest states
def _coords(p):
    nx, ny, nz = p["nx"], p["ny"], p["nz"]
    z = (np.arange(nz) + 0.5) / nz * p["lz"]
    return np.broadcast_to(z[:, None, None], (nz, ny, nx)).copy()


def test_rest_state_equal_densities_stays_zero(oracle_lib):
    """rho_s = rho_f, uniform porosity, zero pressures and velocity: nothing drives motion."""
    O = oracle_lib
    p = _base(6, 5, 7, rhos_g=1.0, rhof_g=1.0)
    st = O.make_state(p, np.full((7, 5, 6), p["phi0"]))
    for _ in range(3):
        rc, iters, res = O.step(st)
        assert rc == 0 and iters == p["nup"]
    for k in ("Vx", "Vy", "Vz", "Pt", "Pf", "txx", "txy", "Rz"):
        assert np.all(st[k] == 0.0), k
    np.testing.assert_allclose(st["phi"], p["phi0"], rtol=1e-14)


@pytest.mark.parametrize("phi_fac", [1.0, 1.5])
def test_hydrostatic_rest_state_does_not_move(oracle_lib, phi_fac):
    """Uniform porosity, compaction off, Pf hydrostatic w.r.t. (rho_f - rho_BG) g and Pt in
    balance with the buoyancy (phi - phi0)(rho_f - rho_s) g: no Darcy flux, no net force.
    Pins the gravity signs of Eqs. 19-20."""
    O = oracle_lib
    p = _base(6, 5, 8, compaction_on=0)
    phi0 = p["phi0"]
    phi = phi_fac * phi0
    rho_bg = phi0 * p["rhof_g"] + (1 - phi0) * p["rhos_g"]
    rog = phi * p["rhof_g"] + (1 - phi) * p["rhos_g"] - rho_bg
    z = _coords(p)
    Pf = (rho_bg - p["rhof_g"]) * (z - 0.5)
    Pt = -rog * (z - 0.5)
    st = O.make_state(p, np.full(z.shape, phi), fields=dict(Pf=Pf, Pt=Pt))
    for _ in range(3):
        rc, iters, res = O.step(st)
        assert rc == 0, (rc, res)
    np.testing.assert_allclose(st["Pf"], Pf, rtol=0, atol=1e-13)
    np.testing.assert_allclose(st["Pt"], Pt, rtol=0, atol=1e-13)
    for k in ("Vx", "Vy", "Vz"):
        assert np.abs(st[k]).max() < 1e-12, k
    np.testing.assert_allclose(st["phi"], phi, rtol=1e-14)


# ---------------------------------------------------------------------- conservation
def test_divergences_telescope_to_zero(oracle_lib):
    """Free slip (zero normal V) and zero normal Darcy flux: sum over cells of div V and of
    div qD vanish to round-off, for any state, also after PT iterations."""
    O = oracle_lib
    p = _base(7, 6, 5)
    rs = I.random_state(p, seed=11)
    st = O.make_state(p, rs["phi"], fields={k: v for k, v in rs.items() if k != "phi"})
    O.begin_step(st)
    for it0 in (0, 30):
        if it0:
            rc, _ = O.iterate_n(st, 0, it0)
            assert rc == 0
        dv, _ = O.divergence(p, st["Vx"], st["Vy"], st["Vz"], st["Pt"], st["Pf"], st["Pto"],
                             st["Pfo"], st["phi"], st["eta"])
        perm, _ = O.coefficients(p, st["phi"])
        qx, qy, qz, dq = O.darcy(p, st["Pf"], perm)
        h = (p["lx"] / 7, p["ly"] / 6, p["lz"] / 5)
        vol = h[0] * h[1] * h[2]
        for field, face_terms in ((dv, np.abs(st["Vx"]).sum() / h[0] + np.abs(st["Vy"]).sum() / h[1] +
                                   np.abs(st["Vz"]).sum() / h[2]),
                                  (dq, np.abs(qx).sum() / h[0] + np.abs(qy).sum() / h[1] +
                                   np.abs(qz).sum() / h[2])):
            assert abs(field.sum() * vol) <= 1e-13 * face_terms * vol


# ---------------------------------------------------------------------- symmetry
def test_mirror_symmetry_of_centred_anomaly(oracle_lib):
    O = oracle_lib
    p = I.c1_params(16)
    st = O.make_state(p, I.gaussian_porosity(p))
    O.begin_step(st)
    rc, _ = O.iterate_n(st, 0, 300)
    assert rc == 0
    phi, Vx, Vy, Vz = st["phi"], st["Vx"], st["Vy"], st["Vz"]
    sc = np.abs(phi).max()
    np.testing.assert_allclose(phi, phi[:, :, ::-1], rtol=0, atol=1e-12 * sc)
    np.testing.assert_allclose(phi, phi[:, ::-1, :], rtol=0, atol=1e-12 * sc)
    np.testing.assert_allclose(phi, phi.transpose(0, 2, 1), rtol=0, atol=1e-12 * sc)
    sv = np.abs(Vz).max()
    assert sv > 0
    np.testing.assert_allclose(Vx, -Vx[:, :, ::-1], rtol=0, atol=1e-12 * sv)
    np.testing.assert_allclose(Vy, -Vy[:, ::-1, :], rtol=0, atol=1e-12 * sv)
    np.testing.assert_allclose(Vz, Vz[:, :, ::-1], rtol=0, atol=1e-12 * sv)
    np.testing.assert_allclose(Vx, Vy.transpose(0, 2, 1), rtol=0, atol=1e-12 * sv)
    for k in ("Pt", "Pf", "mu", "eta"):
        a = st[k]
        np.testing.assert_allclose(a, a[:, :, ::-1], rtol=0, atol=1e-12 * np.abs(a).max())


# -------------------------------------------------------------- residual reduction
@pytest.mark.slow
def test_workload_32_converges_with_monotone_residual(oracle_lib):
    """The 32^3 single-step workload reaches max-norm residual 1e-8 under the 20000 cap, and
    the running maximum of the residual over windows of 32 checks decreases window by window."""
    O = oracle_lib
    p = I.c1_params(32)
    st = O.make_state(p, I.gaussian_porosity(p))
    O.begin_step(st)
    hist, it = [], 0
    while it < p["max_iter"]:
        rc, res = O.iterate_n(st, it, p["nup"])
        it += p["nup"]
        assert rc == 0
        r = max(res.values())
        hist.append(r)
        if r < p["tol"]:
            break
    assert hist[-1] < p["tol"] and it < p["max_iter"]
    w = 32
    wmax = [max(hist[i:i + w]) for i in range(0, len(hist) - w + 1, w)]
    assert all(b < a for a, b in zip(wmax, wmax[1:])), wmax
    # physics moved: the fluid, lighter than the background, rises; the fluid pressure builds
    # at the top (decompaction, Pf > Pt) and drops at the bottom (compaction, Pf < Pt)
    pf = st["Pf"].mean(axis=(1, 2))
    assert np.all(np.diff(pf) > 0)
    d = st["Pf"] - st["Pt"]
    assert d[-1].min() > 0 and d[0].max() < 0


# --------------------------------------------------------------- brute-force Newton
_VARS = ("Vx", "Vy", "Vz", "Pt", "Pf", "phi", "mu", "eta")


def _interior_masks(p):
    nx, ny, nz = p["nx"], p["ny"], p["nz"]
    mx = np.zeros((nz, ny, nx + 1), bool); mx[:, :, 1:-1] = True
    my = np.zeros((nz, ny + 1, nx), bool); my[:, 1:-1, :] = True
    mz = np.zeros((nz + 1, ny, nx), bool); mz[1:-1, :, :] = True
    mc = np.ones((nz, ny, nx), bool)
    return dict(Vx=mx, Vy=my, Vz=mz, Pt=mc, Pf=mc, phi=mc, mu=mc, eta=mc)


def _pack(st, masks):
    """Unknown vector; the viscosities enter through their logarithms (positive by design)."""
    return np.concatenate([(np.log(st[k]) if k in ("mu", "eta") else st[k])[masks[k]] for k in _VARS])


def _unpack(st, masks, x):
    o = 0
    for k in _VARS:
        n = int(masks[k].sum())
        st[k][masks[k]] = np.exp(x[o:o + n]) if k in ("mu", "eta") else x[o:o + n]
        o += n


def _resid(O, st, masks):
    r = O.system_residual(st)
    m = masks
    return np.concatenate([r["Vx"][m["Vx"]], r["Vy"][m["Vy"]], r["Vz"][m["Vz"]], r["pt"].ravel(),
                           r["pf"].ravel(), r["L"].ravel(), r["mu"].ravel(), r["eta"].ravel()])


@pytest.mark.parametrize("R_weak", [1.0, 0.01])
def test_pt_fixed_point_equals_newton_root(oracle_lib, R_weak):
    """Tiny nonlinear problem (power law active, compaction, weakening): Newton on the
    implicit-step residual from the old state, with a central-difference Jacobian and dense LU,
    converges to the same state as the PT + Picard iteration."""
    O = oracle_lib
    p = _base(3, 4, 5, lx=1.0, ly=1.2, lz=1.4, tau0=1e-2, R_weak=R_weak, dt=2e-3,
              tol=1e-12, max_iter=2000000)
    phi = I.gaussian_porosity(p, centres=((0.45, 0.55, 0.5),), width=0.3)
    st0 = O.make_state(p, phi)
    masks = _interior_masks(p)
    # PT solution of one step
    st = st0.copy()
    rc, iters, res = O.step(st)
    assert rc == 0, (rc, iters, res)
    # damped Newton from the old state; with weakening the old state (Pf = Pt = 0) sits on the
    # switch of Eq. 9 where finite differences straddle its jump, so that case starts from an
    # early PT iterate instead (still far from the answer, pressures off the switch)
    nw = st0.copy()
    O.begin_step(nw)
    if R_weak != 1.0:
        rc, r0 = O.iterate_n(nw, 0, 60)
        assert rc == 0 and max(r0.values()) > 1e-3
    x = _pack(nw, masks)
    scale = np.concatenate([np.full(int(masks[k].sum()), s) for k, s in
                            zip(_VARS, (1e-3, 1e-3, 1e-3, 1e-2, 1e-2, 1e-2, 1.0, 1.0))])
    r = _resid(O, nw, masks)
    for newton_it in range(60):
        if np.abs(r).max() < 1e-13:
            break
        J = np.empty((r.size, x.size))
        for j in range(x.size):
            h = 1e-6 * max(abs(x[j]), scale[j])
            xp, xm = x.copy(), x.copy()
            xp[j] += h; xm[j] -= h
            _unpack(nw, masks, xp); rp = _resid(O, nw, masks)
            _unpack(nw, masks, xm); rm = _resid(O, nw, masks)
            J[:, j] = (rp - rm) / (2 * h)
        dx = np.linalg.solve(J, r)
        lam = 1.0
        while True:                                    # backtracking on the residual norm
            xt = x - lam * dx
            _unpack(nw, masks, xt)
            rt = _resid(O, nw, masks)
            if np.all(np.isfinite(rt)) and np.linalg.norm(rt) < np.linalg.norm(r) or lam < 1e-4:
                break
            lam *= 0.5
        x, r = xt, rt
    _unpack(nw, masks, x)
    assert np.abs(_resid(O, nw, masks)).max() < 1e-11
    mus = st["mu"]
    assert mus.min() < 0.95 * p["mu0"]                       # the power law is active
    if R_weak != 1.0:
        assert np.any(st["Pf"] > st["Pt"]) and np.any(st["Pf"] < st["Pt"])
    for k in _VARS:
        a, b = st[k], nw[k]
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-9 * max(np.abs(b).max(), 1e-30), err_msg=k)
