"""Unit pins of the oracle's discrete operators against closed forms.

Second-order centred differences on the staggered grid of Fig. 1 (thesis Art. 1) are exact on
polynomials of degree <= 2, so each operator is checked against the continuum expression of a
random quadratic field evaluated at the staggered positions. These catch wrong signs, indices,
transposed operands and dropped terms in the building blocks of one PT iteration.
"""
import numpy as np
import pytest

import pt_inputs as I


def _grid(nx, ny, nz, lx=1.0, ly=1.3, lz=0.9):
    p = I.c1_params(nx, ny, nz)
    p.update(lx=lx, ly=ly, lz=lz)
    return p


def _coords(p):
    nx, ny, nz = p["nx"], p["ny"], p["nz"]
    dx, dy, dz = p["lx"] / nx, p["ly"] / ny, p["lz"] / nz
    xc, yc, zc = (np.arange(nx) + 0.5) * dx, (np.arange(ny) + 0.5) * dy, (np.arange(nz) + 0.5) * dz
    xf, yf, zf = np.arange(nx + 1) * dx, np.arange(ny + 1) * dy, np.arange(nz + 1) * dz
    return dict(xc=xc, yc=yc, zc=zc, xf=xf, yf=yf, zf=zf)


def _mesh(z, y, x):
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return X, Y, Z


class Quad:
    """f = c0 + c.x + x^T A x (A symmetric), with its exact gradient and Hessian."""

    def __init__(self, rng, scale=1.0):
        self.c0 = rng.standard_normal() * scale
        self.c = rng.standard_normal(3) * scale
        a = rng.standard_normal((3, 3)) * scale
        self.A = 0.5 * (a + a.T)

    def __call__(self, X, Y, Z):
        A, c = self.A, self.c
        return (self.c0 + c[0] * X + c[1] * Y + c[2] * Z + A[0, 0] * X * X + A[1, 1] * Y * Y +
                A[2, 2] * Z * Z + 2 * A[0, 1] * X * Y + 2 * A[0, 2] * X * Z + 2 * A[1, 2] * Y * Z)

    def grad(self, X, Y, Z):
        A, c = self.A, self.c
        return [c[i] + 2 * (A[i, 0] * X + A[i, 1] * Y + A[i, 2] * Z) for i in range(3)]

    def hess(self):
        return 2 * self.A


def test_divergence_exact_on_quadratics(oracle_lib):
    O = oracle_lib
    p = _grid(7, 6, 5)
    g = _coords(p)
    rng = np.random.default_rng(1)
    V = [Quad(rng) for _ in range(3)]
    Vx = V[0](*_mesh(g["zc"], g["yc"], g["xf"]))
    Vy = V[1](*_mesh(g["zc"], g["yf"], g["xc"]))
    Vz = V[2](*_mesh(g["zf"], g["yc"], g["xc"]))
    Xc = _mesh(g["zc"], g["yc"], g["xc"])
    z = np.zeros_like(Xc[0])
    divV, divVn = O.divergence(p, Vx, Vy, Vz, z, z, z, z, np.full_like(z, 0.01), np.ones_like(z))
    exact = V[0].grad(*Xc)[0] + V[1].grad(*Xc)[1] + V[2].grad(*Xc)[2]
    np.testing.assert_allclose(divV, exact, rtol=0, atol=1e-12)
    np.testing.assert_allclose(divVn, exact, rtol=0, atol=1e-12)   # pressures zero


def test_darcy_flux_divergence_exact_and_zero_boundary_flux(oracle_lib):
    """Uniform k: div qD = -k lap(Pf) in cells whose faces are all interior; boundary faces
    carry no flux (Eq. 34), so boundary cells see only their interior faces."""
    O = oracle_lib
    p = _grid(8, 7, 6)
    p["rhos_g"] = p["rhof_g"]          # no buoyancy term in the flux
    g = _coords(p)
    rng = np.random.default_rng(2)
    f = Quad(rng)
    Xc = _mesh(g["zc"], g["yc"], g["xc"])
    Pf = f(*Xc)
    phi = np.full(Pf.shape, p["phi0"] * 1.5)
    perm, rog = O.coefficients(p, phi)
    np.testing.assert_allclose(perm, p["k0"] * 1.5 ** 3, rtol=1e-15)   # Eq. 23
    np.testing.assert_allclose(rog, 0.0, atol=1e-15)
    qx, qy, qz, div = O.darcy(p, Pf, perm)
    k = perm[0, 0, 0]
    lap = np.trace(f.hess())
    inner = (slice(1, -1),) * 3
    np.testing.assert_allclose(div[inner], -k * lap, rtol=1e-10, atol=1e-10)
    for q, sl in ((qx, (Ellipsis, 0)), (qx, (Ellipsis, -1)), (qy, (slice(None), 0)),
                  (qy, (slice(None), -1)), (qz, 0), (qz, -1)):
        assert np.all(q[sl] == 0.0)
    # interior face flux = -k * dPf/dn at the face midpoint (exact for quadratics)
    Xfx = _mesh(g["zc"], g["yc"], g["xf"])
    np.testing.assert_allclose(qx[:, :, 1:-1], -k * f.grad(*Xfx)[0][:, :, 1:-1], rtol=1e-11, atol=1e-11)


def test_darcy_gravity_sign(oracle_lib):
    """Gravity along -z: with Pf = 0 a fluid lighter than the background rises (qz > 0)."""
    O = oracle_lib
    p = _grid(4, 4, 6)
    phi = np.full((6, 4, 4), p["phi0"])
    perm, _ = O.coefficients(p, phi)
    _, _, qz, _ = O.darcy(p, np.zeros_like(phi), perm)
    rho_bg = p["phi0"] * p["rhof_g"] + (1 - p["phi0"]) * p["rhos_g"]
    np.testing.assert_allclose(qz[1:-1], p["k0"] * (rho_bg - p["rhof_g"]), rtol=1e-14)
    assert np.all(qz[1:-1] > 0)


def _stress_setup(p, rng, dtS, mu_val):
    g = _coords(p)
    V = [Quad(rng) for _ in range(3)]
    Vx = V[0](*_mesh(g["zc"], g["yc"], g["xf"]))
    Vy = V[1](*_mesh(g["zc"], g["yf"], g["xc"]))
    Vz = V[2](*_mesh(g["zf"], g["yc"], g["xc"]))
    sh = I.field_shapes(p["nx"], p["ny"], p["nz"])
    zc = np.zeros(sh["centre"])
    divV, divVn = O_div(p, Vx, Vy, Vz)
    mu = np.full(sh["centre"], mu_val)
    return g, V, (Vx, Vy, Vz), divV, divVn, mu, sh, zc


def O_div(p, Vx, Vy, Vz):
    import oracle as O
    z = np.zeros((p["nz"], p["ny"], p["nx"]))
    return O.divergence(p, Vx, Vy, Vz, z, z, z, z, np.full_like(z, 0.01), np.ones_like(z))


@pytest.mark.parametrize("beta_n", [0.0, 10.0])
def test_momentum_exact_on_quadratic_velocity(oracle_lib, beta_n):
    """F_i = d_j tau_ij - d_i Pt for a quadratic V, uniform mu, zero old stress (Eqs. 19, 21):
    mu_e [lap V_i + (1/3 + 2 beta_n) d_i div V] - d_i Pt with mu_e = mu / (1 + xi)."""
    O = oracle_lib
    p = _grid(9, 8, 7)
    p["beta_n"] = beta_n
    rng = np.random.default_rng(3)
    dtS, mu_val = 0.013, 0.7
    g, V, (Vx, Vy, Vz), divV, divVn, mu, sh, zc = _stress_setup(p, rng, dtS, mu_val)
    told = (zc, zc, zc, np.zeros(sh["txy"]), np.zeros(sh["txz"]), np.zeros(sh["tyz"]))
    tau = O.stress(p, dtS, Vx, Vy, Vz, divV, divVn, mu, told)
    # a linear total pressure
    Xc = _mesh(g["zc"], g["yc"], g["xc"])
    gp = rng.standard_normal(3)
    Pt = gp[0] * Xc[0] + gp[1] * Xc[1] + gp[2] * Xc[2]
    F = O.momentum(p, tau, Pt, zc)
    xi = mu_val / (p["G"] * dtS)
    mue = mu_val / (1 + xi)
    H = [v.hess() for v in V]
    grad_div = np.array([H[0][0, i] + H[1][1, i] + H[2][2, i] for i in range(3)])
    for d, (Fd, pos) in enumerate(zip(F, (("zc", "yc", "xf"), ("zc", "yf", "xc"), ("zf", "yc", "xc")))):
        exact = mue * (np.trace(H[d]) + (1.0 / 3.0 + 2.0 * beta_n) * grad_div[d]) - gp[d]
        # faces whose stencil touches no boundary edge
        sl = [slice(1, -1)] * 3
        sl[2 - d] = slice(1, -1)
        Fin = Fd[tuple(sl)]
        np.testing.assert_allclose(Fin, exact, rtol=1e-9, atol=1e-9 * max(1, abs(exact)))
    # boundary faces carry no residual
    assert np.all(F[0][:, :, 0] == 0) and np.all(F[0][:, :, -1] == 0)
    assert np.all(F[2][0] == 0) and np.all(F[2][-1] == 0)


def test_buoyancy_sign_in_momentum(oracle_lib):
    """A porosity excess (lighter column) gives an upward force F_z > 0 (Eq. 19, g along -z)."""
    O = oracle_lib
    p = _grid(4, 4, 6)
    sh = I.field_shapes(4, 4, 6)
    phi = np.full(sh["centre"], 2 * p["phi0"])
    perm, rog = O.coefficients(p, phi)
    assert np.all(rog < 0)
    z = np.zeros(sh["centre"])
    tau = (z, z, z, np.zeros(sh["txy"]), np.zeros(sh["txz"]), np.zeros(sh["tyz"]))
    F = O.momentum(p, tau, z, rog)
    np.testing.assert_allclose(F[2][1:-1], -rog[0, 0, 0], rtol=1e-14)
    assert np.all(F[2][1:-1] > 0)


def test_maxwell_backward_euler_identity_and_limits(oracle_lib):
    """Eq. 21 (Eq. 5) in backward-Euler form: (tau - tau_o) / (2 G dtS) + tau / (2 mu) equals the
    deviatoric strain rate; limits G -> inf (viscous) and mu -> inf (elastic)."""
    O = oracle_lib
    p = _grid(6, 5, 7)
    rng = np.random.default_rng(4)
    dtS = 0.02
    g, V, (Vx, Vy, Vz), divV, divVn, mu, sh, zc = _stress_setup(p, rng, dtS, 0.9)
    mu = 0.5 + rng.uniform(size=sh["centre"])
    told = tuple(rng.standard_normal(sh[k]) for k in ("centre", "centre", "centre", "txy", "txz", "tyz"))
    tau = O.stress(p, dtS, Vx, Vy, Vz, divV, divVn, mu, told)
    Xc = _mesh(g["zc"], g["yc"], g["xc"])
    G = p["G"]
    for d in range(3):
        edot = V[d].grad(*Xc)[d] - divV / 3.0
        lhs = (tau[d] - told[d]) / (2 * G * dtS) + tau[d] / (2 * mu)
        np.testing.assert_allclose(lhs, edot, rtol=1e-10, atol=1e-10)
    # xy edges, interior: strain rate 1/2 (dVx/dy + dVy/dx) at the edge; edge mu = mean of 4
    Xe = _mesh(g["zc"], g["yf"], g["xf"])
    exy = 0.5 * (V[0].grad(*Xe)[1] + V[1].grad(*Xe)[0])
    mue = 0.25 * (mu[:, :-1, :-1] + mu[:, 1:, :-1] + mu[:, :-1, 1:] + mu[:, 1:, 1:])
    t = tau[3][:, 1:-1, 1:-1]
    lhs = (t - told[3][:, 1:-1, 1:-1]) / (2 * G * dtS) + t / (2 * mue)
    np.testing.assert_allclose(lhs, exy[:, 1:-1, 1:-1], rtol=1e-10, atol=1e-10)
    # boundary edges are stress free (free slip)
    assert np.all(tau[3][:, 0, :] == 0) and np.all(tau[3][:, :, -1] == 0)
    assert np.all(tau[4][0] == 0) and np.all(tau[5][:, -1, :] == 0)
    # viscous limit: G -> inf gives tau = 2 mu edot
    pv = dict(p, G=1e14)
    tv = O.stress(pv, dtS, Vx, Vy, Vz, divV, divVn, mu, told)
    np.testing.assert_allclose(tv[0], 2 * mu * (V[0].grad(*Xc)[0] - divV / 3), rtol=1e-9, atol=1e-9)
    # elastic limit: mu -> inf gives tau = tau_o + 2 G dtS edot
    big = np.full(sh["centre"], 1e14)
    te = O.stress(p, dtS, Vx, Vy, Vz, divV, divVn, big, told)
    np.testing.assert_allclose(te[1], told[1] + 2 * G * dtS * (V[1].grad(*Xc)[1] - divV / 3),
                               rtol=1e-9, atol=1e-9)


def test_advection_log_form_exact_on_linear_porosity(oracle_lib):
    """V . grad log(1 - phi) for (1 - phi) linear and uniform interior face velocities."""
    O = oracle_lib
    p = _grid(8, 7, 6)
    g = _coords(p)
    sh = I.field_shapes(8, 7, 6)
    Xc = _mesh(g["zc"], g["yc"], g["xc"])
    b = np.array([0.003, -0.002, 0.004])
    omp = 0.98 + b[0] * Xc[0] + b[1] * Xc[1] + b[2] * Xc[2]
    phi = 1 - omp
    v = np.array([0.3, -0.7, 1.1])
    Vx = np.full(sh["Vx"], v[0]); Vy = np.full(sh["Vy"], v[1]); Vz = np.full(sh["Vz"], v[2])
    adv = O.advection(p, Vx, Vy, Vz, phi)
    exact = (v @ b) / omp
    inner = (slice(1, -1),) * 3
    np.testing.assert_allclose(adv[inner], exact[inner], rtol=1e-12)


def test_tau_II_and_power_law_target_simple_shear(oracle_lib):
    """Simple shear Vx = gamma (y - ly/2): tau_xy = 2 mu_e edot_xy = mu_e gamma on interior
    edges, tau_II = |tau_xy| at centres away from the y-walls; the Picard target is Eq. 24."""
    O = oracle_lib
    p = _grid(6, 8, 5)
    p["tau0"] = 0.01
    g = _coords(p)
    sh = I.field_shapes(6, 8, 5)
    gamma = 0.37
    X, Y, Z = _mesh(g["zc"], g["yc"], g["xf"])
    Vx = gamma * (Y - p["ly"] / 2)
    Vy, Vz = np.zeros(sh["Vy"]), np.zeros(sh["Vz"])
    phi = np.full(sh["centre"], p["phi0"])
    st = O.make_state(p, phi, fields=dict(Vx=Vx))
    O.begin_step(st)
    mu0 = p["mu0"]
    xi = mu0 / (p["G"] * st.dtS)
    assert abs(xi - p["xsi_w"]) < 1e-15              # dtS makes the largest xi equal xsi_w
    r = O.system_residual(st)
    tII = mu0 / (1 + xi) * gamma
    mus = mu0 / (1 + (tII / p["tau0"]) ** (p["n_pow"] - 1))
    inner = (slice(None), slice(1, -1), slice(1, -1))
    np.testing.assert_allclose(r["mu"][inner], np.log(mu0) - np.log(mus), rtol=1e-12)


def test_bulk_viscosity_target_and_weakening(oracle_lib):
    """Eqs. 25-26: eta* = eta0 mu / phi, times R_weak where Pf > Pt (tie -> no weakening)."""
    O = oracle_lib
    p = _grid(4, 3, 5)
    sh = I.field_shapes(4, 3, 5)
    rng = np.random.default_rng(5)
    phi = p["phi0"] * (1 + rng.uniform(size=sh["centre"]))
    Pt = rng.standard_normal(sh["centre"]) * 1e-3
    Pf = Pt + rng.choice([-1.0, 0.0, 1.0], size=sh["centre"]) * 1e-4
    st = O.make_state(p, phi, fields=dict(Pt=Pt, Pf=Pf))
    O.begin_step(st)
    r = O.system_residual(st)
    R = np.where(Pf > Pt, p["R_weak"], 1.0)
    np.testing.assert_allclose(r["eta"], np.log(st["eta"]) - np.log(p["eta0"] * st["mu"] / phi * R),
                               rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(st["eta"], p["eta0"] * p["mu0"] / phi, rtol=1e-15)
