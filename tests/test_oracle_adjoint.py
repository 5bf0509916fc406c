"""CPU adjoint (oracle side): its residual is the C oracle's residual, and its gradient of
J = sum (phi^N - phi_target)^2 w.r.t. the log-permeability field matches central finite
differences of the C oracle's converged forward runs."""
import numpy as np
import pytest

import oracle as O
import pt_inputs as I

torch = pytest.importorskip("torch")


def _setup(n=(6, 5, 7), seed=0):
    from oracle import adjoint as A
    p = A.adjoint_params(I.c1_params(*n))
    rng = np.random.default_rng(seed)
    phi = I.gaussian_porosity(p, centres=((0.45, 0.55, 0.5),), width=0.3)
    theta = 0.3 * rng.standard_normal(phi.shape)
    return A, p, phi, theta, rng


def test_torch_residual_equals_c_oracle_residual():
    A, p, phi, theta, rng = _setup()
    rs = I.random_state(p, seed=4, scale=1e-3)
    fields = {k: v for k, v in rs.items() if k in ("Vx", "Vy", "Vz", "Pt", "Pf")}
    st = O.make_state(p, rs["phi"], logk=theta, fields=fields)
    O.begin_step(st)
    st["eta"][...] = p["eta0"] * p["mu0"] / st["phi"]         # converged Picard state in scope
    for k in ("txxo", "tyyo", "tzzo", "txyo", "txzo", "tyzo"):
        st[k][...] = 0.0
    st.dtS = p["mu0"] / (p["G"] * p["xsi_w"])
    r = O.system_residual(st)
    u = A.state_u(st)
    old = dict(Pto=A._t(st["Pto"]), Pfo=A._t(st["Pfo"]), Lo=A._t(st["Lo"]))
    F = A.residual(p, u, old, A._t(theta))
    pairs = [("Fx", r["Vx"][:, :, 1:-1]), ("Fy", r["Vy"][:, 1:-1, :]), ("Fz", r["Vz"][1:-1]),
             ("Fpt", r["pt"]), ("Fpf", r["pf"]), ("FL", r["L"])]
    for k, ref in pairs:
        got = F[k].numpy()
        np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12 * max(1.0, np.abs(ref).max()), err_msg=k)


@pytest.mark.slow
def test_adjoint_gradient_matches_finite_differences():
    A, p, phi, theta, rng = _setup()
    N = 3
    tgt_theta = theta + 0.5 * rng.standard_normal(theta.shape)
    target = A.forward(p, phi, tgt_theta, N)[-1]["phi"]
    states = A.forward(p, phi, theta, N)
    assert p["dt"] * N < p["mu0"] / (p["G"] * p["xsi_w"])     # no old-stress refresh in the window
    grad = A.gradient(p, states, theta, target)
    assert np.abs(grad).max() > 0
    for d in range(3):
        v = rng.standard_normal(theta.shape)
        eps = 1e-5
        Jp = A.misfit(A.forward(p, phi, theta + eps * v, N)[-1]["phi"], target)
        Jm = A.misfit(A.forward(p, phi, theta - eps * v, N)[-1]["phi"], target)
        fd = (Jp - Jm) / (2 * eps)
        ad = float(np.sum(grad * v))
        assert abs(ad - fd) <= 1e-4 * abs(fd), (d, ad, fd)


def _setup_pl(n=(6, 5, 7), seed=0):
    """Power law on (Eq. 24, n = 3, tau0 = 0.04 as in the benchmark): over the first steps from
    rest mu falls to 0.1-0.3 mu0 on this grid, so the Picard row is far from trivial."""
    from oracle import adjoint as A
    p = A.adjoint_params(I.c1_params(*n), powerlaw=True)
    rng = np.random.default_rng(seed)
    phi = I.gaussian_porosity(p, centres=((0.45, 0.55, 0.5),), width=0.3)
    theta = 0.3 * rng.standard_normal(phi.shape)
    return A, p, phi, theta, rng


def test_torch_residual_with_power_law_equals_c_oracle_residual():
    """With mu an unknown: the momentum, pressure and porosity rows use the moduli
    2 mu/(1+xi) at centres and edges and eta = eta0 mu / phi; the Picard row is
    log mu - log mu*(tau_II); xi = mu / (G dtS) with dtS = max(mu_prev) / (G xsi_w)."""
    A, p, phi, theta, rng = _setup_pl()
    rs = I.random_state(p, seed=6, scale=1e-2)
    fields = {k: v for k, v in rs.items() if k in ("Vx", "Vy", "Vz", "Pt", "Pf")}
    st = O.make_state(p, rs["phi"], logk=theta, fields=fields)
    O.begin_step(st)
    mu = p["mu0"] * (0.3 + 0.7 * rng.uniform(size=st["mu"].shape))
    mu_prev = p["mu0"] * (0.5 + 0.5 * rng.uniform(size=st["mu"].shape))
    st["mu"][...] = mu
    st["eta"][...] = p["eta0"] * mu / st["phi"]               # eta at its fixed point (R = 1)
    for k in ("txxo", "tyyo", "tzzo", "txyo", "txzo", "tyzo"):
        st[k][...] = 0.0
    st.dtS = mu_prev.max() / (p["G"] * p["xsi_w"])
    r = O.system_residual(st)
    assert np.abs(r["eta"]).max() < 1e-13
    u = A.state_u(st)
    old = dict(Pto=A._t(st["Pto"]), Pfo=A._t(st["Pfo"]), Lo=A._t(st["Lo"]), mu_o=A._t(mu_prev))
    F = A.residual(p, u, old, A._t(theta))
    pairs = [("Fx", r["Vx"][:, :, 1:-1]), ("Fy", r["Vy"][:, 1:-1, :]), ("Fz", r["Vz"][1:-1]),
             ("Fpt", r["pt"]), ("Fpf", r["pf"]), ("FL", r["L"]), ("Fmu", r["mu"])]
    for k, ref in pairs:
        got = F[k].numpy()
        np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12 * max(1.0, np.abs(ref).max()), err_msg=k)
    assert np.abs(r["mu"]).max() > 0.1                       # the power law is far from inactive


@pytest.mark.slow
def test_adjoint_gradient_with_power_law_matches_finite_differences():
    A, p, phi, theta, rng = _setup_pl()
    N = 3
    tgt_theta = theta + 0.5 * rng.standard_normal(theta.shape)
    target = A.forward(p, phi, tgt_theta, N)[-1]["phi"]
    states = A.forward(p, phi, theta, N)
    mus = [s["mu"] for s in states[1:]]
    assert min(m.min() for m in mus) < 0.9 * p["mu0"]          # the power law acts
    # no old-stress refresh inside the window: accumulated time stays below every step's dtS
    assert (N - 1) * p["dt"] < min(m.max() for m in [states[0]["mu"]] + mus[:-1]) / (p["G"] * p["xsi_w"])
    grad = A.gradient(p, states, theta, target)
    assert np.abs(grad).max() > 0
    for d in range(3):
        v = rng.standard_normal(theta.shape)
        eps = 1e-5
        Jp = A.misfit(A.forward(p, phi, theta + eps * v, N)[-1]["phi"], target)
        Jm = A.misfit(A.forward(p, phi, theta - eps * v, N)[-1]["phi"], target)
        fd = (Jp - Jm) / (2 * eps)
        ad = float(np.sum(grad * v))
        assert abs(ad - fd) <= 1e-4 * abs(fd), (d, ad, fd)
