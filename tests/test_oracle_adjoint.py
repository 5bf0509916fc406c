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
