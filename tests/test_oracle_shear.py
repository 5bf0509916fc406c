"""Oracle pins for the applied background shear (thesis Art. 1 Eqs. 32-33, Section 3.1): the
background flow V_bg = (tau_bg/mu0)(y - ly/2) e_x enters the xy strain rate only.

* A uniform state (phi = phi0, equal densities: no buoyancy) under background shear is a
  rest state: the unknown velocity
  stays zero and every xy-edge, the wall edges included, carries the Maxwell stress of the
  background strain rate, tau_xy = 2 mu (tau_bg / (2 mu0)) / (1 + xi) (Eq. 21, closed form).
* With the power law on, the converged uniform viscosity is the root of the scalar fixed point
  mu = mu0 / (1 + (tau_xy(mu) / tau0)^(n-1)) (Eq. 24), solved here by bracketing.
* A centred anomaly under background shear gives a solution invariant under the half turn
  about the vertical axis through the box centre (V_x, V_y odd; V_z, pressures, phi, tau_xy even).
"""
import numpy as np
import pytest

import oracle as O
import pt_inputs as I


def _uniform(p):
    return np.full((p["nz"], p["ny"], p["nx"]), p["phi0"])


@pytest.mark.parametrize("tau_bg", [1.0, -0.3])
def test_uniform_background_shear_is_a_rest_state_with_the_maxwell_stress(tau_bg):
    p = I.shear_params(6, 5, 8)
    p.update(powerlaw_on=0, tau_bg=tau_bg, tol=1e-12, max_iter=200000, rhos_g=1.0, rhof_g=1.0)
    st = O.make_state(p, _uniform(p))
    rc, iters, res = O.step(st)
    assert rc == 0, (iters, res)
    for k in ("Vx", "Vy", "Vz", "Pt", "Pf"):
        assert np.abs(st[k]).max() <= 1e-12, k
    # first step: dtS = mu0 / (G xsi_w), so xi = mu / (G dtS) = xsi_w = 1
    expect = 2.0 * p["mu0"] * (tau_bg / (2.0 * p["mu0"])) / (1.0 + p["xsi_w"])
    np.testing.assert_allclose(st["txy"], expect, rtol=1e-13, atol=0)   # every edge, walls included
    assert np.abs(st["txz"]).max() == 0.0 and np.abs(st["tyz"]).max() == 0.0


def test_power_law_viscosity_under_background_shear_is_the_scalar_fixed_point():
    scipy = pytest.importorskip("scipy.optimize")
    p = I.shear_params(5, 4, 6)
    p.update(tol=1e-12, max_iter=400000, rhos_g=1.0, rhof_g=1.0)
    st = O.make_state(p, _uniform(p))
    rc, iters, res = O.step(st)
    assert rc == 0, (iters, res)
    mu0, tau_bg, tau0, n = p["mu0"], p["tau_bg"], p["tau0"], p["n_pow"]

    def tau_xy(mu):                      # xi = mu / (G dtS) = mu / mu0 at the first step
        return 2.0 * mu * (tau_bg / (2.0 * mu0)) / (1.0 + mu / mu0)

    root = scipy.brentq(lambda m: m - mu0 / (1.0 + (abs(tau_xy(m)) / tau0) ** (n - 1.0)), 1e-8, mu0)
    np.testing.assert_allclose(st["mu"], root, rtol=1e-9)
    np.testing.assert_allclose(st["txy"], tau_xy(st["mu"].mean()), rtol=1e-9)
    assert np.abs(st["Vx"]).max() <= 1e-11


def test_centred_anomaly_under_background_shear_has_half_turn_symmetry():
    p = I.shear_params(10, 10, 12)
    p.update(max_iter=200000)
    phi = I.ellipsoid_porosity(p, centre=(0.5, 0.5, 0.4), axes=(14.0, 14.0, 14.0))
    st = O.make_state(p, phi)
    rc, iters, res = O.step(st)
    assert rc == 0, (iters, res)
    turn = lambda a: a[:, ::-1, ::-1]
    scale = {k: max(np.abs(st[k]).max(), 1e-30) for k in ("Vx", "Vy", "Vz", "Pt", "Pf", "txy")}
    assert scale["Vx"] > 1e-3 and scale["Vz"] > 1e-3          # the anomaly drives a flow
    np.testing.assert_allclose(st["Vx"], -turn(st["Vx"]), rtol=0, atol=1e-11 * scale["Vx"])
    np.testing.assert_allclose(st["Vy"], -turn(st["Vy"]), rtol=0, atol=1e-11 * scale["Vy"])
    for k in ("Vz", "Pt", "Pf", "txy"):
        np.testing.assert_allclose(st[k], turn(st[k]), rtol=0, atol=1e-11 * scale[k], err_msg=k)
    np.testing.assert_allclose(st["phi"], turn(st["phi"]), rtol=1e-13, atol=0)
