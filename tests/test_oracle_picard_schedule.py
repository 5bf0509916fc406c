"""Pins of the oracle's Picard relaxation (Eqs. 24-26 with log-space relaxation) and of its
elastic stress sub-step schedule (the appendix two-phase script's dtS / dt_cum rule).

* One Picard update on a uniform state whose stresses are known in closed form gives
  mu1 = mu*^r_mu mu^(1 - r_mu) and eta1 = eta*^r_eta eta^(1 - r_eta), eta* = eta0 mu1 / phi1 R:
  swapping r and 1 - r, relaxing in linear space, or building eta* from the unrelaxed mu fails.
* With mu* fixed (power law off) repeated updates contract log(mu / mu*) by exactly (1 - r_mu)
  per update.
* The old stresses are refreshed at the first step and then exactly on the steps whose
  accumulated time since the last refresh has reached dtS = max(mu) / (G xsi_w) (a tie
  included), and the accumulated time restarts there.
"""
import numpy as np
import pytest

import pt_inputs as I


def _uniform_state(O, p, mu_a, eta_a, tau_o, Pt=0.0, Pf=0.0, phi=0.02):
    sh = I.field_shapes(p["nx"], p["ny"], p["nz"])
    c = sh["centre"]
    fields = dict(mu=np.full(c, mu_a), eta=np.full(c, eta_a), Pt=np.full(c, Pt), Pf=np.full(c, Pf),
                  txx=np.full(c, tau_o[0]), tyy=np.full(c, tau_o[1]), tzz=np.full(c, tau_o[2]))
    return O.make_state(p, np.full(c, phi), fields=fields, init_visc=False)


def _params(**over):
    p = I.c1_params(5, 4, 6)
    # equal densities: a uniform state has no buoyancy and no Darcy flux, V stays zero
    p.update(rhos_g=1.0, rhof_g=1.0, beta_n=0.0, rel_mu=0.1, rel_eta=0.3, tau0=0.04)
    p.update(over)
    return p


@pytest.mark.parametrize("Pf, rel_mu", [(0.0, 0.1), (2e-3, 0.1), (0.0, 0.7)])
def test_one_picard_update_is_log_space_relaxation(oracle_lib, Pf, rel_mu):
    O = oracle_lib
    p = _params(rel_mu=rel_mu)
    mu_a, eta_a = 1.7, 123.0
    tau_o = (0.03, -0.01, -0.02)
    st = _uniform_state(O, p, mu_a, eta_a, tau_o, Pf=Pf)
    O.begin_step(st)                     # first step: tau_o = tau, dtS = mu_a / (G xsi_w)
    xi = mu_a / (p["G"] * st.dtS)
    assert abs(xi - p["xsi_w"]) < 1e-14
    rc, res = O.iteration(st, p["nup"])  # iteration number nup: the Picard update runs
    assert rc == 0 and res is not None
    # V = 0, beta_n = 0: the Maxwell step (Eq. 21) leaves tau = tau_o xi / (1 + xi)
    tau = np.array(tau_o) * xi / (1.0 + xi)
    tII = np.sqrt(0.5 * np.sum(tau ** 2))
    mus = p["mu0"] / (1.0 + (tII / p["tau0"]) ** (p["n_pow"] - 1.0))        # Eq. 24
    mu1 = mus ** rel_mu * mu_a ** (1.0 - rel_mu)
    for n in ("Vx", "Vy", "Vz"):
        assert np.all(st[n] == 0.0)
    for n in ("Pt", "Pf", "phi"):
        assert np.ptp(st[n]) == 0.0
    Pt1, Pf1, phi1 = st["Pt"].flat[0], st["Pf"].flat[0], st["phi"].flat[0]
    R = p["R_weak"] if Pf1 > Pt1 else 1.0                                      # Eq. 25
    etas = p["eta0"] * mu1 / phi1 * R                                          # Eq. 26
    eta1 = etas ** p["rel_eta"] * eta_a ** (1.0 - p["rel_eta"])
    np.testing.assert_allclose(st["mu"], mu1, rtol=1e-13)
    np.testing.assert_allclose(st["eta"], eta1, rtol=1e-13)
    assert (R < 1.0) == (Pf > 0)
    # the mistakes this pins: r <-> 1 - r, relaxation in linear space, eta* from the old mu
    assert abs(mus ** (1 - rel_mu) * mu_a ** rel_mu - mu1) > 1e-3 * mu1
    assert abs(rel_mu * mus + (1 - rel_mu) * mu_a - mu1) > 1e-4 * mu1
    eta_wrong = (p["eta0"] * mu_a / phi1 * R) ** p["rel_eta"] * eta_a ** (1.0 - p["rel_eta"])
    assert abs(eta_wrong - eta1) > 1e-3 * eta1
    # the reported Picard change is the unrelaxed log distance (Eqs. 24, 26 residual)
    want = max(abs(np.log(mus) - np.log(mu_a)), abs(np.log(etas) - np.log(eta_a)))
    assert abs(res["r_pic"] - want) <= 1e-13 * want


def test_repeated_picard_updates_contract_by_one_minus_r(oracle_lib):
    """Power law off, so mu* = mu0 at every update: after m updates
    log(mu_m / mu0) = (1 - r_mu)^m log(mu_a / mu0)."""
    O = oracle_lib
    p = _params(powerlaw_on=0, rel_mu=0.25, mu0=1.3)
    mu_a = 4.0
    st = _uniform_state(O, p, mu_a, 50.0, (0.0, 0.0, 0.0))
    O.begin_step(st)
    for m in range(1, 5):
        for it in range((m - 1) * p["nup"] + 1, m * p["nup"] + 1):
            rc, _ = O.iteration(st, it)
            assert rc == 0
        want = p["mu0"] * np.exp((1 - p["rel_mu"]) ** m * np.log(mu_a / p["mu0"]))
        np.testing.assert_allclose(st["mu"], want, rtol=1e-13)


def _refresh_steps(nsteps, dt, dtS):
    """Steps (1-based) whose start refreshes the old stresses: the first one, then each step at
    whose start the time accumulated since the last refresh has reached dtS."""
    out, since = [], 0.0
    for s in range(1, nsteps + 1):
        if s == 1 or since >= dtS:
            out.append(s)
            since = 0.0
        since += dt
    return out


@pytest.mark.parametrize("dt, want", [(0.25, [1, 5, 9]), (0.3, [1, 5, 9]), (0.4, [1, 4, 7, 10])])
def test_old_stress_refresh_schedule(oracle_lib, dt, want):
    """mu stays exactly mu0 = 1 (power law off; log-space relaxation of log 1 = 0), so
    dtS = 1 / (G xsi_w) = 1 with G = xsi_w = 1. dt = 0.25 makes the accumulated time hit dtS
    exactly on the 5th step (a tie, refreshed: the rule is 'reached', not 'exceeded');
    dt = 0.3 passes it there, dt = 0.4 on the 4th."""
    O = oracle_lib
    p = I.c1_params(6, 5, 7)
    p.update(powerlaw_on=0, G=1.0, xsi_w=1.0, dt=dt, mu0=1.0)
    rs = I.random_state(p, seed=11, scale=1e-3)
    st = O.make_state(p, rs["phi"], fields={k: v for k, v in rs.items() if k != "phi"})
    nsteps = 10
    assert _refresh_steps(nsteps, dt, 1.0) == want
    got = []
    last_end = {n: st[n].copy() for n in ("txx", "tyy", "tzz", "txy", "txz", "tyz")}
    kept = None
    for s in range(1, nsteps + 1):
        O.begin_step(st)
        assert st.dtS == 1.0
        refreshed = all(np.array_equal(st[n + "o"], last_end[n]) for n in last_end)
        if refreshed:
            got.append(s)
            assert st.dt_cum == 0.0
            kept = {n: st[n + "o"].copy() for n in last_end}
        else:
            for n in last_end:                    # the old stresses of the last refresh stay
                np.testing.assert_array_equal(st[n + "o"], kept[n])
        rc, _ = O.iterate_n(st, 0, 2)
        assert rc == 0
        O.end_step(st)
        for n in last_end:
            assert not np.array_equal(st[n], last_end[n])      # the stresses moved this step
            last_end[n] = st[n].copy()
    assert got == want, (got, want)
