"""The background-shear workload (thesis Art. 1 Section 3.1, Eqs. 32-33; Table 2 scaled down)
on the GPU against the FP64 oracle: same iteration count -> fields within 1e-10 (max-rel,
normwise), for the FP64-lean, step-by-step and double-float forms, over two physical steps (the second uses
the old stresses of the first, wall edges included); the mixed-precision form's converged step
within the porosity bar 1e-5, with plain and with multigrid correction solves; the sub-domain
form bitwise equal to the undivided grid."""
import numpy as np
import pytest

import oracle as O
import pt_inputs as I

pytestmark = pytest.mark.gpu

FIELDS = ("Vx", "Vy", "Vz", "Pt", "Pf", "phi", "mu", "eta", "txy")


def _solver():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_08716_gb300.solver import PTSolver
    return PTSolver


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("mode", (0, 2, 3))
@pytest.mark.parametrize("dims, niter", [((16, 14, 24), 450), ((9, 11, 13), 300)])
def test_shear_iterations_match_oracle(dims, niter, mode):
    PTSolver = _solver()
    p = I.shear_params(*dims, dt=2e-3)   # dt > dtS: step 2 refreshes the old stresses (walls too)
    p["precision"] = mode
    phi = I.ellipsoid_porosity(p, centre=(0.45, 0.52, 0.3), axes=(14.0, 12.0, 9.0))
    s = PTSolver(p, phi)
    st = O.make_state(p, phi)
    for step in range(2):
        s.step_begin()
        s.iterate(0, niter)
        s.step_end()
        O.begin_step(st)
        rc, res = O.iterate_n(st, 0, niter)
        O.end_step(st)
        assert rc == 0
        errs = {n: rel(s.get(n), st[n]) for n in FIELDS}
        assert max(errs.values()) <= 1e-10, (step, errs)
    assert np.abs(st["txy"][:, 0, 1:-1]).min() > 0        # the walls carry the background stress
    s.close()


def test_shear_mixed_precision_step_matches_oracle():
    PTSolver = _solver()
    p = I.shear_params(12, 12, 20)
    p["tol"] = 1e-8
    phi = I.ellipsoid_porosity(p, centre=(0.5, 0.5, 0.3), axes=(14.0, 14.0, 8.0))
    st = O.make_state(p, phi)
    rc, iters, res = O.step(st)
    assert rc == 0, res
    q = dict(p, precision=1)
    s = PTSolver(q, phi)
    r = s.step(raise_on_notconv=True)
    assert r["status"] == 0
    assert rel(s.get("phi"), st["phi"]) <= 1e-5
    s.close()


def test_shear_multigrid_step_matches_oracle():
    """The background strain rate enters the FP64 residuals only: multigrid correction solves
    (three levels, 12 x 12 x 20 -> 6 x 6 x 10 -> 3 x 3 x 5) reach the oracle's converged step."""
    PTSolver = _solver()
    p = I.shear_params(12, 12, 20)
    p["tol"] = 1e-8
    phi = I.ellipsoid_porosity(p, centre=(0.5, 0.5, 0.3), axes=(14.0, 14.0, 8.0))
    st = O.make_state(p, phi)
    rc, iters, res = O.step(st)
    assert rc == 0, res
    s = PTSolver(dict(p, precision=1, mg_levels=3), phi)
    r = s.step(raise_on_notconv=True)
    assert r["status"] == 0
    assert rel(s.get("phi"), st["phi"]) <= 1e-5
    for name in ("Pt", "Pf", "Vx"):
        assert rel(s.get(name), st[name]) <= 1e-4, name
    s.close()


def test_shear_decomposed_equals_undivided_bitwise():
    _solver()
    from paper_2207_08716_gb300.solver import PTDomains
    p = I.shear_params(20, 18, 24)
    p["max_iter"] = 450
    phi = I.ellipsoid_porosity(p, centre=(0.45, 0.5, 0.3), axes=(14.0, 14.0, 9.0))
    out = []
    for parts in ((1, 1, 1), (2, 1, 2)):
        d = PTDomains(p, phi, parts=parts)
        reps = [d.step() for _ in range(2)]
        d.gather()
        out.append((reps, {k: d.get(k) for k in FIELDS}))
        d.close()
    assert out[0][0] == out[1][0]
    for k in FIELDS:
        np.testing.assert_array_equal(out[1][1][k], out[0][1][k], err_msg=k)
