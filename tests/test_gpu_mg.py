"""Multigrid-accelerated FP32 correction solves (pt_num.mg_levels >= 2; each grid ceil(n / 2) cells
per direction of the one above, nested for even n, not nested for odd n): each correction problem
of the FP32 + FP64 defect-correction step is solved by geometric-multigrid V-cycles smoothed by
the PT sweep instead of plain PT iterations. The outer FP64 loop, its residuals and its fixed
point are unchanged, so a converged step must reach the FP64 oracle's converged step within the
FP32 form's porosity bar (1e-5 relative) and agree with the plain FP32 form's converged step; the
V-cycles must need fewer finest-grid sweeps than the plain iteration needs iterations."""
import numpy as np
import pytest

import oracle as O
import pt_inputs as I

pytestmark = pytest.mark.gpu

PHI_TOL = 1e-5          # stated porosity error bar of the mixed-precision form


def _solver():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_08716_gb300.solver import PTSolver
    return PTSolver


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("dims, levels", [((32, 32, 32), 3), ((32, 24, 40), 4), ((16, 16, 16), 2),
                                          ((33, 27, 41), 3), ((31, 31, 31), 4)])
def test_multigrid_step_reaches_the_oracle_solution(dims, levels):
    PTSolver = _solver()
    p = I.c1_params(*dims)
    p.update(precision=1, mg_levels=levels)
    phi = I.gaussian_porosity(p)
    s = PTSolver(p, phi)
    rep = s.step()
    assert rep["status"] == 0, rep
    assert max(rep["r_v"], rep["r_pt"], rep["r_pf"], rep["r_pic"]) < p["tol"]
    st = O.make_state(dict(p, precision=0, mg_levels=0), phi)
    rc, _, _ = O.step(st)
    assert rc == 0
    e_phi = rel(s.get("phi"), st["phi"])
    assert e_phi <= PHI_TOL, e_phi
    for name in ("Pt", "Pf", "Vz"):
        assert rel(s.get(name), st[name]) <= 1e-4, name
    s.close()


@pytest.mark.parametrize("levels", (0, 3))
def test_fp32_step_with_heterogeneous_permeability_reaches_the_oracle_solution(levels):
    """A log-permeability prefactor field (k = k0 e^logk (phi/phi0)^3, Eq. 23; a Gaussian random
    field of standard deviation 0.5, k varying over a factor ~10) and an off-centre anomaly: the
    plain and the multigrid correction solves (coarse k the covered-fraction mean) reach the
    oracle's converged step."""
    PTSolver = _solver()
    p = I.c1_params(24, 20, 28)
    phi = I.gaussian_porosity(p, centres=((0.45, 0.55, 0.4),))
    logk = I.gaussian_random_field((28, 20, 24), seed=4, corr_len=0.15, std=0.5)
    st = O.make_state(p, phi, logk=logk)
    rc, _, _ = O.step(st)
    assert rc == 0
    s = PTSolver(dict(p, precision=1, mg_levels=levels, max_iter=200000), phi, logk=logk)
    rep = s.step()
    assert rep["status"] == 0, rep
    assert rel(s.get("phi"), st["phi"]) <= PHI_TOL
    for name in ("Pt", "Pf", "Vz"):
        assert rel(s.get(name), st[name]) <= 1e-4, name
    s.close()


def test_multigrid_and_plain_fp32_steps_agree_and_multigrid_sweeps_less():
    PTSolver = _solver()
    p = I.c1_params(64)
    p.update(precision=1, max_iter=200000)
    phi = I.gaussian_porosity(p)
    plain = PTSolver(p, phi)
    rp = plain.step()
    mg = PTSolver(dict(p, mg_levels=5), phi)
    rm = mg.step()
    assert rp["status"] == 0 and rm["status"] == 0, (rp, rm)
    assert rel(mg.get("phi"), plain.get("phi")) <= PHI_TOL
    assert rm["iters"] < rp["iters"], (rm["iters"], rp["iters"])
    plain.close()
    mg.close()


def test_multigrid_two_steps_carry_the_state():
    """Two converged steps (old stresses, stress sub-step, damped residual carried between them)
    against the oracle's two steps."""
    PTSolver = _solver()
    p = I.c1_params(16, 16, 32)
    p.update(precision=1, mg_levels=3)
    phi = I.gaussian_porosity(p)
    s = PTSolver(p, phi)
    for _ in range(2):
        assert s.step()["status"] == 0
    st = O.make_state(dict(p, precision=0, mg_levels=0), phi)
    for _ in range(2):
        assert O.step(st)[0] == 0
    assert rel(s.get("phi"), st["phi"]) <= PHI_TOL
    s.close()
