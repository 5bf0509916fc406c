"""Mixed precision (PT_FP32): FP32 PT iterations on the correction of an FP64 defect-correction
loop must reach the FP64 tolerance and the FP64 oracle's solution (porosity bar 1e-5 relative)."""
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


@pytest.mark.parametrize("dims", [(32, 32, 32), (24, 20, 28)])
def test_fp32_step_reaches_fp64_solution(dims):
    PTSolver = _solver()
    p = I.c1_params(*dims)
    p["precision"] = 1
    phi = I.gaussian_porosity(p)
    s = PTSolver(p, phi)
    rep = s.step()
    assert rep["status"] == 0, rep
    assert max(rep["r_v"], rep["r_pt"], rep["r_pf"], rep["r_pic"]) < p["tol"]
    st = O.make_state(dict(p, precision=0), phi)
    rc, iters, res = O.step(st)
    assert rc == 0
    e_phi = rel(s.get("phi"), st["phi"])
    assert e_phi <= PHI_TOL, e_phi
    # both are converged to the same residual tolerance: the other fields agree closely too
    for name in ("Pt", "Pf", "Vz"):
        assert rel(s.get(name), st[name]) <= 1e-4, name
    s.close()


def test_fp32_fixed_iterations_reduce_the_fp64_residual():
    """One outer iteration with 300 FP32 correction iterations lowers the FP64 residual."""
    PTSolver = _solver()
    p = I.c1_params(40, 36, 33)
    p["precision"] = 1
    s = PTSolver(p, I.gaussian_porosity(p))
    s.step_begin()
    r0 = s.iterate(0, 300)
    r1 = s.iterate(300, 300)
    m0 = max(r0["r_v"], r0["r_pt"], r0["r_pf"])
    m1 = max(r1["r_v"], r1["r_pt"], r1["r_pf"])
    assert np.isfinite(m1) and m1 < 0.5 * m0, (m0, m1)
    s.close()
