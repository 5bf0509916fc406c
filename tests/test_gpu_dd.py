"""Sub-domain (halo-exchange) form: the grid split into parts that exchange one-cell halos
after every PT iteration gives bitwise the result of the undivided grid run by the same
kernels (the thesis's claim for its multi-GPU decomposition, Art. 2), for even and uneven
splits, with and without a log-permeability field; and the single-instance FP64-lean solver's
result to 1e-12 (different kernels, same arithmetic up to multiply-add fusion)."""
import numpy as np
import pytest

import pt_inputs as I

pytestmark = pytest.mark.gpu

FIELDS = ("Vx", "Vy", "Vz", "Pt", "Pf", "phi", "txx", "tyy", "tzz", "txy", "txz", "tyz", "mu", "eta")


def _torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _run(p, phi, parts, logk, nsteps):
    from paper_2207_08716_gb300.solver import PTDomains
    d = PTDomains(p, phi, parts=parts, logk=logk)
    reps = [d.step() for _ in range(nsteps)]
    d.gather()
    out = {k: d.get(k) for k in FIELDS}
    d.close()
    return reps, out


@pytest.mark.parametrize("parts", [(2, 2, 2), (3, 1, 2), (1, 4, 1)])
def test_decomposed_equals_undivided_bitwise(parts):
    _torch()
    dims = (26, 20, 18)
    p = I.c1_params(*dims)
    p["max_iter"] = 600                    # a fixed iteration budget (the cap) per step
    phi = I.gaussian_porosity(p, centres=((0.42, 0.55, 0.47),), width=0.15)
    logk = I.gaussian_random_field(phi.shape, seed=9, corr_len=0.15, std=0.4)
    ref_reps, ref = _run(p, phi, (1, 1, 1), logk, 2)
    reps, got = _run(p, phi, parts, logk, 2)
    for a, b in zip(reps, ref_reps):
        assert a == b, (a, b)
    for k in FIELDS:
        np.testing.assert_array_equal(got[k], ref[k], err_msg=k)


def test_decomposed_converged_step_matches_single_solver():
    _torch()
    from paper_2207_08716_gb300.solver import PTSolver
    dims = (24, 20, 16)
    p = I.c1_params(*dims)
    phi = I.gaussian_porosity(p, centres=((0.5, 0.45, 0.5),), width=0.15)
    reps, got = _run(p, phi, (2, 2, 2), None, 1)
    assert reps[0]["status"] == 0, reps
    s = PTSolver(p, phi)
    r = s.step()
    assert r["iters"] == reps[0]["iters"], (r, reps)
    for k in FIELDS:
        ref = s.get(k)
        err = np.abs(got[k] - ref).max() / max(np.abs(ref).max(), 1e-300)
        assert err <= 1e-12, (k, err)
    s.close()
