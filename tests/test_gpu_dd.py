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


@pytest.mark.parametrize("parts", [(2, 2, 2), (3, 1, 2)])
def test_decomposed_matches_oracle_after_fixed_iterations(parts):
    """Against the FP64 oracle itself (not the undivided GPU run): two physical steps capped at
    a fixed iteration count (not converged, so both sides take exactly the cap), with a
    log-permeability field; all 14 fields within the FP64 parity bar 1e-10."""
    _torch()
    import oracle as O
    dims = (26, 20, 18)
    p = I.c1_params(*dims)
    p["max_iter"] = 240
    phi = I.gaussian_porosity(p, centres=((0.42, 0.55, 0.47),), width=0.15)
    logk = I.gaussian_random_field(phi.shape, seed=9, corr_len=0.15, std=0.4)
    reps, got = _run(p, phi, parts, logk, 2)
    st = O.make_state(p, phi, logk=logk)
    for s in range(2):
        rc, iters, res = O.step(st)
        assert rc == -2 and iters == p["max_iter"], (rc, iters)       # capped, like the GPU run
        assert reps[s]["status"] == -2 and reps[s]["iters"] == iters, reps[s]
        for k in ("r_v", "r_pt", "r_pf", "r_pic"):
            assert abs(reps[s][k] - res[k]) <= 1e-8 * abs(res[k]) + 1e-14, (s, k, reps[s][k], res[k])
    for k in FIELDS:
        err = np.abs(got[k] - st[k]).max() / max(np.abs(st[k]).max(), 1e-300)
        assert err <= 1e-10, (parts, k, err)
