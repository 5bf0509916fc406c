"""Multigrid (FAS V-cycle) reactive step on the GPU (rx_mg_* C ABI; thesis Art. 3, Eqs. 8-10
with the thesis's proposed multigrid acceleration) against the FP64 multigrid oracle.

Bars: FP64 fields after the same number of V-cycles within 1e-10 (max-rel, normwise); FP64
converged steps with the same cycle counts; the FP32 form within 1e-5 normwise of the FP64 oracle
(single-precision rounding of the iterate and of the change criterion, as for the plain solver).
At the full 256 x 256 x 1024 workload, the oracle evaluates the step equations on the
neighbourhood of sampled cells of the converged GPU state: the residual left there must be within
the change tolerance (one sweep's correction), in FP64 and in FP32.
"""
import numpy as np
import pytest

import pt_inputs as I
from oracle import rx as R

pytestmark = pytest.mark.gpu

FIELDS = ("Pf", "phi", "Xs", "R")
MG = dict(levels=3, nu_pre=2, nu_post=2, nu_coarse=30, max_cycles=200, omega=6.0 / 7.0)


def _solver():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_08716_gb300.solver import RXSolver
    return RXSolver


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("dims, levels, ncyc, dt", [((16, 16, 64), 4, 3, 1e-5), ((12, 10, 24), 2, 4, 1e-4),
                                                     ((24, 20, 40), 3, 3, 1e-5), ((8, 8, 8), 1, 2, 1e-5),
                                                     ((32, 16, 48), 5, 2, 1e-5)])
def test_fixed_cycles_match_oracle_fp64(dims, levels, ncyc, dt):
    RXSolver = _solver()
    p = I.rx_params(*dims, dt=dt)
    Pf, phi, Xs = I.rx_initial(p)
    mg = dict(MG, levels=levels)
    s = RXSolver(p, Pf + 0.01, phi, Xs, mg=mg)
    st = R.RxState(p, Pf + 0.01, phi, Xs)
    for _ in range(2):
        rep = s.mg_cycles(ncyc)
        rc, ch = R.mg_cycles(st, mg, ncyc)
        assert rc == 0 and rep["iters"] == ncyc
        errs = {k: rel(s.get(k), st[k]) for k in FIELDS}
        assert max(errs.values()) <= 1e-10, errs
        assert abs(rep["r_v"] - ch) <= 1e-6 * ch + 1e-15, (rep["r_v"], ch)     # floor: rounding of the fields
    s.close()


def test_converged_steps_match_oracle_fp64():
    RXSolver = _solver()
    p = I.rx_params(16, 16, 64, dt=1e-5)
    Pf, phi, Xs = I.rx_initial(p)
    mg = dict(MG, levels=4)
    s = RXSolver(p, Pf, phi, Xs, mg=mg)
    st = R.RxState(p, Pf, phi, Xs)
    for _ in range(3):
        rep = s.mg_step(raise_on_notconv=True)
        rc, cycles, ch = R.mg_step(st, mg)
        assert rc == 0 and rep["iters"] == cycles, (rep, cycles)
    for k in FIELDS:
        assert rel(s.get(k), st[k]) <= 1e-10, k
    s.close()


def test_fp32_converged_steps_are_within_single_precision_bar():
    RXSolver = _solver()
    from paper_2207_08716_gb300 import native as N
    p = I.rx_params(16, 16, 64, dt=1e-5)
    Pf, phi, Xs = I.rx_initial(p)
    mg = dict(MG, levels=4)
    s = RXSolver(dict(p, precision=N.PT_FP32), Pf, phi, Xs, mg=mg)
    st = R.RxState(p, Pf, phi, Xs)
    for _ in range(3):
        s.mg_step(raise_on_notconv=True)
        rc, cycles, ch = R.mg_step(st, mg)
        assert rc == 0
    for k in ("Pf", "phi", "Xs"):
        assert rel(s.get(k), st[k]) <= 1e-5, (k, rel(s.get(k), st[k]))
    s.close()


def test_multigrid_and_plain_steps_reach_the_same_fixed_point():
    RXSolver = _solver()
    p = I.rx_params(16, 16, 64, dt=1e-4)
    p.update(tol=1e-13, max_iter=400000)
    Pf, phi, Xs = I.rx_initial(p)
    a = RXSolver(p, Pf, phi, Xs, mg=dict(MG, levels=4))
    b = RXSolver(p, Pf, phi, Xs)
    ra = a.mg_step(raise_on_notconv=True)
    rb = b.step(raise_on_notconv=True)
    assert 20 * ra["iters"] < rb["iters"], (ra, rb)
    for k in FIELDS:
        assert rel(a.get(k), b.get(k)) <= 1e-8, (k, rel(a.get(k), b.get(k)))
    a.close()
    b.close()


def test_diverging_step_is_reported():
    RXSolver = _solver()
    from paper_2207_08716_gb300 import native as N
    from paper_2207_08716_gb300.solver import PTError
    p = I.rx_params(8, 8, 32, dt=1e-2)
    Pf, phi, Xs = I.rx_initial(p)
    for prec in (N.PT_FP64, N.PT_FP32):
        s = RXSolver(dict(p, precision=prec), Pf, phi, Xs, mg=MG)
        with pytest.raises(PTError) as e:
            s.mg_step()
        assert e.value.code == N.PT_ENAN
        s.close()
        s = RXSolver(dict(p, precision=prec, max_iter=2000), Pf, phi, Xs)
        with pytest.raises(PTError) as e:
            s.step()
        assert e.value.code == N.PT_ENAN
        s.close()


def _window_residuals(p, u, old, cells, omega):
    """Oracle step equations (f = 0) at each sampled cell, evaluated on the cell's neighbourhood
    clipped to the box: a cell's equations read only itself and its six neighbours, and the
    clipped window's walls are the box's own where the cell touches them."""
    h = (p["lx"] / p["nx"], p["ly"] / p["ny"], p["lz"] / p["nz"])
    out = []
    for (k, j, i) in cells:
        lo = [max(c - 1, 0) for c in (k, j, i)]
        hi = [min(c + 2, n) for c, n in zip((k, j, i), (p["nz"], p["ny"], p["nx"]))]
        sl = tuple(slice(a, b) for a, b in zip(lo, hi))
        shape = [b - a for a, b in zip(lo, hi)]
        q = dict(p, nz=shape[0], ny=shape[1], nx=shape[2], lz=shape[0] * h[2], ly=shape[1] * h[1],
                 lx=shape[2] * h[0])
        gP, gphi, gX, den, _ = R.mg_equations(q, [a[sl] for a in u], [a[sl] for a in old], omega=omega)
        c = (k - lo[0], j - lo[1], i - lo[2])
        out.append((gP[c] / den[c], gphi[c], gX[c]))
    return np.array(out)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_full_size_converged_state_has_no_residual_at_sampled_cells(precision):
    RXSolver = _solver()
    from paper_2207_08716_gb300 import native as N
    n = 256
    p = I.rx_params(n)
    prec = N.PT_FP64 if precision == "fp64" else N.PT_FP32
    Pf, phi, Xs = I.rx_initial(p)
    mg = dict(MG, levels=7, max_cycles=60)
    s = RXSolver(dict(p, precision=prec), Pf, phi, Xs, mg=mg)
    rep = s.mg_step(raise_on_notconv=True)
    assert rep["iters"] <= 30, rep
    u = [s.get(k) for k in ("Pf", "phi", "Xs")]
    s.close()
    rng = np.random.default_rng(7)
    cells = [(int(rng.integers(0, 4 * n)), int(rng.integers(0, n)), int(rng.integers(0, n))) for _ in range(40)]
    cells += [(0, 0, 0), (4 * n - 1, n - 1, n - 1), (2 * n, n // 2, 0), (25, n // 2, n // 2), (102, n // 2, n // 2)]
    r = _window_residuals(p, u, (Pf, phi, Xs), cells, mg["omega"])
    tol = p["tol"]
    slack = 10.0 if precision == "fp64" else 100.0
    assert np.abs(r[:, 0]).max() <= slack * tol * p["pf_scale"], np.abs(r[:, 0]).max()
    assert np.abs(r[:, 1]).max() <= slack * tol, np.abs(r[:, 1]).max()
    assert np.abs(r[:, 2]).max() <= slack * tol, np.abs(r[:, 2]).max()
