"""Reactive porosity-wave solver (rx_* C ABI; thesis Art. 3, Eqs. 8-10) against the FP64 oracle.

Bars: FP64 fields after the same iteration count within 1e-10 (max-rel, normwise; the thesis's
FP64 verification bar); FP64 converged steps with the same iteration counts; the FP32 form
(the precision the thesis ran this solver in) within 1e-5 normwise of the FP64 oracle after
converged steps: single-precision rounding (6e-8 relative) of the iterate and of the change
criterion (tol 2e-8) bounds the converged fields' error well below that.
"""
import numpy as np
import pytest

import pt_inputs as I
from oracle import rx as R

pytestmark = pytest.mark.gpu

FIELDS = ("Pf", "phi", "Xs", "R")


def _solver():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_08716_gb300.solver import RXSolver
    return RXSolver


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("dims, niter, Da", [((12, 10, 40), 95, 100.0), ((7, 9, 13), 60, 0.01),
                                              ((33, 17, 70), 40, 100.0)])
def test_fixed_iterations_match_oracle_fp64(dims, niter, Da):
    RXSolver = _solver()
    p = I.rx_params(*dims, Da=Da, dt=1e-5)
    Pf, phi, Xs = I.rx_initial(p)
    s = RXSolver(p, Pf + 0.01, phi, Xs)
    st = R.RxState(p, Pf + 0.01, phi, Xs)
    for _ in range(2):
        rep = s.iterate(niter)
        rc, ch = R.iterate_n(st, niter)
        assert rc == 0
        errs = {k: rel(s.get(k), st[k]) for k in FIELDS}
        assert max(errs.values()) <= 1e-10, errs
    s.close()


def test_converged_steps_match_oracle_fp64():
    RXSolver = _solver()
    p = I.rx_params(10, 10, 40)
    Pf, phi, Xs = I.rx_initial(p)
    s = RXSolver(p, Pf, phi, Xs)
    st = R.RxState(p, Pf, phi, Xs)
    for _ in range(3):
        rep = s.step(raise_on_notconv=True)
        rc, iters, ch = R.step(st)
        assert rc == 0 and rep["iters"] == iters, (rep, iters)
    for k in FIELDS:
        assert rel(s.get(k), st[k]) <= 1e-10, k
    s.close()


def test_fp32_converged_steps_are_within_single_precision_bar():
    RXSolver = _solver()
    from paper_2207_08716_gb300 import native as N
    p = I.rx_params(12, 12, 48)
    Pf, phi, Xs = I.rx_initial(p)
    s = RXSolver(dict(p, precision=N.PT_FP32), Pf, phi, Xs)
    st = R.RxState(p, Pf, phi, Xs)
    for _ in range(3):
        s.step(raise_on_notconv=True)
        rc, iters, ch = R.step(st)
        assert rc == 0
    for k in ("Pf", "phi", "Xs"):
        assert rel(s.get(k), st[k]) <= 1e-5, (k, rel(s.get(k), st[k]))
    s.close()
