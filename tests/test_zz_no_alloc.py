"""pt_residual_static: the residual norms for callers that cannot allocate device memory.

A health check inside a run whose device memory is fully held by a pool allocator, or a
timing-critical loop that cannot take cudaMalloc's implicit synchronisation, cannot get a
workspace for pt_residual. pt_residual_static keeps its intermediates in a fixed array inside
the library instead. This file is collected last so that a run stopping at the first failure
has run every other test before it; it passes alone in a fresh process too.
"""
import ctypes as C

import numpy as np
import pytest

import pt_inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-10   # the parity tolerance of the other GPU tests


def _setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_08716_gb300 import native as N
    from paper_2207_08716_gb300.solver import PTSolver
    return torch, N, PTSolver


def test_static_residual_matches_context_residual_on_two_calls():
    torch, N, PTSolver = _setup()
    p = I.c1_params(20, 18, 16)
    rs = I.random_state(p, seed=21, scale=1e-3)
    fields = {k: v for k, v in rs.items() if k != "phi"}
    s = PTSolver(p, rs["phi"], fields=fields)
    s.step_begin()                      # first step: old fields = current fields, dtS from mu0
    want = s.residual()
    assert want["status"] == 0 and want["r_v"] > 0
    f = s.f
    fs = N.Fields(*[f[k].data_ptr() for k in N.FIELD_NAMES], None)
    old = N.OldFields(*[f[k].data_ptr() for k in ("Pt", "Pf", "txx", "tyy", "tzz", "txy", "txz", "tyz")])
    dtS = p["mu0"] / (p["G"] * p["xsi_w"])
    grid, phys, num = N.grid_from(p), N.phys_from(p), N.num_from(p)
    lib = N.load()
    for call in range(2):
        rep = N.Report()
        rc = lib.pt_residual_static(C.byref(grid), C.byref(phys), C.byref(num), C.byref(fs),
                                    C.byref(old), dtS, s.stream.cuda_stream, C.byref(rep))
        assert rc == 0 and rep.status == 0, (call, rc)
        got = rep.as_dict()
        for k in ("r_v", "r_pt", "r_pf", "r_pic"):
            assert abs(got[k] - want[k]) <= TOL * abs(want[k]) + 1e-300, (call, k, got[k], want[k])
    # the inputs were only read
    np.testing.assert_array_equal(s.get("mu"), np.full((16, 18, 20), p["mu0"]))
    s.close()


def test_static_residual_rejects_grids_beyond_its_array():
    torch, N, PTSolver = _setup()
    p = I.c1_params(128)
    grid, phys, num = N.grid_from(p), N.phys_from(p), N.num_from(p)
    dummy = 1 << 20
    fs = N.Fields(*([dummy] * 14), None)
    old = N.OldFields(*([dummy] * 8))
    rep = N.Report()
    rc = N.load().pt_residual_static(C.byref(grid), C.byref(phys), C.byref(num), C.byref(fs),
                                     C.byref(old), 0.02, None, C.byref(rep))
    assert rc == N.PT_ESPACE and rep.status == N.PT_ESPACE
