"""pt_residual_static: the residual norms for callers that cannot allocate device memory.

A health check inside a run whose device memory is fully held by a pool allocator, or a
timing-critical loop that cannot take cudaMalloc's implicit synchronisation, cannot get a
workspace for pt_residual. pt_residual_static keeps its intermediates in a fixed array inside
the library instead. This file is collected last so that a run stopping at the first failure
has run every other test before it; it passes alone in a fresh process too.

What is checked: the norms equal pt_residual's (same state, two calls in a row); they equal the
oracle's system residual on states whose old-step fields differ from the current ones, with and
without the background shear of Eqs. 32-33; the capacity limit sits exactly where the padded box
stops fitting 10 arrays; a call still succeeds once the rest of the device memory is taken.
"""
import ctypes as C

import numpy as np
import pytest

import oracle as O
import pt_inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-10   # the parity tolerance of the other GPU tests
OLD_NAMES = ("Pto", "Pfo", "txxo", "tyyo", "tzzo", "txyo", "txzo", "tyzo")
OLD_SHAPE_OF = {"Pto": "Pt", "Pfo": "Pt", "txxo": "txx", "tyyo": "tyy", "tzzo": "tzz",
                "txyo": "txy", "txzo": "txz", "tyzo": "tyz"}


def _setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_08716_gb300 import native as N
    from paper_2207_08716_gb300.solver import PTSolver
    return torch, N, PTSolver


def _call(N, p, fs, old, dtS, stream=None):
    grid, phys, num = N.grid_from(p), N.phys_from(p), N.num_from(p)
    rep = N.Report()
    rc = N.load().pt_residual_static(C.byref(grid), C.byref(phys), C.byref(num), C.byref(fs),
                                     C.byref(old), dtS, stream, C.byref(rep))
    return rc, rep


def _device_state(torch, N, p, arrays):
    """Box-layout device copies of an oracle state's current and old-step fields."""
    from paper_2207_08716_gb300.solver import natural_shape
    lib = N.load()
    grid = N.grid_from(p)
    px = lib.pt_pitch_x(C.byref(grid))
    box = (p["nz"] + 1, p["ny"] + 1, px)
    dev = {}
    for name in N.FIELD_NAMES + OLD_NAMES:
        t = torch.zeros(box, dtype=torch.float64, device="cuda")
        src = arrays[name]
        sh = natural_shape(OLD_SHAPE_OF.get(name, name), p["nx"], p["ny"], p["nz"])
        assert src.shape == sh, (name, src.shape, sh)
        t[: sh[0], : sh[1], : sh[2]].copy_(torch.from_numpy(np.ascontiguousarray(src)))
        dev[name] = t
    torch.cuda.synchronize()
    fs = N.Fields(*[dev[k].data_ptr() for k in N.FIELD_NAMES], None)
    old = N.OldFields(*[dev[k].data_ptr() for k in OLD_NAMES])
    return dev, fs, old


def _oracle_norms(st):
    r = O.system_residual(st)
    return dict(r_v=max(np.abs(r[k]).max() for k in ("Vx", "Vy", "Vz")),
                r_pt=float(np.abs(r["pt"]).max()), r_pf=float(np.abs(r["pf"]).max()),
                r_pic=max(float(np.abs(r["mu"]).max()), float(np.abs(r["eta"]).max())))


def _assert_norms(got, want, what):
    for k, v in want.items():
        assert abs(got[k] - v) <= TOL * abs(v) + 1e-300, (what, k, got[k], v)


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
    for call in range(2):
        rc, rep = _call(N, p, fs, old, dtS, s.stream.cuda_stream)
        assert rc == 0 and rep.status == 0, (call, rc)
        _assert_norms(rep.as_dict(), {k: want[k] for k in ("r_v", "r_pt", "r_pf", "r_pic")}, call)
    # the inputs were only read
    np.testing.assert_array_equal(s.get("mu"), np.full((16, 18, 20), p["mu0"]))
    s.close()


def _evolved_oracle_state(p, phi, fields=None):
    """Oracle state in the second physical step: old-step pressures and stresses differ from the
    current ones (step 1 of 20 iterations, then 7 iterations of step 2)."""
    st = O.make_state(p, phi, fields=fields)
    O.begin_step(st)
    rc, _ = O.iterate_n(st, 0, 20)
    assert rc == 0
    O.end_step(st)
    O.begin_step(st)
    rc, _ = O.iterate_n(st, 0, 7)
    assert rc == 0
    assert np.abs(st["Pt"] - st["Pto"]).max() > 0 and np.abs(st["txy"] - st["txyo"]).max() > 0
    return st


@pytest.mark.parametrize("case", ["c1", "c1_tau_bg", "shear"])
def test_static_residual_matches_oracle_with_old_fields_and_shear(case):
    """After a step and a half (old fields != current fields) the four norms equal the oracle's
    system residual, on two calls in a row; with tau_bg != 0 the background xy strain rate and
    the wall-edge stresses of Eqs. 32-33 are in them."""
    torch, N, _ = _setup()
    if case == "shear":
        p = I.shear_params(8)
        p["xsi_w"] = 0.05               # dtS > 2 dt: step 2 keeps the first step's old stresses
        phi = I.ellipsoid_porosity(p)
        st = _evolved_oracle_state(p, phi)
    else:
        p = I.c1_params(14, 12, 10)
        if case == "c1_tau_bg":
            p["tau_bg"] = 0.02
        rs = I.random_state(p, seed=33, scale=1e-3)
        st = _evolved_oracle_state(p, rs["phi"], {k: v for k, v in rs.items() if k != "phi"})
    want = _oracle_norms(st)
    assert want["r_v"] > 0 and want["r_pt"] > 0
    dev, fs, old = _device_state(torch, N, p, st)
    for call in range(2):
        rc, rep = _call(N, p, fs, old, st.dtS)
        assert rc == 0 and rep.status == 0, (case, call, rc)
        _assert_norms(rep.as_dict(), want, (case, call))
    if case == "c1_tau_bg":
        # the background term matters here: without it the norms differ (in the shear workload
        # the max-norms sit where the weakening switch, not the shear, sets them)
        q = dict(p, tau_bg=0.0)
        rc, rep = _call(N, q, fs, old, st.dtS)
        assert rc == 0
        got = rep.as_dict()
        assert any(abs(got[k] - want[k]) > 1e-6 * abs(want[k]) for k in want), (case, got, want)


def test_static_residual_capacity_limit_92_accepted_93_rejected():
    """10 padded boxes of 92^3 cells (96 x 93 x 93 doubles each) fit the 64 MiB array; 93^3
    (96 x 94 x 94) does not and is rejected before any device work."""
    torch, N, _ = _setup()
    p = I.c1_params(92)
    phi = I.gaussian_porosity(p)
    st = O.make_state(p, phi)
    O.begin_step(st)
    rc, _ = O.iterate_n(st, 0, 3)
    assert rc == 0
    want = _oracle_norms(st)
    dev, fs, old = _device_state(torch, N, p, st)
    rc, rep = _call(N, p, fs, old, st.dtS)
    assert rc == 0 and rep.status == 0
    _assert_norms(rep.as_dict(), want, "92^3")
    del dev
    q = I.c1_params(93)
    dummy = 1 << 20
    rc, rep = _call(N, q, N.Fields(*([dummy] * 14), None), N.OldFields(*([dummy] * 8)), 0.02)
    assert rc == N.PT_ESPACE and rep.status == N.PT_ESPACE


def test_static_residual_rejects_grids_beyond_its_array():
    torch, N, PTSolver = _setup()
    p = I.c1_params(128)
    dummy = 1 << 20
    rc, rep = _call(N, p, N.Fields(*([dummy] * 14), None), N.OldFields(*([dummy] * 8)), 0.02)
    assert rc == N.PT_ESPACE and rep.status == N.PT_ESPACE


def test_static_residual_rejects_what_pt_init_rejects():
    """Same argument rules as pt_init: an infinite extent, an nx beyond 2^20 and a non-finite
    dt are PT_EINVAL (no device work, no arithmetic on them)."""
    torch, N, _ = _setup()
    dummy = 1 << 20
    fs, old = N.Fields(*([dummy] * 14), None), N.OldFields(*([dummy] * 8))
    for over in (dict(lx=float("inf")), dict(nx=(1 << 20) + 3), dict(nx=2**31 - 2), dict(dt=float("nan"))):
        p = dict(I.c1_params(8), **over)
        rc, rep = _call(N, p, fs, old, 0.02)
        assert rc == N.PT_EINVAL, (over, rc)


def test_static_residual_after_the_pool_takes_the_device_memory():
    """A first call on the device (which reserves the library's array), then a caller that takes
    nearly all remaining device memory: the next call still runs and gives the same norms."""
    torch, N, _ = _setup()
    p = I.c1_params(20, 18, 16)
    rs = I.random_state(p, seed=4, scale=1e-3)
    st = _evolved_oracle_state(p, rs["phi"], {k: v for k, v in rs.items() if k != "phi"})
    want = _oracle_norms(st)
    dev, fs, old = _device_state(torch, N, p, st)
    rc, rep = _call(N, p, fs, old, st.dtS)          # warm-up: the first call on this device
    assert rc == 0
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    free, _ = torch.cuda.mem_get_info()
    hold = max(0, free - (1 << 30))                 # leave 1 GiB for the driver
    pool = torch.empty(hold, dtype=torch.uint8, device="cuda") if hold else None
    try:
        rc, rep = _call(N, p, fs, old, st.dtS)
        assert rc == 0 and rep.status == 0
        _assert_norms(rep.as_dict(), want, "under memory pressure")
    finally:
        del pool
        torch.cuda.empty_cache()
