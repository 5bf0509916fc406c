"""The C-ABI library builds, loads and exports every symbol include/*.h declares;
host-only logic (sizes, layout, argument validation) is checked without a GPU."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", h)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names += re.findall(r"^[A-Za-z_][\w \*]*?\b((?:pt|rx)_\w+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2207_08716_gb300 import native
    return native.load()


def test_every_declared_symbol_is_exported_and_bound(lib):
    from paper_2207_08716_gb300 import native
    declared = _declared_functions()
    assert len(declared) >= 11, declared
    for name in declared:
        assert hasattr(lib, name), name                    # dlsym succeeds
        assert name in native.SIGNATURES, name             # the binding declares it


def test_layout_sizes(lib):
    from paper_2207_08716_gb300 import native as N
    for (nx, ny, nz), px in (((32, 32, 32), 48), ((511, 511, 511), 512), ((15, 3, 2), 16),
                             ((1, 1, 1), 16), ((48, 40, 36), 64)):
        g = N.Grid(nx, ny, nz, 1.0, 1.0, 1.0)
        assert lib.pt_pitch_x(C.byref(g)) == px
        assert lib.pt_field_elems(C.byref(g)) == px * (ny + 1) * (nz + 1)
        num = N.num_from(__import__("pt_inputs").c1_params(nx, ny, nz))
        ws = lib.pt_workspace_size(C.byref(g), C.byref(num))
        assert ws >= 23 * px * (ny + 1) * (nz + 1) * 8
    bad = N.Grid(0, 4, 4, 1.0, 1.0, 1.0)
    assert lib.pt_field_elems(C.byref(bad)) == 0
    assert lib.pt_pitch_x(C.byref(N.Grid(4, 4, 4, -1.0, 1.0, 1.0))) == 0


def test_init_rejects_bad_arguments_before_touching_the_device(lib):
    """Validation happens on the host: each bad argument returns PT_EINVAL / PT_ESPACE and
    leaves the context null, without any CUDA call (this runs on a machine without a GPU)."""
    import pt_inputs as I
    from paper_2207_08716_gb300 import native as N
    p = I.c1_params(8)
    g, ph, num = N.grid_from(p), N.phys_from(p), N.num_from(p)
    aligned = 1 << 20
    fs = N.Fields(*([aligned] * 14), None)
    ws = lib.pt_workspace_size(C.byref(g), C.byref(num))
    ctx = C.c_void_p(1234)

    def call(g=g, ph=ph, num=num, fs=fs, w=aligned * 2, wb=ws):
        return lib.pt_init(C.byref(ctx), C.byref(g), C.byref(ph), C.byref(num), C.byref(fs), w, wb,
                           None, 0)

    assert call(g=N.Grid(0, 8, 8, 1, 1, 1)) == N.PT_EINVAL and ctx.value is None
    nb = N.num_from(dict(p, dt=0.0))
    assert call(num=nb) == N.PT_EINVAL
    nb = N.num_from(dict(p, nup=0))
    assert call(num=nb) == N.PT_EINVAL
    pb = N.phys_from(dict(p, phi0=1.5))
    assert call(ph=pb) == N.PT_EINVAL
    assert call(fs=N.Fields(*([aligned] * 13), 0, None)) == N.PT_EINVAL      # null eta
    assert call(fs=N.Fields(*([aligned + 8] + [aligned] * 13), None)) == N.PT_EINVAL  # misaligned
    assert call(w=aligned * 2 + 16) == N.PT_EINVAL                            # workspace alignment
    assert call(wb=ws - 1) == N.PT_ESPACE
    assert lib.pt_step(None, None) == N.PT_EINVAL
    # multigrid of the correction problem: FP32 only; each level ceil(n / 2) cells per direction,
    # the coarsest at least 2
    assert call(num=N.num_from(dict(p, mg_levels=3))) == N.PT_EINVAL                 # FP64 form
    assert call(num=N.num_from(dict(p, mg_levels=3, precision=N.PT_FP32)), wb=1) == N.PT_ESPACE  # 8 -> 4 -> 2
    assert call(num=N.num_from(dict(p, mg_levels=4, precision=N.PT_FP32))) == N.PT_EINVAL  # 8 -> ... -> 1
    p7 = I.c1_params(7, 6, 5)
    g7 = N.grid_from(p7)
    assert call(g=g7, num=N.num_from(dict(p7, mg_levels=3, precision=N.PT_FP32)), wb=1) == N.PT_ESPACE  # 4, 3, 3 -> 2
    assert call(g=g7, num=N.num_from(dict(p7, mg_levels=4, precision=N.PT_FP32))) == N.PT_EINVAL   # -> 1


def test_multigrid_workspace_adds_the_coarse_grids(lib):
    import pt_inputs as I
    from paper_2207_08716_gb300 import native as N
    p = dict(I.c1_params(32), precision=N.PT_FP32)
    g = N.grid_from(p)
    plain = lib.pt_workspace_size(C.byref(g), C.byref(N.num_from(p)))
    mg = lib.pt_workspace_size(C.byref(g), C.byref(N.num_from(dict(p, mg_levels=3))))

    def fbytes(n):   # one FP32 array of an n^3 grid's padded box, 256-byte aligned
        px = -(-(n + 1) // 16) * 16
        return -(-(px * (n + 1) * (n + 1) * 4) // 256) * 256

    def tables(nf, nc):   # the transfer tables of 3 directions (9 nc + 6 nf + 7 words each)
        return 3 * (-(-((9 * nc + 6 * nf + 7) * 4) // 256) * 256)
    assert mg - plain == 2 * fbytes(32) + 25 * (fbytes(16) + fbytes(8)) + tables(32, 16) + tables(16, 8)
    # an odd grid: 33 -> 17 -> 9 cells per direction
    p = dict(I.c1_params(33), precision=N.PT_FP32)
    g = N.grid_from(p)
    plain = lib.pt_workspace_size(C.byref(g), C.byref(N.num_from(p)))
    mg = lib.pt_workspace_size(C.byref(g), C.byref(N.num_from(dict(p, mg_levels=3))))
    assert mg - plain == 2 * fbytes(33) + 25 * (fbytes(17) + fbytes(9)) + tables(33, 17) + tables(17, 9)
    assert lib.pt_iterate(None, 0, 1, None) == N.PT_EINVAL
    assert lib.pt_strerror(N.PT_ENOTCONV).decode().startswith("PT iteration cap")


def test_decomposition_sizes_are_validated_on_the_host(lib):
    """pt_dd_workspace_size / pt_dd_init reject splits with fewer than 2 cells per part, bad part
    counts and FP32 precision before any CUDA call (runs without a GPU)."""
    import pt_inputs as I
    from paper_2207_08716_gb300 import native as N
    p = I.c1_params(10, 9, 8)
    g, ph, num = N.grid_from(p), N.phys_from(p), N.num_from(p)
    parts = lambda *v: (C.c_int32 * 3)(*v)
    assert lib.pt_dd_workspace_size(C.byref(g), C.byref(num), parts(1, 1, 1)) > 0
    assert lib.pt_dd_workspace_size(C.byref(g), C.byref(num), parts(5, 4, 4)) > 0
    assert lib.pt_dd_workspace_size(C.byref(g), C.byref(num), parts(6, 1, 1)) == 0   # 10 / 6 < 2 cells
    assert lib.pt_dd_workspace_size(C.byref(g), C.byref(num), parts(0, 1, 1)) == 0
    one = lib.pt_dd_workspace_size(C.byref(g), C.byref(num), parts(1, 1, 1))
    eight = lib.pt_dd_workspace_size(C.byref(g), C.byref(num), parts(2, 2, 2))
    assert eight > one                                   # halos and per-part boxes cost memory
    fs = N.Fields(*([None] * 15))
    h = C.c_void_p()
    aligned = 1 << 20
    num32 = N.num_from(dict(p, precision=N.PT_FP32))
    assert lib.pt_dd_init(C.byref(h), C.byref(g), C.byref(ph), C.byref(num32), C.byref(fs), parts(2, 2, 2),
                          aligned, eight, None) == N.PT_EINVAL
    assert lib.pt_dd_init(C.byref(h), C.byref(g), C.byref(ph), C.byref(num), C.byref(fs), parts(6, 1, 1),
                          aligned, eight, None) == N.PT_EINVAL
    assert lib.pt_dd_init(C.byref(h), C.byref(g), C.byref(ph), C.byref(num), C.byref(fs), parts(2, 2, 2),
                          aligned, 16, None) == N.PT_ESPACE
    assert not h.value


def test_multigrid_hierarchy_is_validated_on_the_host(lib):
    """rx_mg_workspace_size / rx_mg_init reject hierarchies whose grids do not halve evenly, bad
    sweep counts and weights before any CUDA call (runs without a GPU)."""
    import pt_inputs as I
    from paper_2207_08716_gb300 import native as N
    p = I.rx_params(16, 16, 40)                          # 40 = 8 * 5: at most 4 levels
    g = N.Grid(p["nx"], p["ny"], p["nz"], p["lx"], p["ly"], p["lz"])
    num = N.RxNum(p["dt"], p["tol"], p["cfl_div"], p["pf_scale"], p["max_iter"], p["nup"], N.PT_FP64)
    mg = lambda **kw: N.RxMg(*[kw.get(k, d) for k, d in (("levels", 4), ("nu_pre", 2), ("nu_post", 2),
                                                        ("nu_coarse", 20), ("max_cycles", 50))],
                             kw.get("omega", 6.0 / 7.0))
    base = lib.rx_workspace_size(C.byref(g), C.byref(num))
    four = lib.rx_mg_workspace_size(C.byref(g), C.byref(num), C.byref(mg()))
    assert base > 0 and four > base
    assert lib.rx_mg_workspace_size(C.byref(g), C.byref(num), C.byref(mg(levels=1))) == base
    for bad in (dict(levels=5), dict(levels=0), dict(levels=17), dict(nu_post=0), dict(nu_coarse=0),
                dict(nu_pre=-1), dict(max_cycles=0), dict(omega=0.0), dict(omega=1.2)):
        assert lib.rx_mg_workspace_size(C.byref(g), C.byref(num), C.byref(mg(**bad))) == 0, bad
    assert lib.rx_mg_workspace_size(C.byref(g), C.byref(num), C.byref(mg(levels=1, nu_post=0))) == base
    ph = N.RxPhys(*[float(p[k]) for k in ("phi0", "k0", "eta", "rhof", "rhos", "g", "beta_d", "beta_s",
                                          "beta_f", "beta_x", "dX", "xs_max", "tau")])
    aligned = 1 << 20
    fs = N.RxFields(aligned, aligned, aligned, aligned)
    h = C.c_void_p()
    assert lib.rx_mg_init(C.byref(h), C.byref(g), C.byref(ph), C.byref(num), C.byref(mg(levels=5)), C.byref(fs),
                          aligned, four, None) == N.PT_EINVAL
    assert lib.rx_mg_init(C.byref(h), C.byref(g), C.byref(ph), C.byref(num), C.byref(mg()), C.byref(fs),
                          aligned, four - 1, None) == N.PT_ESPACE
    assert not h.value
    assert lib.rx_mg_step(None, None) == N.PT_EINVAL
    assert lib.rx_mg_cycles(None, 1, None) == N.PT_EINVAL


def test_batch_rejects_mixed_precisions_on_the_host(lib):
    """An ensemble is all PT_FP64 or all PT_FP32; a mix is rejected before any CUDA call."""
    import pt_inputs as I
    from paper_2207_08716_gb300 import native as N
    ps = [I.c1_params(8), dict(I.c1_params(10), precision=N.PT_FP32)]
    G = (N.Grid * 2)(*[N.grid_from(p) for p in ps])
    P = (N.Phys * 2)(*[N.phys_from(p) for p in ps])
    U = (N.Num * 2)(*[N.num_from(p) for p in ps])
    F = (N.Fields * 2)(*[N.Fields(*([None] * 15)) for _ in ps])
    ws = lib.pt_batch_workspace_size(2, G, U)
    assert ws > 0
    h = C.c_void_p()
    assert lib.pt_batch_init(C.byref(h), 2, G, P, U, F, 1 << 20, ws, None) == N.PT_EINVAL
    assert not h.value
