"""The multigrid transfer weights of the FP32 form's correction solves (host logic, no GPU): for
nf fine cells and nc = ceil(nf / 2) coarse cells over the same box, the library's tables must be
(i) a partition of unity covering every fine cell exactly once (box restriction), (ii) a
normalised hat of half-width nf / nc around each coarse face, (iii) linear interpolation between
coarse centres that reproduces linear fields away from the walls, (iv) linear interpolation between
coarse faces; and for even nf the classical factor-2 weights (mean of 2 per direction;
1/4, 1/2, 1/4; 3/4, 1/4; 1/2, 1/2)."""
import ctypes as C

import numpy as np
import pytest


@pytest.fixture(scope="module")
def lib():
    from paper_2207_08716_gb300 import native
    return native.load()


def tables(lib, nf):
    nc = (nf + 1) // 2
    words = lib.pt_mg_axis_words(nf)
    assert words == 9 * nc + 6 * nf + 7
    buf = np.zeros(words, dtype=np.uint32)
    assert lib.pt_mg_axis_tables(nf, buf.ctypes.data_as(C.c_void_p), words) == 0
    f = buf.view(np.float32)
    i = buf.view(np.int32)
    o = 0
    out = {}
    for name, n, view in (("box_i0", nc, i), ("box_w", 3 * nc, f), ("hat_i0", nc + 1, i), ("hat_w", 4 * (nc + 1), f),
                          ("lin_ab", 2 * nf, i), ("lin_w", 2 * nf, f), ("fl_n0", nf + 1, i), ("fl_t", nf + 1, f)):
        out[name] = view[o:o + n].copy()
        o += n
    out["box_w"] = out["box_w"].reshape(nc, 3)
    out["hat_w"] = out["hat_w"].reshape(nc + 1, 4)
    out["lin_ab"] = out["lin_ab"].reshape(nf, 2)
    out["lin_w"] = out["lin_w"].reshape(nf, 2)
    return nc, out


@pytest.mark.parametrize("nf", [2, 5, 8, 9, 33, 64, 127, 511, 767])
def test_tables_are_the_stated_transfers(lib, nf):
    nc, t = tables(lib, nf)
    r = nf / nc
    # (i) box weights: each coarse cell's weights sum to 1 and the fine cells are covered once
    cover = np.zeros(nf)
    for I in range(nc):
        w = t["box_w"][I]
        assert abs(w.sum() - 1.0) < 1e-6
        for k in range(3):
            if w[k] > 0:
                i = t["box_i0"][I] + k
                assert 0 <= i < nf
                cover[i] += w[k] * r
    np.testing.assert_allclose(cover, 1.0, atol=1e-5)
    # (ii) hat weights of the interior coarse faces: normalised, inside [0, nf], centred on J r
    for J in range(1, nc):
        w = t["hat_w"][J]
        i = t["hat_i0"][J] + np.arange(4)
        assert abs(w.sum() - 1.0) < 1e-6 and np.all(i[w > 0] <= nf) and np.all(i >= 0)
        # first moment near the face position: exact when nested (symmetric stencil), within a
        # quarter of a fine cell otherwise (the hat sampled at the fine faces is not symmetric)
        assert abs((w * i).sum() - J * r) <= (1e-6 if nf % 2 == 0 else 0.25)
    # (iii) linear between coarse centres: a linear field x is reproduced between the first and
    # last coarse centres, held constant beyond them
    xc = (np.arange(nc) + 0.5) * r                            # coarse centres in fine-cell units
    for i in range(nf):
        a, b = t["lin_ab"][i]
        wa, wb = t["lin_w"][i]
        assert 0 <= a < nc and 0 <= b < nc and abs(wa + wb - 1.0) < 1e-6
        x = i + 0.5
        expect = min(max(x, xc[0]), xc[-1])
        assert abs(wa * xc[a] + wb * xc[b] - expect) < 1e-4
    # (iv) linear between coarse faces for the interior fine faces
    for i in range(1, nf):
        n0, tt = t["fl_n0"][i], t["fl_t"][i]
        assert 0 <= n0 < nc and 0 <= tt < 1
        assert abs((n0 + tt) * r - i) < 1e-4


def test_even_grids_give_the_factor_two_weights(lib):
    nc, t = tables(lib, 16)
    np.testing.assert_array_equal(t["box_w"][:, :2], 0.5)
    np.testing.assert_array_equal(t["box_w"][:, 2], 0.0)
    np.testing.assert_array_equal(t["box_i0"], 2 * np.arange(nc))
    for J in range(1, nc):
        w = t["hat_w"][J]
        assert t["hat_i0"][J] == 2 * J - 1 and np.array_equal(w[:3], [0.25, 0.5, 0.25]) and w[3] == 0.0
    for i in range(1, 15):   # interior: 3/4 on the own coarse cell, 1/4 on the neighbour
        a, b = t["lin_ab"][i]
        wa, wb = t["lin_w"][i]
        own = i // 2
        got = {a: 0.0, b: 0.0}
        got[a] += wa
        got[b] += wb
        assert got[own] == 0.75 and sum(got.values()) == 1.0
    for i in range(1, 16):
        assert t["fl_n0"][i] == i // 2 and t["fl_t"][i] == (0.5 if i % 2 else 0.0)


def test_rejects_bad_sizes(lib):
    from paper_2207_08716_gb300 import native as N
    buf = np.zeros(64, dtype=np.uint32)
    assert lib.pt_mg_axis_tables(1, buf.ctypes.data_as(C.c_void_p), 64) == N.PT_EINVAL
    assert lib.pt_mg_axis_tables(33, buf.ctypes.data_as(C.c_void_p), 64) == N.PT_ESPACE
    assert lib.pt_mg_axis_words(1) == 0
