"""The hand-written device arithmetic of the PT kernels, routine by routine, against CUDA's (and
numpy's) own functions and against each routine's stated error bound (pt_math_check):

* Newton-Raphson reciprocal iteration r' = r + r (1 - x r) on the hardware's approximate FP64
  reciprocal (good to ~2^-20): one step (pseudo-time steps, ~2^-40) and two steps
  (coefficients, rounding);
* the split Taylor series of exp, expm1(d) = E + O and expm1(-d) = E - O, in its two tiers and
  beyond them (CUDA's expm1);
* double-float arithmetic from the error-free transformations of Knuth (two-sum) and Dekker
  (fast two-sum, exact product via FMA): add, subtract, multiply, multiply-add, and the Newton
  reciprocal, square root and m-th root from FP32 seeds.

Double-float inputs are first rounded to double-float (hi = fl32(x), lo = fl32(x - hi)); the
reference is the FP64 result on those rounded inputs.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

EPS = 2.0 ** -53


def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_08716_gb300 import native as N
    return torch, N, N.load()


def _run(fn, a, b=None):
    torch, N, lib = _lib()
    ta = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
    tb = torch.from_numpy(np.ascontiguousarray(b, dtype=np.float64)).cuda() if b is not None else None
    out = torch.empty_like(ta)
    torch.cuda.synchronize()
    rc = lib.pt_math_check(fn, ta.data_ptr(), tb.data_ptr() if tb is not None else None, out.data_ptr(),
                           ta.numel(), None)
    assert rc == 0, rc
    return out.cpu().numpy()


def _df(x):
    """x rounded to double-float, as an FP64 value."""
    hi = np.asarray(x, dtype=np.float64).astype(np.float32)
    lo = (np.asarray(x, dtype=np.float64) - hi.astype(np.float64)).astype(np.float32)
    return hi.astype(np.float64) + lo.astype(np.float64)


def _loguniform(rng, lo, hi, n, signed=False):
    x = np.exp(rng.uniform(np.log(lo), np.log(hi), n))
    if signed:
        x *= rng.choice([-1.0, 1.0], n)
    return x


RCP_PSEUDO, RCP_FULL, EXPM1_POS, EXPM1_NEG = 0, 1, 2, 3
DF_ADD, DF_SUB, DF_MUL, DF_FMA, DF_RCP, DF_SQRT, DF_ROOT, DF_EXPM1_POS, DF_EXPM1_NEG = range(4, 13)


def test_newton_reciprocals_fp64():
    rng = np.random.default_rng(1)
    x = _loguniform(rng, 1e-8, 1e8, 200000)
    ref = 1.0 / x                                   # correctly rounded
    r1 = _run(RCP_PSEUDO, x)
    r2 = _run(RCP_FULL, x)
    e1 = np.abs(r1 - ref) / ref
    e2 = np.abs(r2 - ref) / ref
    assert e1.max() <= 2.0 ** -39, e1.max()           # one Newton step: the ~2^-20 seed's error squared
    assert e2.max() <= 2.0 * EPS, e2.max()            # two steps: within an ulp of the quotient
    torch, _, _ = _lib()
    cu = (1.0 / torch.from_numpy(x).cuda()).cpu().numpy()   # CUDA's own division
    assert np.abs(r2 - cu).max() / np.abs(cu).max() <= 2.0 * EPS


@pytest.mark.parametrize("lo, hi", [(1e-30, 2.0 ** -20), (2.0 ** -20, 2.0 ** -6), (2.0 ** -6, 5.0)])
def test_split_taylor_expm1_fp64(lo, hi):
    rng = np.random.default_rng(2)
    d = _loguniform(rng, lo, hi, 100000, signed=True)
    p, m = _run(EXPM1_POS, d), _run(EXPM1_NEG, d)
    torch, _, _ = _lib()
    cu_p = torch.expm1(torch.from_numpy(d).cuda()).cpu().numpy()
    cu_m = torch.expm1(torch.from_numpy(-d).cuda()).cpu().numpy()
    # truncation below 2^-60 |d| plus a few roundings of the sums E + O, E - O
    for got, ref in ((p, np.expm1(d)), (m, np.expm1(-d)), (p, cu_p), (m, cu_m)):
        err = np.abs(got - ref) / np.abs(ref)
        assert err.max() <= 8 * EPS, (lo, hi, err.max())


def test_double_float_add_sub_mul_fma():
    rng = np.random.default_rng(3)
    n = 200000
    x = _loguniform(rng, 1e-6, 1e6, n, signed=True)
    y = _loguniform(rng, 1e-6, 1e6, n, signed=True)
    y[: n // 4] = -x[: n // 4] * (1 + rng.uniform(-1e-7, 1e-7, n // 4))   # heavy cancellation
    xr, yr = _df(x), _df(y)
    u = 2.0 ** -48
    s = _run(DF_ADD, x, y)
    assert np.all(np.abs(s - (xr + yr)) <= 4 * u * (np.abs(xr) + np.abs(yr)))
    d = _run(DF_SUB, x, y)
    assert np.all(np.abs(d - (xr - yr)) <= 4 * u * (np.abs(xr) + np.abs(yr)))
    p = _run(DF_MUL, x, y)
    assert np.all(np.abs(p - xr * yr) <= 4 * u * np.abs(xr * yr))
    f = _run(DF_FMA, x, y)
    assert np.all(np.abs(f - (xr * yr + xr)) <= 6 * u * (np.abs(xr * yr) + np.abs(xr)))


def test_double_float_newton_rcp_sqrt_root():
    rng = np.random.default_rng(4)
    x = _loguniform(rng, 1e-10, 1e10, 200000)
    xr = _df(x)
    u = 2.0 ** -48
    r = _run(DF_RCP, x)
    assert (np.abs(r - 1.0 / xr) * xr).max() <= 8 * u
    q = _run(DF_SQRT, x)
    assert (np.abs(q - np.sqrt(xr)) / np.sqrt(xr)).max() <= 8 * u
    for m in (2, 3, 10):
        t = _run(DF_ROOT, x, np.full_like(x, m))
        ref = xr ** (1.0 / m)
        assert (np.abs(t - ref) / ref).max() <= 16 * u, m
    assert _run(DF_SQRT, np.array([0.0]))[0] == 0.0


@pytest.mark.parametrize("lo, hi", [(1e-25, 2.0 ** -20), (2.0 ** -20, 2.0 ** -6), (2.0 ** -6, 3.0)])
def test_double_float_split_taylor_expm1(lo, hi):
    rng = np.random.default_rng(5)
    d = _loguniform(rng, lo, hi, 100000, signed=True)
    dr = _df(d)
    p, m = _run(DF_EXPM1_POS, d), _run(DF_EXPM1_NEG, d)
    for got, ref in ((p, np.expm1(dr)), (m, np.expm1(-dr))):
        err = np.abs(got - ref) / np.abs(ref)
        assert err.max() <= 16 * 2.0 ** -48, (lo, hi, err.max())


def test_unknown_routine_is_rejected():
    torch, N, lib = _lib()
    a = torch.ones(4, dtype=torch.float64, device="cuda")
    assert lib.pt_math_check(99, a.data_ptr(), None, a.data_ptr(), 4, None) == N.PT_EINVAL
    assert lib.pt_math_check(DF_ADD, a.data_ptr(), None, a.data_ptr(), 4, None) == N.PT_EINVAL
