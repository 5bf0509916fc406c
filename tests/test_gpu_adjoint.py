"""GPU adjoint (pt_adjoint_forward / pt_adjoint through the C ABI) against the CPU adjoint of
the oracle side and against finite differences of the GPU forward.

Objective: J = sum (phi^N - phi_target)^2 of the porosity after N implicit steps, gradient
with respect to the log-permeability prefactor field (k = k0 e^logk (phi/phi0)^3, Eq. 23).
Bars: the GPU gradient equals the dense-LU CPU adjoint to 1e-6 of its largest entry (both
solve the same transposed systems; the GPU's by pseudo-transient iteration to 1e-12 of the
right-hand side, its forward to 1e-12); directional derivatives match central differences of
the GPU forward to 1e-4 relative along 8 directions; one application of the transposed
stencils equals the CPU residual's autograd vector-Jacobian product to 1e-12 element by
element (and <J v, w> = <v, J^T w>); checkpoint spacing changes nothing (bitwise).
"""
import numpy as np
import pytest

import pt_inputs as I

pytestmark = pytest.mark.gpu


def _torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _params(dims, tol=1e-12, powerlaw=False):
    from oracle import adjoint as A
    p = A.adjoint_params(I.c1_params(*dims), powerlaw)
    p["precision"] = 0
    p["tol"] = tol
    p["max_iter"] = 400000
    return p


def _gpu_gradient(p, phi, theta, target, nsteps, every):
    from paper_2207_08716_gb300.solver import PTSolver
    s = PTSolver(p, phi, logk=theta)
    reps = s.adjoint_forward(nsteps, every)
    assert all(r["status"] == 0 for r in reps), reps
    phiN = s.get("phi")
    g, rep = s.adjoint(2.0 * (phiN - target))
    assert rep["status"] == 0, rep
    out = g.cpu().numpy()
    after = s.get("phi")
    s.close()
    return out, phiN, after, rep


def _gpu_misfit(p, phi, theta, target, nsteps):
    from paper_2207_08716_gb300.solver import PTSolver
    s = PTSolver(p, phi, logk=theta)
    for _ in range(nsteps):
        s.step(raise_on_notconv=True)
    J = float(np.sum((s.get("phi") - target) ** 2))
    s.close()
    return J


def test_gpu_adjoint_equals_cpu_adjoint():
    _torch()
    from oracle import adjoint as A
    dims, N = (6, 5, 7), 3
    p = _params(dims)
    rng = np.random.default_rng(0)
    phi = I.gaussian_porosity(p, centres=((0.45, 0.55, 0.5),), width=0.3)
    theta = 0.3 * rng.standard_normal(phi.shape)
    target = A.forward(p, phi, theta + 0.5 * rng.standard_normal(phi.shape), N)[-1]["phi"]
    states = A.forward(p, phi, theta, N)
    ref = A.gradient(p, states, theta, target)
    got, phiN, after, rep = _gpu_gradient(p, phi, theta, target, N, 2)
    np.testing.assert_allclose(phiN, states[-1]["phi"], rtol=1e-11, atol=0)
    np.testing.assert_array_equal(after, phiN)          # the context is left at step N
    err = np.abs(got - ref).max() / np.abs(ref).max()
    assert err <= 1e-6, (err, rep)


def test_gpu_adjoint_matches_finite_differences_32():
    _torch()
    dims, N = (32, 32, 32), 4
    p = _params(dims, tol=1e-11)
    phi = I.gaussian_porosity(p, centres=((0.5, 0.5, 0.4),))
    theta = I.gaussian_random_field(phi.shape, seed=3, corr_len=0.1, std=0.5)
    target_theta = I.gaussian_random_field(phi.shape, seed=4, corr_len=0.1, std=0.5)
    from paper_2207_08716_gb300.solver import PTSolver
    s = PTSolver(p, phi, logk=target_theta)
    for _ in range(N):
        s.step(raise_on_notconv=True)
    target = s.get("phi")
    s.close()
    grad, _, _, rep = _gpu_gradient(p, phi, theta, target, N, 2)
    assert np.abs(grad).max() > 0
    eps = 1e-3
    for d in range(8):
        v = I.gaussian_random_field(phi.shape, seed=10 + d, corr_len=0.1, std=1.0)
        Jp = _gpu_misfit(p, phi, theta + eps * v, target, N)
        Jm = _gpu_misfit(p, phi, theta - eps * v, target, N)
        fd = (Jp - Jm) / (2 * eps)
        ad = float(np.sum(grad * v))
        assert abs(ad - fd) <= 1e-4 * abs(fd), (d, ad, fd, rep)


def test_transposed_stencils_equal_cpu_vjp():
    """pt_adjoint_apply (J_F^T lam on the GPU's transposed stencils) against the CPU adjoint's
    residual differentiated by autograd: element by element, and the dot-product identity
    <J v, w> = <v, J^T w> with J v from forward-mode differentiation."""
    torch = _torch()
    from oracle import adjoint as A
    from paper_2207_08716_gb300.solver import PTSolver
    dims = (13, 10, 9)
    p = _params(dims, tol=1e-9)
    nx, ny, nz = dims
    phi = I.gaussian_porosity(p, centres=((0.4, 0.55, 0.5),), width=0.2)
    theta = I.gaussian_random_field(phi.shape, seed=5, std=0.5)
    s = PTSolver(p, phi, logk=theta)
    s.step()
    u = {k: A._t(s.get(k)) for k in A.U_KEYS}
    rng = np.random.default_rng(11)
    shapes = I.field_shapes(nx, ny, nz)

    def rand_vec():
        v = {k: rng.standard_normal(shapes.get(k, shapes["centre"])) for k in A.U_KEYS}
        v["Vx"][:, :, 0] = v["Vx"][:, :, -1] = 0.0
        v["Vy"][:, 0, :] = v["Vy"][:, -1, :] = 0.0
        v["Vz"][0] = v["Vz"][-1] = 0.0
        return v

    w = rand_vec()
    got = s.adjoint_apply(w)
    old = dict(Pto=torch.zeros_like(u["Pt"]), Pfo=torch.zeros_like(u["Pt"]), Lo=torch.zeros_like(u["Pt"]))
    uu = {k: v.clone().requires_grad_(True) for k, v in u.items()}
    F = A.residual(p, uu, old, A._t(theta))
    wi = {"Fx": w["Vx"][:, :, 1:-1], "Fy": w["Vy"][:, 1:-1, :], "Fz": w["Vz"][1:-1], "Fpt": w["Pt"],
          "Fpf": w["Pf"], "FL": w["phi"]}
    dot = sum((F[k] * A._t(wi[k])).sum() for k in A.F_KEYS)
    grads = torch.autograd.grad(dot, [uu[k] for k in A.U_KEYS])
    ref = dict(zip(A.U_KEYS, (g.numpy() for g in grads)))
    inner = {"Vx": (slice(None), slice(None), slice(1, -1)), "Vy": (slice(None), slice(1, -1), slice(None)),
             "Vz": (slice(1, -1),)}
    for k in A.U_KEYS:
        sl = inner.get(k, (slice(None),))
        a, r = got[k][sl], ref[k][sl]
        err = np.abs(a - r).max() / max(np.abs(r).max(), 1e-300)
        assert err <= 1e-12, (k, err)
    for k, sl in inner.items():                       # wall faces are not unknowns: zero
        full = np.zeros_like(got[k])
        full[sl] = got[k][sl]
        np.testing.assert_array_equal(got[k], full)
    # dot-product test with a forward-mode J v
    v = rand_vec()

    def Fu(*xs):
        d = residual_in(xs)
        return tuple(d[k] for k in A.F_KEYS)

    def residual_in(xs):
        return A.residual(p, dict(zip(A.U_KEYS, xs)), old, A._t(theta))

    _, Jv = torch.autograd.functional.jvp(Fu, tuple(u[k] for k in A.U_KEYS), tuple(A._t(v[k]) for k in A.U_KEYS))
    lhs = sum(float((Jv[i] * A._t(wi[k])).sum()) for i, k in enumerate(A.F_KEYS))
    vi = {k: v[k][inner.get(k, (slice(None),))] for k in A.U_KEYS}
    gi = {k: got[k][inner.get(k, (slice(None),))] for k in A.U_KEYS}
    rhs = sum(float(np.sum(vi[k] * gi[k])) for k in A.U_KEYS)
    scale = sum(float(np.sum(np.abs(vi[k] * gi[k]))) for k in A.U_KEYS)
    assert abs(lhs - rhs) <= 1e-12 * scale, (lhs, rhs, scale)
    s.close()


def test_checkpoint_spacing_changes_nothing():
    _torch()
    dims, N = (12, 10, 14), 4
    p = _params(dims, tol=1e-10)
    phi = I.gaussian_porosity(p, centres=((0.4, 0.5, 0.5),), width=0.2)
    theta = I.gaussian_random_field(phi.shape, seed=1, std=0.3)
    target = phi * 0.99
    g1, *_ = _gpu_gradient(p, phi, theta, target, N, 1)
    g4, *_ = _gpu_gradient(p, phi, theta, target, N, 4)
    g3, *_ = _gpu_gradient(p, phi, theta, target, N, 3)
    np.testing.assert_array_equal(g1, g4)
    np.testing.assert_array_equal(g3, g4)


def test_autograd_function_gives_the_adjoint_gradient():
    torch = _torch()
    from paper_2207_08716_gb300.adjoint import evolve
    dims, N = (16, 12, 10), 3
    p = _params(dims, tol=1e-10)
    phi = I.gaussian_porosity(p, centres=((0.5, 0.5, 0.5),), width=0.2)
    theta = I.gaussian_random_field(phi.shape, seed=2, std=0.3)
    target = torch.as_tensor(phi * 0.995, device="cuda")
    logk = torch.tensor(theta, dtype=torch.float64, device="cuda", requires_grad=True)
    phiN = evolve(logk, p, phi, N, 2)
    J = ((phiN - target) ** 2).sum()
    J.backward()
    ref, *_ = _gpu_gradient(p, phi, theta, target.cpu().numpy(), N, 2)
    np.testing.assert_array_equal(logk.grad.cpu().numpy(), ref)


def test_adjoint_scope_is_enforced():
    _torch()
    from paper_2207_08716_gb300 import native as Nn
    from paper_2207_08716_gb300.solver import PTError, PTSolver
    p = I.c1_params(8, 8, 8)                       # weakening on (R_weak = 0.01): outside the scope
    phi = I.gaussian_porosity(p)
    s = PTSolver(p, phi)
    with pytest.raises(PTError) as e:
        s.adjoint_forward(2, 1)
    assert e.value.code == Nn.PT_EINVAL
    with pytest.raises(PTError) as e:               # no recorded forward
        s.adjoint(np.zeros_like(phi))
    assert e.value.code == Nn.PT_EINVAL
    s.close()
    q = _params((8, 8, 8), tol=1e-8)
    s = PTSolver(q, phi)
    s.step()                                        # not fresh: the window must start at step 0
    with pytest.raises(PTError):
        s.adjoint_forward(2, 1)
    s.close()


# ------------------------------------------------------------------ power law (Eq. 24) on
def test_transposed_stencils_with_power_law_equal_cpu_vjp():
    """With mu an unknown (Picard fixed-point row): pt_adjoint_apply against autograd's VJP of
    the CPU residual, all seven components element by element, and the dot-product identity."""
    torch = _torch()
    from oracle import adjoint as A
    from paper_2207_08716_gb300.solver import PTSolver
    dims = (13, 10, 9)
    p = _params(dims, tol=1e-9, powerlaw=True)
    nx, ny, nz = dims
    phi = I.gaussian_porosity(p, centres=((0.4, 0.55, 0.5),), width=0.2)
    theta = I.gaussian_random_field(phi.shape, seed=5, std=0.5)
    s = PTSolver(p, phi, logk=theta)
    s.step()
    UK, FK = A.U_KEYS_PL, A.F_KEYS_PL
    u = {k: A._t(s.get(k)) for k in UK}
    assert float(u["mu"].min()) < 0.9 * p["mu0"]            # the power law acts on this state
    rng = np.random.default_rng(11)
    shapes = I.field_shapes(nx, ny, nz)

    def rand_vec():
        v = {k: rng.standard_normal(shapes.get(k, shapes["centre"])) for k in UK}
        v["Vx"][:, :, 0] = v["Vx"][:, :, -1] = 0.0
        v["Vy"][:, 0, :] = v["Vy"][:, -1, :] = 0.0
        v["Vz"][0] = v["Vz"][-1] = 0.0
        return v

    w = rand_vec()
    got = s.adjoint_apply(w)
    z = torch.zeros_like(u["Pt"])
    # the step began from mu = mu0 everywhere: its dtS is mu0 / (G xsi_w)
    old = dict(Pto=z, Pfo=z, Lo=z, mu_o=torch.full_like(u["Pt"], p["mu0"]))
    uu = {k: v.clone().requires_grad_(True) for k, v in u.items()}
    F = A.residual(p, uu, old, A._t(theta))
    wi = {"Fx": w["Vx"][:, :, 1:-1], "Fy": w["Vy"][:, 1:-1, :], "Fz": w["Vz"][1:-1], "Fpt": w["Pt"],
          "Fpf": w["Pf"], "FL": w["phi"], "Fmu": w["mu"]}
    dot = sum((F[k] * A._t(wi[k])).sum() for k in FK)
    grads = torch.autograd.grad(dot, [uu[k] for k in UK])
    ref = dict(zip(UK, (g.numpy() for g in grads)))
    inner = {"Vx": (slice(None), slice(None), slice(1, -1)), "Vy": (slice(None), slice(1, -1), slice(None)),
             "Vz": (slice(1, -1),)}
    for k in UK:
        sl = inner.get(k, (slice(None),))
        a, r = got[k][sl], ref[k][sl]
        err = np.abs(a - r).max() / max(np.abs(r).max(), 1e-300)
        assert err <= 1e-12, (k, err)
    v = rand_vec()

    def Fu(*xs):
        d = A.residual(p, dict(zip(UK, xs)), old, A._t(theta))
        return tuple(d[k] for k in FK)

    _, Jv = torch.autograd.functional.jvp(Fu, tuple(u[k] for k in UK), tuple(A._t(v[k]) for k in UK))
    lhs = sum(float((Jv[i] * A._t(wi[k])).sum()) for i, k in enumerate(FK))
    vi = {k: v[k][inner.get(k, (slice(None),))] for k in UK}
    gi = {k: got[k][inner.get(k, (slice(None),))] for k in UK}
    rhs = sum(float(np.sum(vi[k] * gi[k])) for k in UK)
    scale = sum(float(np.sum(np.abs(vi[k] * gi[k]))) for k in UK)
    assert abs(lhs - rhs) <= 1e-12 * scale, (lhs, rhs, scale)
    s.close()


def test_gpu_adjoint_with_power_law_equals_cpu_adjoint():
    """Three converged steps with the power law on (mu falls to 0.1-0.3 mu0): the GPU gradient
    equals the dense-LU CPU adjoint's, which includes the dtS = max(mu_prev) / (G xsi_w) carry."""
    _torch()
    from oracle import adjoint as A
    dims, N = (6, 5, 7), 3
    p = _params(dims, powerlaw=True)
    rng = np.random.default_rng(0)
    phi = I.gaussian_porosity(p, centres=((0.45, 0.55, 0.5),), width=0.3)
    theta = 0.3 * rng.standard_normal(phi.shape)
    target = A.forward(p, phi, theta + 0.5 * rng.standard_normal(phi.shape), N)[-1]["phi"]
    states = A.forward(p, phi, theta, N)
    ref = A.gradient(p, states, theta, target)
    got, phiN, after, rep = _gpu_gradient(p, phi, theta, target, N, 2)
    np.testing.assert_allclose(phiN, states[-1]["phi"], rtol=1e-10, atol=0)
    np.testing.assert_array_equal(after, phiN)
    err = np.abs(got - ref).max() / np.abs(ref).max()
    assert err <= 1e-6, (err, rep)


def test_gpu_adjoint_with_power_law_matches_finite_differences_32():
    _torch()
    dims, N = (32, 32, 32), 4
    p = _params(dims, tol=1e-11, powerlaw=True)
    phi = I.gaussian_porosity(p, centres=((0.5, 0.5, 0.4),))
    theta = I.gaussian_random_field(phi.shape, seed=3, corr_len=0.1, std=0.5)
    target_theta = I.gaussian_random_field(phi.shape, seed=4, corr_len=0.1, std=0.5)
    from paper_2207_08716_gb300.solver import PTSolver
    s = PTSolver(p, phi, logk=target_theta)
    for _ in range(N):
        s.step(raise_on_notconv=True)
    target = s.get("phi")
    s.close()
    grad, _, _, rep = _gpu_gradient(p, phi, theta, target, N, 2)
    assert np.abs(grad).max() > 0
    # dtS = max(mu_prev) / (G xsi_w) is not smooth where the cell holding the maximum changes: on
    # this run the two largest mu of step 2 differ by 3e-5 relative, and a perturbation of 1e-3
    # along some directions moves the maximum to the other cell (central differences then mix two
    # one-sided derivatives; measured 2.6e-3 off, against 2e-8 at eps = 1e-4 and 5e-10 at 3e-5)
    eps = 1e-4
    for d in range(8):
        v = I.gaussian_random_field(phi.shape, seed=10 + d, corr_len=0.1, std=1.0)
        Jp = _gpu_misfit(p, phi, theta + eps * v, target, N)
        Jm = _gpu_misfit(p, phi, theta - eps * v, target, N)
        fd = (Jp - Jm) / (2 * eps)
        ad = float(np.sum(grad * v))
        assert abs(ad - fd) <= 1e-4 * abs(fd), (d, ad, fd, rep)
