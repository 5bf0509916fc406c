"""GPU adjoint (pt_adjoint_forward / pt_adjoint through the C ABI) against the CPU adjoint of
the oracle side and against finite differences of the GPU forward.

Objective: J = sum (phi^N - phi_target)^2 of the porosity after N implicit steps, gradient
with respect to the log-permeability prefactor field (k = k0 e^logk (phi/phi0)^3, Eq. 23).
Bars: the GPU gradient equals the dense-LU CPU adjoint to 1e-6 of its largest entry (both
solve the same transposed systems; the GPU's by pseudo-transient iteration to 1e-12 of the
right-hand side, its forward to 1e-12); directional derivatives match central differences of
the GPU forward to 1e-4 relative; checkpoint spacing changes nothing (bitwise).
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


def _params(dims, tol=1e-12):
    from oracle import adjoint as A
    p = A.adjoint_params(I.c1_params(*dims))
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
    rng = np.random.default_rng(7)
    eps = 1e-3
    for d in range(2):
        v = I.gaussian_random_field(phi.shape, seed=10 + d, corr_len=0.1, std=1.0)
        Jp = _gpu_misfit(p, phi, theta + eps * v, target, N)
        Jm = _gpu_misfit(p, phi, theta - eps * v, target, N)
        fd = (Jp - Jm) / (2 * eps)
        ad = float(np.sum(grad * v))
        assert abs(ad - fd) <= 1e-4 * abs(fd), (d, ad, fd, rep)
    del rng


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
    p = I.c1_params(8, 8, 8)                       # power law on: outside the adjoint's scope
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
