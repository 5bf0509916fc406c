"""Porosity evolution as a differentiable PyTorch function of the log-permeability field.

``evolve(logk, params, phi0, nsteps)`` runs `nsteps` implicit steps of the two-phase solver
(thesis Art. 1, Eqs. 17-27, in the adjoint's scope: no weakening, beta_n = 0; the power law of
Eq. 24 as the parameters set it) on the GPU and returns the porosity after the last step; its backward is the discrete adjoint of
the converged steps (pt_adjoint of the C ABI), so ``torch.autograd`` gives dJ/dlogk for any
objective J of the final porosity. Forward and backward both run in the CUDA library.
"""
from __future__ import annotations

import torch

from .solver import PTSolver


def adjoint_scope(params: dict) -> dict:
    """Parameters restricted to the adjoint's scope: no weakening (R = 1; Eq. 25 is a step
    function), beta_n = 0, no background shear; the power law (Eq. 24) stays as given."""
    q = dict(params)
    q.update(R_weak=1.0, beta_n=0.0, compaction_on=1, tau_bg=0.0)
    return q


class _Evolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, logk, params, phi0, nsteps, ckpt_every):
        solver = PTSolver(adjoint_scope(params), phi0, logk=logk.detach(), device=logk.device)
        ctx.reports = solver.adjoint_forward(nsteps, ckpt_every)
        ctx.solver = solver
        nz, ny, nx = params["nz"], params["ny"], params["nx"]
        torch.cuda.current_stream(logk.device).synchronize()
        return solver.f["phi"][:nz, :ny, :nx].clone()

    @staticmethod
    def backward(ctx, grad_phi):
        grad, rep = ctx.solver.adjoint(grad_phi.detach())
        ctx.adjoint_report = rep
        return grad, None, None, None, None


def evolve(logk: torch.Tensor, params: dict, phi0, nsteps: int, ckpt_every: int | None = None) -> torch.Tensor:
    """Porosity after `nsteps` steps, differentiable w.r.t. `logk` (cell-centred, CUDA, FP64)."""
    if logk.device.type != "cuda" or logk.dtype != torch.float64:
        raise ValueError("logk must be a float64 CUDA tensor")
    return _Evolve.apply(logk, params, phi0, nsteps, ckpt_every)
