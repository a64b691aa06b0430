"""Differentiable solve: u = A(a)^{-1} b as a torch.autograd.Function.

The forward pass is the ASMG-preconditioned CG solve of the C ABI.  The
backward pass solves the adjoint system A lambda = dL/du with the same
solver (A is symmetric) and forms the element sensitivities with the
library's per-element kernel:
    dL/da_e = -lambda_e^T K_e^(1) u_e,   dL/db = lambda.
Coefficient updates rebuild the coefficient-dependent operators
(amg_update_coefficients); the geometry-only setup is reused.
"""
from __future__ import annotations

import numpy as np
import torch

from . import asmg


class CoefficientSolver:
    """A Solver whose element coefficients can change between solves."""

    def __init__(self, mesh, precision: int = asmg.ASMG_MIXED, rtol: float = 1e-8, **overrides):
        self.solver = asmg.Solver(mesh, precision=precision, **overrides)
        self.rtol = rtol
        self._coeff = None if mesh.coeff is None else np.array(mesh.coeff, dtype=np.float64, copy=True)
        self.free = torch.from_numpy(mesh.bflag == 0)
        self.last_iterations = []

    def set_coefficients(self, coeff: torch.Tensor):
        c = coeff.detach().to(torch.float64).contiguous()
        ch = c.cpu().numpy()
        if self._coeff is None or not np.array_equal(ch, self._coeff):
            asmg.amg_update_coefficients(self.solver.h, c)
            self._coeff = ch.copy()

    def solve(self, b: torch.Tensor) -> torch.Tensor:
        u, rc, it, _ = self.solver.solve(b.contiguous(), rtol=self.rtol)
        self.last_iterations.append(it)
        if rc != asmg.ASMG_OK:
            raise asmg.AsmgError(rc, f"solve did not converge in {it} iterations")
        return u


class SolveFn(torch.autograd.Function):
    """u = SolveFn.apply(coeff, b, cs): coeff [ne], b [nv] (CUDA float64)."""

    @staticmethod
    def forward(ctx, coeff, b, cs: CoefficientSolver):
        cs.set_coefficients(coeff)
        u = cs.solve(b)
        ctx.save_for_backward(u)
        ctx.cs = cs
        return u

    @staticmethod
    def backward(ctx, grad_u):
        (u,) = ctx.saved_tensors
        cs = ctx.cs
        lam = cs.solve(grad_u.to(torch.float64).contiguous())      # adjoint: A lambda = dL/du
        g = cs.solver.element_grad(u, lam)                           # dL/da_e = -lambda_e^T K_e^(1) u_e
        return g, lam, None


def inversion_loss_and_grad(cs: CoefficientSolver, g: torch.Tensor, b: torch.Tensor, u_obs: torch.Tensor):
    """L = 1/2 ||u(exp g) - u_obs||^2 over free dofs and dL/dg (one forward and one adjoint solve)."""
    g = g.detach().clone().requires_grad_(True)
    u = SolveFn.apply(torch.exp(g), b, cs)
    free = cs.free.to(u.device)
    loss = 0.5 * ((u - u_obs)[free] ** 2).sum()
    loss.backward()
    return loss.detach(), g.grad.detach(), u.detach()
