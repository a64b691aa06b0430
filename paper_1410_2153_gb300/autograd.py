"""Differentiable solve: u = A(a)^{-1} b as a torch.autograd.Function.

The forward pass is the ASMG-preconditioned CG solve of the C ABI.  The
backward pass solves the adjoint system A lambda = dL/du with the same
solver (A is symmetric) and forms the element sensitivities with the
library's per-element kernel:
    dL/da_e = -lambda_e^T K_e^(1) u_e,   dL/db = lambda,
or, for the log-parametrisation a = exp(g) (LogSolveFn), the same kernel with
the chain-rule factor a_e applied on the device: dL/dg_e = a_e dL/da_e.
Coefficient updates rebuild the coefficient-dependent operators
(amg_update_coefficients, amg_set_log_coefficients); the geometry-only setup
is reused.  This module only marshals tensors: every step of the solve and
of the gradient runs in the library.
"""
from __future__ import annotations

import torch

from . import asmg


class CoefficientSolver:
    """A Solver whose element coefficients can change between solves."""

    def __init__(self, mesh, precision: int = asmg.ASMG_MIXED, rtol: float = 1e-8, **overrides):
        self.solver = asmg.Solver(mesh, precision=precision, **overrides)
        self.rtol = rtol
        self._set = None          # (kind, device copy) of the coefficients the handle holds
        self.free = torch.from_numpy(mesh.bflag == 0)
        self.last_iterations = []

    def _changed(self, kind: str, c: torch.Tensor) -> bool:
        # compared on the device: no copy of the coefficient field to the host
        return self._set is None or self._set[0] != kind or not torch.equal(self._set[1], c)

    def set_coefficients(self, coeff: torch.Tensor):
        c = coeff.detach().to(torch.float64).contiguous()
        if self._changed("a", c):
            asmg.amg_update_coefficients(self.solver.h, c)
            self._set = ("a", c.clone())

    def set_log_coefficients(self, g: torch.Tensor):
        c = g.detach().to(torch.float64).contiguous()
        if self._changed("g", c):
            asmg.amg_set_log_coefficients(self.solver.h, c)
            self._set = ("g", c.clone())

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


class LogSolveFn(torch.autograd.Function):
    """u = LogSolveFn.apply(g, b, cs) with a = exp(g): g [ne], b [nv] (CUDA float64)."""

    @staticmethod
    def forward(ctx, g, b, cs: CoefficientSolver):
        cs.set_log_coefficients(g)
        u = cs.solve(b)
        ctx.save_for_backward(u)
        ctx.cs = cs
        return u

    @staticmethod
    def backward(ctx, grad_u):
        (u,) = ctx.saved_tensors
        cs = ctx.cs
        lam = cs.solve(grad_u.to(torch.float64).contiguous())      # adjoint: A lambda = dL/du
        dg = cs.solver.element_grad_log(u, lam)                      # dL/dg_e = -a_e lambda_e^T K_e^(1) u_e
        return dg, lam, None


def inversion_loss_and_grad(cs: CoefficientSolver, g: torch.Tensor, b: torch.Tensor, u_obs: torch.Tensor):
    """L = 1/2 ||u(exp g) - u_obs||^2 over free dofs and dL/dg (one forward and one adjoint solve).

    The misfit is the caller's loss; the solves, exp(g) and the chain rule run in the library."""
    g = g.detach().clone().requires_grad_(True)
    u = LogSolveFn.apply(g, b, cs)
    free = cs.free.to(u.device)
    loss = 0.5 * ((u - u_obs)[free] ** 2).sum()
    loss.backward()
    return loss.detach(), g.grad.detach(), u.detach()
