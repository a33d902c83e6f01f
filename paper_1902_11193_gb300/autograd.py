"""torch.autograd wrappers of the permeability solve.

    k = permeability(mask, tau, Lambda, F, set_="E")      # tensors in, scalar out
    k.backward()                                          # tau.grad, Lambda.grad, F.grad

permeability(): forward() runs the forward solve to convergence through the
C ABI (lbm_run_to_convergence) and returns k along the drive direction (the
largest |F_j|); backward() runs the steady fixed-point adjoint (lbm_adjoint)
on the same converged state, so no time history is kept.

transient_permeability(): k after n steps from rest, differentiated through
those n steps (lbm_adjoint_transient).  The library takes k(n) and its
gradient in one checkpointed forward-and-reverse sweep, so forward() runs it
and backward() returns the stored gradient.

All work happens in the library's CUDA kernels; torch only carries the
scalars.
"""
from __future__ import annotations

import numpy as np
import torch

from . import lbm


class PermeabilityFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, tau, Lambda, F, mask, set_, tol, adjoint_tol, options):
        F64 = F.detach().to(torch.float64).cpu().numpy()
        solver = lbm.LBMSolver(mask, set_, float(tau), float(Lambda), tuple(F64), **options)
        rc, _ = solver.run_to_convergence(tol)
        if rc != 0:
            raise lbm.LBMError(rc, "PermeabilityFn forward did not converge")
        d = int(np.argmax(np.abs(F64)))
        k = solver.permeability()[d]
        ctx.solver = solver
        ctx.adjoint_tol = adjoint_tol
        ctx.set_ = set_
        return torch.tensor(k, dtype=torch.float64)

    @staticmethod
    def backward(ctx, grad_k):
        g = ctx.solver.adjoint(ctx.adjoint_tol)
        ctx.solver.close()
        return _grads(g, ctx.set_, grad_k) + (None, None, None, None, None)


def _grads(g, set_, grad_k):
    gk = grad_k.to(torch.float64)
    dLambda = g["dLambda"] if set_ in ("E", lbm.SET_E) else 0.0
    dLambda = 0.0 if np.isnan(dLambda) else dLambda
    return (gk * g["dtau"], gk * dLambda, gk * torch.tensor(g["dF"], dtype=torch.float64))


class TransientPermeabilityFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, tau, Lambda, F, mask, set_, n, options):
        F64 = F.detach().to(torch.float64).cpu().numpy()
        solver = lbm.LBMSolver(mask, set_, float(tau), float(Lambda), tuple(F64), **options)
        try:
            ctx.g = solver.adjoint_transient(int(n))
        finally:
            solver.close()
        ctx.set_ = set_
        return torch.tensor(ctx.g["k"], dtype=torch.float64)

    @staticmethod
    def backward(ctx, grad_k):
        return _grads(ctx.g, ctx.set_, grad_k) + (None, None, None, None)


def permeability(mask, tau, Lambda, F, set_="E", tol=1e-10, adjoint_tol=1e-9, **options):
    """Differentiable permeability k(tau, Lambda, F) of a voxel image.

    tau, Lambda: scalar tensors; F: 3-vector tensor.  Lambda only matters for
    Set E (its gradient is zero for the other sets).  `options` are passed to
    LBMSolver (precision, layout, linear_eq, check_interval, ...)."""
    as_t = lambda v: v if torch.is_tensor(v) else torch.tensor(v, dtype=torch.float64)
    return PermeabilityFn.apply(as_t(tau), as_t(Lambda), as_t(F), mask, set_, tol, adjoint_tol,
                                options)


def transient_permeability(mask, tau, Lambda, F, n, set_="E", **options):
    """Differentiable permeability after n steps from rest, k_n(tau, Lambda, F):
    the value lbm_permeability gives once n steps have run.  Arguments as for
    permeability(); n is the number of steps."""
    as_t = lambda v: v if torch.is_tensor(v) else torch.tensor(v, dtype=torch.float64)
    return TransientPermeabilityFn.apply(as_t(tau), as_t(Lambda), as_t(F), mask, set_, int(n),
                                         options)
