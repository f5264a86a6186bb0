"""Differentiable P_k solve: u = A(kappa)^{-1} b with a hand-written backward.

A_h (Eq. 7) is symmetric and linear in each element coefficient kappa_e, so for a loss
L(u) with g = dL/du the adjoint solve A_h lambda = g (same operator, same
preconditioner) gives
    dL/db       = lambda
    dL/dkappa_e = -lambda_e^T Khat_e u_e      (Khat_e: element matrix with kappa_e = 1)
Both solves and the element-wise gradient run in libpkasp's CUDA kernels.
"""
from __future__ import annotations

import torch

from .solver import Problem


class PkPoissonSolve(torch.autograd.Function):
    """u = PkPoissonSolve.apply(kappa, b, problem, setup_kwargs)

    kappa: [n_tets] float64 (CUDA or CPU; a CUDA tensor reaches the library as a device
    pointer), b: [n_h] float64 CUDA load vector, or [n_h, ncols] for several right-hand
    sides solved as one block (then dL/dkappa is the sum of the columns' gradients,
    summed by the library, and dL/db the block of adjoint solutions).
    problem: an assembled :class:`Problem`; it is re-assembled for this kappa and its
    preconditioner rebuilt on every forward call.
    """

    @staticmethod
    def forward(ctx, kappa, b, problem: Problem, setup_kwargs=None):
        kw = dict(setup_kwargs or {})
        problem.set_kappa(kappa.detach())
        problem.setup(**kw)
        u, st = problem.solve(b.detach().contiguous())
        ctx.problem = problem
        ctx.stats = st
        ctx.kappa_device = kappa.device
        ctx.kappa_dtype = kappa.dtype
        ctx.save_for_backward(u)
        return u

    @staticmethod
    def backward(ctx, g):
        problem = ctx.problem
        (u,) = ctx.saved_tensors
        lam, _ = problem.solve_adjoint(g.contiguous())
        dkappa = problem.grad_kappa(u, lam)
        return dkappa.to(device=ctx.kappa_device, dtype=ctx.kappa_dtype), lam, None, None


def solve(kappa, b, problem: Problem, **setup_kwargs):
    """Differentiable solve; see :class:`PkPoissonSolve`."""
    return PkPoissonSolve.apply(kappa, b, problem, setup_kwargs)
