"""Differentiable BDDC-PCG solve: u(sigma) = A(sigma)^-1 b with gradients by
the adjoint method.

forward   setup of the BDDC preconditioner for the element conductivities
          sigma (host, float64), then u = A(sigma)^-1 b by BDDC-PCG (library).
backward  lambda = A^-1 (dL/du) by a second BDDC-PCG solve on the same
          handle (A is symmetric), then
              dL/dsigma_e = - sum_k lambda_k,e^T K_ref u_k,e
          (library kernel `bddc_elem_grad`), and dL/db = lambda.

For L = J(sigma) = 1/2 ||u - u_obs||^2 the upstream gradient dL/du is
u - u_obs, so backward computes exactly the adjoint gradient of J. Vectors
hold all (ne+1)^dim nodes; Dirichlet entries of b and of dL/du are ignored
and those of u and lambda are 0.
"""
from __future__ import annotations

import numpy as np

from . import BDDC


def _function():
    import torch

    class _Solve(torch.autograd.Function):
        @staticmethod
        def forward(ctx, sigma, b, dim, ne, elem_subdomain, n_sub, rtol, maxit, options):
            sig = sigma.detach().to("cpu", torch.float64).contiguous().numpy()
            nrhs = 1 if b.dim() == 1 else int(b.shape[1])
            h = BDDC(dim, ne, sig, np.asarray(elem_subdomain, dtype=np.int32), n_sub, nrhs_max=nrhs, **options)
            u, res = h.pcg_solve(b.detach().contiguous(), rtol=rtol, maxit=maxit)
            if res.status != 0:
                raise RuntimeError(f"BDDC-PCG forward solve: status {res.status}, iterations {list(res.iters)}")
            ctx.h, ctx.rtol, ctx.maxit = h, rtol, maxit
            ctx.sigma_device, ctx.sigma_dtype = sigma.device, sigma.dtype
            ctx.forward_iters = list(res.iters)
            ctx.save_for_backward(u)
            return u

        @staticmethod
        def backward(ctx, gu):
            (u,) = ctx.saved_tensors
            lam, res = ctx.h.pcg_solve(gu.detach().contiguous(), rtol=ctx.rtol, maxit=ctx.maxit)
            if res.status != 0:
                raise RuntimeError(f"BDDC-PCG adjoint solve: status {res.status}, iterations {list(res.iters)}")
            g = ctx.h.elem_grad(u, lam)
            return (g.to(ctx.sigma_device, ctx.sigma_dtype), lam, None, None, None, None, None, None, None)

    return _Solve


_SOLVE = None


def solve(sigma, b, dim: int, ne: int, elem_subdomain, n_sub: int, rtol: float = 1e-8, maxit: int = 1000,
          **options):
    """u = A(sigma)^-1 b, differentiable in sigma (any device, float64 values
    > 0, length ne^dim) and in b (CUDA float64, [n_nodes] or [n_nodes, nrhs]).

    `options` go to `BDDC` (precision, constraints, coarse, tensor_cores, ...).
    Each call sets the preconditioner up for the given sigma.
    """
    global _SOLVE
    if _SOLVE is None:
        _SOLVE = _function()
    return _SOLVE.apply(sigma, b, dim, ne, elem_subdomain, n_sub, rtol, maxit, options)
