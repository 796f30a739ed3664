"""Implicit-adjoint autograd for screened Poisson solves.

Forward solves A(sigma) u_b = f_b for a batch of right-hand sides through
hj_solve.  Backward runs the adjoint through hj_solve_adjoint with the same
handle (same cycles and precision).  That call solves A^T lambda_b = dL/du_b
and forms dL/df_b = lambda_b and dL/dsigma = -sum_b lambda_b * u_b in one fused
kernel.  No iterate of the forward solve is stored: memory is O(grid).

Tensors use the library's padded grid layout (``alloc_grid``): f is
(B, rows, ld) or (rows, ld) float64 on the GPU, with zero Dirichlet data on the
ghost ring; sigma is (rows, ld) float64 (ghost entries ignored) or None.
"""
from __future__ import annotations

import torch

from . import (HJ_ERR_NOT_CONVERGED, HJ_OK, HJ_PREC_BF16CORR_IR, HJ_PREC_F32_IR, HJError, Solver,
               _stream_handle, hj_solve_adjoint_batched, hj_solve_batched, make_params)


def _batchable(solver, nrhs):
    # several right-hand sides of one 2D refinement solve share persistent launches
    return nrhs > 1 and solver.dim == 2 and solver.params.precision in (HJ_PREC_F32_IR, HJ_PREC_BF16CORR_IR)


class HJSolve(torch.autograd.Function):
    """u = HJSolve.apply(f, sigma, stencil, params).

    stencil: object with dim, nx, ny, cW, cE, cS, cN, cD, sigma_const
    params:  an hj_params (see make_params); tol applies to both the forward
             solve and the adjoint solve."""

    @staticmethod
    def forward(ctx, f, sigma, stencil, params):
        batched = f.dim() == 3
        fb = f if batched else f.unsqueeze(0)
        solver = Solver(stencil, params, sigma=None if sigma is None else sigma.detach().contiguous())
        u = torch.zeros_like(fb)
        fd = fb.detach().contiguous()
        if _batchable(solver, fb.shape[0]):
            code = hj_solve_batched(solver.h, [solver.desc] * fb.shape[0], [fd[b].data_ptr() for b in range(fb.shape[0])],
                                    [u[b].data_ptr() for b in range(fb.shape[0])], _stream_handle(None))
            if code not in (HJ_OK, HJ_ERR_NOT_CONVERGED):
                raise HJError(code, "HJSolve forward (batched)")
        else:
            for b in range(fb.shape[0]):
                out = solver.solve(fd[b], u[b], check=False)
                if out["status"] not in (HJ_OK, HJ_ERR_NOT_CONVERGED):
                    raise HJError(out["status"], "HJSolve forward")
        ctx.solver = solver
        ctx.batched = batched
        ctx.has_sigma = sigma is not None
        ctx.save_for_backward(u)
        return u if batched else u[0]

    @staticmethod
    def backward(ctx, grad_u):
        (u,) = ctx.saved_tensors
        solver = ctx.solver
        g = grad_u if ctx.batched else grad_u.unsqueeze(0)
        g = g.contiguous()
        dl_df = torch.zeros_like(u)
        dl_dsig = None
        dsig_b = None
        if ctx.has_sigma and ctx.needs_input_grad[1]:
            dl_dsig = torch.zeros_like(u[0])
            dsig_b = torch.zeros_like(u[0])
        B = u.shape[0]
        if _batchable(solver, B):
            code = hj_solve_adjoint_batched(solver.h, [g[b].data_ptr() for b in range(B)],
                                            [u[b].data_ptr() for b in range(B)],
                                            [dl_df[b].data_ptr() for b in range(B)],
                                            0 if dl_dsig is None else dl_dsig.data_ptr(), _stream_handle(None))
            if code not in (HJ_OK, HJ_ERR_NOT_CONVERGED):
                raise HJError(code, "HJSolve backward (batched)")
        else:
            for b in range(B):
                out = solver.adjoint(g[b], u[b], dl_df[b], dsig_b, check=False)
                if out["status"] not in (HJ_OK, HJ_ERR_NOT_CONVERGED):
                    raise HJError(out["status"], "HJSolve backward")
                if dsig_b is not None:
                    dl_dsig += dsig_b
        solver.close()
        ctx.solver = None
        grad_f = dl_df if ctx.batched else dl_df[0]
        return (grad_f if ctx.needs_input_grad[0] else None), dl_dsig, None, None


def solve_screened(f, sigma, stencil, **params):
    """Differentiable solve of A(sigma) u = f (see HJSolve)."""
    return HJSolve.apply(f, sigma, stencil, make_params(**params))
