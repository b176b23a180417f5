"""Differentiable pressure solve: p = A(log k)^{-1} q with an adjoint backward pass.

``pressure(logk, q, grid)`` assembles the two-point-flux matrix on the GPU, builds the
combined-preconditioned solver and solves A p = q.  Its backward pass solves the adjoint system
A lambda = dJ/dp with the same solver handle (A is symmetric) and contracts with dA/dlog k in one
CUDA kernel (cpc_tpfa_gradient), so dJ/dlog k for any scalar loss J(p) built from torch ops costs
one extra solve.  dJ/dq = lambda is returned as well.  All steps run in libcpc.so.
"""
from __future__ import annotations

from dataclasses import dataclass

import torch

from . import cpc


@dataclass(frozen=True)
class Grid:
    nx: int
    ny: int
    nz: int
    kz_ratio: float
    dirichlet: int


class PressureSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, logk, q, grid: Grid, tol: float, maxit: int, options: dict):
        rowptr, col, val = cpc.tpfa_assemble(grid.nx, grid.ny, grid.nz, logk, grid.kz_ratio, grid.dirichlet)
        solver = cpc.Solver(rowptr, col, val, **options)
        p, iters, status, _ = solver.solve(q.contiguous(), tol=tol, maxit=maxit, hist=False)
        if status != 0:
            raise cpc.CpcError(status, "forward pressure solve")
        ctx.save_for_backward(logk, p)
        ctx.solver, ctx.grid, ctx.tol, ctx.maxit = solver, grid, tol, maxit
        ctx.iters = [iters]
        return p

    @staticmethod
    def backward(ctx, grad_p):
        logk, p = ctx.saved_tensors
        g = ctx.grid
        lam, iters, status, _ = ctx.solver.solve(grad_p.contiguous(), tol=ctx.tol, maxit=ctx.maxit, hist=False)
        if status != 0:
            raise cpc.CpcError(status, "adjoint solve")
        ctx.iters.append(iters)
        grad_logk = cpc.tpfa_gradient(g.nx, g.ny, g.nz, logk, g.kz_ratio, g.dirichlet, lam, p)
        return grad_logk, lam, None, None, None, None


def pressure(logk: torch.Tensor, q: torch.Tensor, grid: Grid, tol: float = 1e-10, maxit: int = 2000,
             **options) -> torch.Tensor:
    """Pressure p solving A(logk) p = q; differentiable in logk and q.  options go to cpc.Solver
    (default: the combined preconditioner with the red-black IC(0) ordering)."""
    opts = dict(precond="bco", ic_order="colour")
    opts.update(options)
    return PressureSolve.apply(logk, q, grid, tol, maxit, opts)


def well_pressures(p: torch.Tensor, well_cells: torch.Tensor) -> torch.Tensor:
    """Mean pressure of each well; well_cells is [nwells, cells_per_well] (device, int64)."""
    return p[well_cells].mean(dim=1)
