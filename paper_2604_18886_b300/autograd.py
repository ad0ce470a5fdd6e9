"""Differentiable octree Poisson solve (torch.autograd.Function over libocg).

The paper has no gradient; this is the adjoint of its solve.  forward(b, beta) sets the
hierarchy up for the face fractions beta (ocg_setup_hierarchy) and solves A p = b by PCG
(Alg. 1).  backward(dL/dp) solves the adjoint system A^T lambda = dL/dp (Alg. 1 on A^T
preconditioned by the transposed cycle M^T, ocg_pcg_solve with OCG_SOLVE_TRANSPOSE) and
returns
    dL/db    = lambda
    dL/dbeta = ocg_face_grad(p, lambda)   (-lambda^T dA/dbeta_f p per face).
Under pure Neumann walls p and lambda are the zero-mean representatives.  Marshalling
only: every arithmetic step runs in libocg's kernels.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import torch

from . import solver as S


@dataclass
class SolveOptions:
    tol: float = 1e-6
    precision: str = "mixed"
    max_iter: int = 200
    adjoint_tol: float | None = None        # defaults to tol
    adjoint_precision: str | None = None    # defaults to precision
    mg: object = field(default_factory=S.mg_params)
    # a hierarchy on the same tree and walls to refresh in place for each beta
    # (ocg_hier_update_beta) instead of setting one up per call; its backward must run
    # before the next forward that uses it
    hierarchy: object = None


class PoissonSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, b, beta, tree, bc, opts):
        beta32 = beta.detach().to(torch.float32).contiguous()
        if opts.hierarchy is not None:
            hier = opts.hierarchy
            hier.update_beta(beta32)
        else:
            hier = S.Hierarchy(tree, beta32, bc, opts.mg)
        p, st = hier.solve(b.detach().to(torch.float64).contiguous(), tol=opts.tol,
                           precision=opts.precision, max_iter=opts.max_iter)
        ctx.hier = hier
        ctx.opts = opts
        ctx.beta_dtype = beta.dtype
        ctx.forward_stats = st
        ctx.save_for_backward(p)
        return p

    @staticmethod
    def backward(ctx, grad_p):
        (p,) = ctx.saved_tensors
        o = ctx.opts
        lam, st = ctx.hier.solve(grad_p.detach().to(torch.float64).contiguous(),
                                 tol=o.adjoint_tol or o.tol,
                                 precision=o.adjoint_precision or o.precision,
                                 max_iter=o.max_iter, transpose=True)
        dbeta = ctx.hier.face_grad(p, lam)
        return lam, dbeta.to(ctx.beta_dtype), None, None, None


def poisson_solve(b, beta, tree, bc, **kw):
    """p = A(beta)^{-1} b on `tree` (solver.Octree) with wall codes `bc`; differentiable
    in b (float64, canonical leaf order) and beta (canonical face order).  Keywords: the
    fields of SolveOptions (hierarchy=h reuses h, refreshed for each beta)."""
    return PoissonSolve.apply(b, beta, tree, tuple(bc), SolveOptions(**kw))
