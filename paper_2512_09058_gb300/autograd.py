"""torch.autograd.Function over the cyq factor/solve and its adjoint.

``kkt_solve(solver, Q, R, S, A, B, Sigma, q, r, c, x0)`` returns the KKT
solution z (records [u^k | x^{k+1} | lambda^k]) of every instance in the
solver's batch.  Its backward pass calls ``cyq_solve_adjoint``: K is
symmetric, so w = K^{-1} dL/dz reuses the stored factor, and the gradients
with respect to Q, R, S, A, B, Sigma, q, r, c and x0 are per-stage outer
products of w and z (implicit differentiation of K z = b).  All arithmetic
runs in the CUDA library; this module only wires tensors.

The factor is borrowed from the solver: if the same solver factors another
problem before this node's backward runs, the backward pass factors the
saved inputs again (recomputation instead of keeping one factor per node).
"""
from __future__ import annotations

import torch

from . import cyq

_ORDER = ("Q", "R", "S", "A", "B", "Sigma", "q", "r", "c", "x0")
_GRAD = {"Q": "dQ", "R": "dR", "S": "dS", "A": "dA", "B": "dB", "Sigma": "dSigma",
         "q": "dq", "r": "dr", "c": "dc", "x0": "dx0"}


class KKTSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, solver: "cyq.Solver", Q, R, S, A, B, Sigma, q, r, c, x0):
        args = [t.contiguous() if t is not None else None for t in (Q, R, S, A, B, Sigma, q, r, c, x0)]
        Q, R, S, A, B, Sigma, q, r, c, x0 = args
        solver.factor(Q, R, S, A, B, Sigma)
        b = solver.build_rhs(q, r, c, x0)
        z = solver.solve(b)
        ctx.solver = solver
        ctx.version = solver.factor_version
        ctx.has = [t is not None for t in args]
        ctx.save_for_backward(*[t for t in args if t is not None], z)
        return z

    @staticmethod
    def backward(ctx, gz):
        saved = list(ctx.saved_tensors)
        z = saved.pop()
        it = iter(saved)
        vals = dict(zip(_ORDER, [next(it) if h else None for h in ctx.has]))
        solver = ctx.solver
        if solver.factor_version != ctx.version:
            solver.factor(vals["Q"], vals["R"], vals["S"], vals["A"], vals["B"], vals["Sigma"])
        want = ["w"] + [_GRAD[k] for k, need in zip(_ORDER, ctx.needs_input_grad[1:]) if need]
        g = solver.solve_adjoint(vals["x0"], z, gz.contiguous(), want=tuple(want))
        grads = [g.get(_GRAD[k]) if need else None for k, need in zip(_ORDER, ctx.needs_input_grad[1:])]
        return (None, *grads)


def kkt_solve(solver, Q, R, S, A, B, Sigma, q, r, c, x0):
    """Differentiable batched KKT solve (see module docstring)."""
    return KKTSolve.apply(solver, Q, R, S, A, B, Sigma, q, r, c, x0)
