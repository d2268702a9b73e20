"""Differentiable Helmholtz solve p = H^(theta)^-1 b.

Backward (adjoint): H^ is symmetric, so lambda = H^^-1 (dL/dp) is one more
solve with the same V-cycle preconditioner; dL/db = lambda and
dL/dtheta_K = -lambda^T (dH^/dtheta_K) p, which only involves the two vertical
faces of cell K and is evaluated by the library's face-contraction kernel.
Only p (and theta) are saved; the operator is re-assembled from theta in the
backward pass.
"""
import torch


class HelmholtzSolve(torch.autograd.Function):
    """p = HelmholtzSolve.apply(hierarchy, b, theta, solve_kwargs, backward_kwargs)

    b, theta: FP64 CUDA tensors over the finest level's cells (COLUMN layout);
    theta may be None (then no gradient for it).  solve_kwargs /
    backward_kwargs are passed to Hierarchy.solve for the forward and the
    adjoint solve.
    """

    @staticmethod
    def forward(ctx, hierarchy, b, theta, solve_kwargs=None, backward_kwargs=None):
        solve_kwargs = dict(solve_kwargs or {})
        hierarchy.assemble(theta=theta)
        p, info = hierarchy.solve(b, **solve_kwargs)
        ctx.hierarchy = hierarchy
        ctx.backward_kwargs = dict(backward_kwargs or solve_kwargs)
        ctx.info = info
        ctx.save_for_backward(p, theta if theta is not None else torch.empty(0))
        ctx.has_theta = theta is not None
        return p

    @staticmethod
    def backward(ctx, grad_p):
        p, theta = ctx.saved_tensors
        h = ctx.hierarchy
        h.assemble(theta=theta if ctx.has_theta else None)
        lam, _ = h.solve(grad_p.contiguous(), **ctx.backward_kwargs)
        grad_theta = h.theta_grad(p, lam) if (ctx.has_theta and ctx.needs_input_grad[2]) else None
        grad_b = lam if ctx.needs_input_grad[1] else None
        return None, grad_b, grad_theta, None, None
