"""torch.autograd.Function over the fused forward + adjoint kernels.

The fused kernel already produces the exact gradient together with the
value (reverse mode, Sec. 1-2 of the paper), so forward() runs it once and
keeps the gradient; backward() only scales it by the incoming adjoint.
Only theta is differentiable; the data are constants of the problem.
Second derivatives are not provided (backward is once-differentiable).
"""
import torch
from torch.autograd.function import once_differentiable

from . import cg


class FitObjective(torch.autograd.Function):
    """F(theta) for one parameter vector theta [P]; returns a 0-d tensor."""

    @staticmethod
    def forward(ctx, theta, problem):
        value, grad = cg.gradient(problem, theta.detach().contiguous())
        ctx.save_for_backward(grad)
        return value

    @staticmethod
    @once_differentiable
    def backward(ctx, g_out):
        (grad,) = ctx.saved_tensors
        return g_out * grad, None


class FitObjectiveBatch(torch.autograd.Function):
    """F(theta_h) for H parameter points thetas [H, P] on one problem; returns [H]."""

    @staticmethod
    def forward(ctx, thetas, problem):
        values, grads = cg.batch_gradient(problem, thetas.detach().contiguous())
        ctx.save_for_backward(grads)
        return values

    @staticmethod
    @once_differentiable
    def backward(ctx, g_out):
        (grads,) = ctx.saved_tensors
        return g_out[:, None] * grads, None


def fit_objective(theta, problem):
    """Differentiable objective value: fit_objective(theta, pb).backward() fills theta.grad."""
    if theta.dim() == 1:
        return FitObjective.apply(theta, problem)
    return FitObjectiveBatch.apply(theta, problem)
