"""torch.autograd wrappers of the MW transforms.

The transforms are linear in their complex input, so the vector-Jacobian
product PyTorch needs is the Hermitian adjoint: for y = A x, grad_x = A^H grad_y
(PyTorch's convention for complex tensors: the gradient of a real loss is
dL/dRe + i dL/dIm).  The backward passes call the library's adjoint entry points
(mw_forward_adjoint, mw_inverse_adjoint); the Wigner-Delta planes are recomputed
there, nothing beyond the plan is kept between forward and backward.
"""
import torch

from .mw import Plan


class MWForward(torch.autograd.Function):
    """f_lm = forward(map), differentiable in map."""

    @staticmethod
    def forward(ctx, maps, plan: Plan):
        ctx.plan = plan
        return plan.forward(maps)

    @staticmethod
    def backward(ctx, grad_flm):
        return ctx.plan.forward_adjoint(grad_flm.contiguous()), None


class MWInverse(torch.autograd.Function):
    """map = inverse(f_lm), differentiable in f_lm."""

    @staticmethod
    def forward(ctx, flm, plan: Plan):
        ctx.plan = plan
        return plan.inverse(flm)

    @staticmethod
    def backward(ctx, grad_map):
        return ctx.plan.inverse_adjoint(grad_map.contiguous()), None


def mw_forward(maps, plan: Plan):
    return MWForward.apply(maps, plan)


def mw_inverse(flm, plan: Plan):
    return MWInverse.apply(flm, plan)
