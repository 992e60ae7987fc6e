"""Phi as a torch.autograd.Function whose backward is the CUDA gridding adjoint.

For a real image x and y = Phi x, PyTorch's complex autograd hands backward the
gradient g_y = dL/dRe(y) + i dL/dIm(y); the chain rule through the real-linear
map gives dL/dx = Re(Phi^H g_y), which is exactly pd_apply_phi_adj (gridding
G^T, inverse FFT, crop and pre-compensation, Sec. 2).
"""
import torch


class PhiFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, plan):
        ctx.plan = plan
        return plan.pd_apply_phi(x.contiguous())

    @staticmethod
    def backward(ctx, grad_y):
        plan = ctx.plan
        g = grad_y.contiguous()
        if g.dtype != plan.cplx_dtype:
            g = g.to(plan.cplx_dtype)
        return plan.pd_apply_phi_adj(g), None


def phi(x, plan):
    """y = Phi x with gradient Re(Phi^H g)."""
    return PhiFunction.apply(x, plan)
