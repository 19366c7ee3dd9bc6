"""torch.autograd.Function over the hand-written adjoint kernel (goo_nll_grad).

forward(theta) calls goo_nll_grad once and saves the gradient; backward returns
grad_output * dNLL/dtheta.  theta is a CPU float64 tensor (the minimiser's vector).
"""
import numpy as np
import torch

from .goo import precision_code


class GooNLL(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, model, dataset, precision="f32"):
        th = theta.detach().to("cpu", torch.float64).numpy()
        nll, g = model.nll_grad(dataset, th, precision_code(precision))
        ctx.save_for_backward(torch.from_numpy(np.asarray(g)).to(theta.dtype))
        return theta.new_tensor(nll)

    @staticmethod
    def backward(ctx, grad_output):
        (g,) = ctx.saved_tensors
        return grad_output * g.to(grad_output.device), None, None, None


def nll(theta, model, dataset, precision="f32"):
    return GooNLL.apply(theta, model, dataset, precision)
