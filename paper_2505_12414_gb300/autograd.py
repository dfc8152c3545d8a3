"""torch.autograd.Function around the fused NLL+gradient kernel.

forward(theta) runs nll_eval_grad once (the kernel computes the analytic gradient in the
same pass as the NLL, paper Sec. 2.1 and 2.2) and keeps dNLL/dtheta; backward returns
grad_output * dNLL/dtheta.  Marshalling only: the arithmetic is in the CUDA library.
"""
import numpy as np
import torch

from . import nll_eval_grad


class NLLFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, model_handle):
        th = theta.detach().to("cpu", torch.float64).numpy()
        nll, grad = nll_eval_grad(model_handle, th)
        ctx.save_for_backward(torch.from_numpy(np.asarray(grad)).to(theta.device, theta.dtype))
        return theta.new_tensor(nll)

    @staticmethod
    def backward(ctx, grad_output):
        (g,) = ctx.saved_tensors
        return grad_output * g, None


def nll(model, theta):
    """NLL(theta) of a Model (or raw handle) as a differentiable torch scalar."""
    handle = getattr(model, "handle", model)
    return NLLFunction.apply(theta, handle)
