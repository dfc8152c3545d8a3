"""torch.autograd.Function around the fused NLL+gradient kernel and the Hessian pass.

forward(theta) runs nll_eval_grad once (the kernel computes the analytic gradient in the
same pass as the NLL, paper Sec. 2.1 and 2.2) and keeps dNLL/dtheta; backward returns
grad_output * dNLL/dtheta.  With create_graph=True the returned gradient is itself
differentiable: its backward is the Hessian-vector product H v with the analytic Hessian of
nll_eval_hess (Sec. 2.1), so torch.autograd.functional.hessian and double backward work
(twice differentiable; third derivatives are not provided).  Marshalling only: the
arithmetic is in the CUDA library.
"""
import numpy as np
import torch

from . import nll_eval_grad, nll_eval_hess


def _host(theta):
    return theta.detach().to("cpu", torch.float64).numpy()


class _GradFunction(torch.autograd.Function):
    """g(theta) = dNLL/dtheta (already computed by the forward pass); backward: H v."""

    @staticmethod
    def forward(ctx, theta, g, model_handle):
        ctx.save_for_backward(theta)
        ctx.handle = model_handle
        return g.clone()

    @staticmethod
    def backward(ctx, v):
        (theta,) = ctx.saved_tensors
        if getattr(ctx, "H", None) is None:  # one Hessian pass per graph node (hessian() asks n times)
            _, _, H = nll_eval_hess(ctx.handle, _host(theta))
            ctx.H = torch.from_numpy(np.asarray(H))
        Ht = ctx.H.to(v.device, v.dtype)
        return Ht @ v, None, None  # H is symmetric


class NLLFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, model_handle):
        nll, grad = nll_eval_grad(model_handle, _host(theta))
        ctx.save_for_backward(theta, torch.from_numpy(np.asarray(grad)).to(theta.device, theta.dtype))
        ctx.handle = model_handle
        return theta.new_tensor(nll)

    @staticmethod
    def backward(ctx, grad_output):
        theta, g = ctx.saved_tensors
        if torch.is_grad_enabled():  # create_graph: the gradient must be differentiable in theta
            g = _GradFunction.apply(theta, g, ctx.handle)
        return grad_output * g, None


def nll(model, theta):
    """NLL(theta) of a Model (or raw handle) as a torch scalar, differentiable twice."""
    handle = getattr(model, "handle", model)
    return NLLFunction.apply(theta, handle)
