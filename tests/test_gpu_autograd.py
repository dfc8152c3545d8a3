"""The torch.autograd.Function around the fused kernel: backward is the kernel's analytic
gradient, agrees with central finite differences of forward, and with the oracle at 1e7
weighted events."""
import numpy as np
import pytest

import oracle
from paper_2505_12414_gb300 import synth

pytestmark = pytest.mark.gpu


def test_backward_matches_kernel_gradient_and_finite_differences(gpu_lib):
    import torch

    from paper_2505_12414_gb300 import autograd

    cols = synth.kstar4d(20000, stream=31)
    m = gpu_lib.Model(gpu_lib.NLL_MODEL_KSTARMUMU4D, synth.RANGES_4D).load(cols)
    th0 = synth.TRUTH_4D + 0.01
    theta = torch.tensor(th0, dtype=torch.float64, requires_grad=True)
    y = autograd.nll(m, theta)
    y.backward()
    nll, g = m.eval_grad(th0)
    assert y.item() == nll
    assert np.array_equal(theta.grad.numpy(), g)
    _, _, s, _ = oracle.nll_grad(oracle.KSTAR4D, synth.RANGES_4D, cols, th0)
    nscale = np.sum(np.abs(np.log(oracle.pdf(oracle.KSTAR4D, synth.RANGES_4D, th0, cols))))
    for k in range(18):
        h = 1e-6 * max(abs(th0[k]), 1.0)
        tp, tm = th0.copy(), th0.copy()
        tp[k] += h
        tm[k] -= h
        with torch.no_grad():
            fd = (autograd.nll(m, torch.tensor(tp)).item() - autograd.nll(m, torch.tensor(tm)).item()) / (2 * h)
        # truncation O(h^2) plus the roundoff of two NLL values of size sum|l| divided by 2h
        assert abs(fd - g[k]) <= 1e-6 * abs(g[k]) + 1e-7 * s[k] + 4e-16 * nscale / h, (k, fd, g[k])
    m.close()


@pytest.mark.slow
def test_backward_against_oracle_10M_weighted(gpu_lib):
    import torch

    from paper_2505_12414_gb300 import autograd

    n = 10_000_000
    cols = synth.kstar4d(n, stream=4)
    w = synth.weights(n, stream=1000007)
    m = gpu_lib.Model(gpu_lib.NLL_MODEL_KSTARMUMU4D, synth.RANGES_4D).load(cols, w)
    th = synth.TRUTH_4D - 0.005
    theta = torch.tensor(th, dtype=torch.float64, device="cuda", requires_grad=True)
    y = autograd.nll(m, theta)
    (2.0 * y).backward()
    rn, rg, rs, st = oracle.nll_grad(oracle.KSTAR4D, synth.RANGES_4D, cols, th, w=w, nthreads=16)
    assert st == 0
    assert abs(y.item() - rn) <= 1e-12 * abs(rn)
    g = theta.grad.cpu().numpy() / 2.0
    assert np.all(np.abs(g - rg) <= 1e-9 * np.abs(rg) + 1e-13 * rs)
    m.close()


def test_second_derivatives_through_autograd(gpu_lib):
    # double backward and torch.autograd.functional.hessian use the analytic Hessian pass
    import torch

    from paper_2505_12414_gb300 import autograd

    cols = synth.kstar4d(20000, stream=32)
    w = synth.weights(20000, stream=33)
    m = gpu_lib.Model(gpu_lib.NLL_MODEL_KSTARMUMU4D, synth.RANGES_4D).load(cols, w)
    th0 = synth.TRUTH_4D + 0.01
    _, g_ref, H_ref = m.eval_hess(th0)
    theta = torch.tensor(th0, dtype=torch.float64, requires_grad=True)
    H = torch.autograd.functional.hessian(lambda t: autograd.nll(m, t), theta)
    assert np.array_equal(H.numpy(), H_ref)
    # Hessian-vector product by double backward
    v = torch.linspace(-1.0, 1.0, 18, dtype=torch.float64)
    y = autograd.nll(m, theta)
    (g,) = torch.autograd.grad(y, theta, create_graph=True)
    assert np.array_equal(g.detach().numpy(), m.eval_grad(th0)[1])
    (hv,) = torch.autograd.grad(g @ v, theta)
    np.testing.assert_allclose(hv.numpy(), H_ref @ v.numpy(), rtol=1e-13, atol=1e-13 * np.abs(H_ref).max())
    # and the Hessian agrees with the oracle
    ref = oracle.nll_hess(oracle.KSTAR4D, synth.RANGES_4D, cols, th0, w=w)
    assert np.all(np.abs(H.numpy() - ref["hess"]) <= 1e-9 * np.abs(ref["hess"]) + 1e-12 * ref["hscale"])
    m.close()
