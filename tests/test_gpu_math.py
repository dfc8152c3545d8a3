"""Accuracy of the kernels' FP64 building blocks on the GPU, against the host libm."""
import numpy as np
import pytest

from paper_2505_12414_gb300 import synth

pytestmark = pytest.mark.gpu


def ulp_err(a, ref):
    return np.abs(a - ref) / np.spacing(np.abs(ref))


def test_table_exponential_accuracy(gpu_lib):
    rs = synth.Stream(21, 0)
    x = np.concatenate([
        (2 * rs.uniform(200000) - 1) * 706.0,          # the whole fast range
        (2 * rs.uniform(200000) - 1) * 40.0,           # the range the likelihood uses
        (2 * rs.uniform(50000) - 1) * 1e-3,            # near zero
        np.array([0.0, -0.0, 1e-300, -1e-300, 5e-324, 706.9, -706.9, np.log(2.0), -np.log(2.0)]),
    ])
    y = gpu_lib.nll_diag_math(0, x)
    ref = np.exp(x)
    assert ulp_err(y, ref).max() <= 2.0
    # the saturated range: 0 below -707, +inf above 707
    big = np.array([-707.0, -800.0, -1e300, -np.inf, 707.0, 1e300, np.inf])
    yb = gpu_lib.nll_diag_math(0, big)
    assert np.all(yb[:4] == 0.0) and np.all(np.isinf(yb[4:]))


def test_reciprocal_accuracy(gpu_lib):
    rs = synth.Stream(22, 0)
    x = np.concatenate([
        np.exp((2 * rs.uniform(200000) - 1) * 60.0),
        -np.exp((2 * rs.uniform(20000) - 1) * 60.0),
        np.array([1.0, 2.0, 3.0, 0.1, 1.0 - 2 ** -52, 1.0 + 2 ** -52]),
    ])
    y = gpu_lib.nll_diag_math(1, x)
    assert ulp_err(y, 1.0 / x).max() <= 1.0
