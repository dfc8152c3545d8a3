"""Accuracy of the kernels' FP64 building blocks on the GPU, against the host libm."""
import numpy as np
import pytest

from paper_2505_12414_gb300 import synth

import test_math_host as hm

pytestmark = pytest.mark.gpu


def ulp_err(a, ref):
    return np.abs(a - ref) / np.spacing(np.abs(ref))


def test_table_exponential_accuracy(gpu_lib, tmp_path):
    # the kernels' exponential takes its argument pre-scaled by S = 1024/ln2; it is integer
    # arithmetic throughout, so the device must reproduce the host build bit for bit
    xs = hm.exp_arguments(21)
    y = gpu_lib.nll_diag_math(0, xs)
    err = hm.ulp_error(y, hm.exp_reference(xs))
    assert float(err.max()) < 0.52, float(err.max())
    host = hm.host_math(hm.host_math_binary(tmp_path), "exp", xs, tmp_path)
    np.testing.assert_array_equal(y.view(np.int64), host.view(np.int64))
    # the saturated range: 0 below -1.04e6 (|x| >= 704), +inf above
    big = np.array([-1.04e6, -2e6, -1e300, -np.inf, 1.04e6, 1e300, np.inf])
    yb = gpu_lib.nll_diag_math(0, big)
    assert np.all(yb[:4] == 0.0) and np.all(np.isinf(yb[4:]))


def test_reciprocal_accuracy(gpu_lib):
    # the hardware single-precision seed refined in integer arithmetic (the host build of the same
    # refinement is checked without a GPU)
    x = hm.rcp_arguments(22)
    y = gpu_lib.nll_diag_math(1, x)
    err = hm.ulp_error(y, np.longdouble(1) / x.astype(np.longdouble))
    assert float(err.max()) < 0.51, float(err.max())
    assert np.all(np.signbit(y) == np.signbit(x))


def test_table_sincos_accuracy(gpu_lib, tmp_path):
    # the 4D kernels take sin/cos phi from the table method (integer arithmetic) for |phi| <= pi;
    # the device reproduces the host build bit for bit
    x = hm.sincos_arguments(23)
    xl = x.astype(np.longdouble)
    host = hm.host_math(hm.host_math_binary(tmp_path), "sincos", x, tmp_path).reshape(-1, 2)
    for col, fn, ref in ((0, 2, np.sin(xl)), (1, 3, np.cos(xl))):
        y = gpu_lib.nll_diag_math(fn, x)
        err = hm.sincos_ulp(y, ref)
        assert float(err.max()) < 1.0, (fn, float(err.max()), x[np.argmax(err)])
        np.testing.assert_array_equal(y.view(np.int64), host[:, col].copy().view(np.int64))


def test_sqrt_accuracy(gpu_lib):
    # the angular basis's square root: the hardware single-precision seed refined in integer
    # arithmetic (the host build of the same refinement is checked without a GPU)
    x = hm.sqrt_arguments(37)
    y = gpu_lib.nll_diag_math(7, x)
    err = hm.ulp_error(y, np.sqrt(x.astype(np.longdouble)))
    assert float(err.max()) < 0.52, (float(err.max()), x[np.argmax(err)])
    sq = np.arange(1, 3000, dtype=np.float64)
    np.testing.assert_array_equal(gpu_lib.nll_diag_math(7, sq * sq), sq)


def test_table_log_accuracy(gpu_lib, tmp_path):
    # the weighted kernels take ln P from the table-driven logarithm (positive normal P)
    rs = synth.Stream(29, 0)
    F = 1.0 + np.arange(129) / 128.0
    x = np.concatenate([
        10.0 ** (600.0 * rs.uniform(200000) - 300.0),                  # the whole normal range
        1.0 + (2.0 * rs.uniform(100000) - 1.0) * 1e-3,                 # around 1
        F, np.nextafter(F, 3.0), np.nextafter(F, 0.0),                  # the table points
        1.0 + (np.arange(128) + 0.5) / 128.0,                           # the rounding edges of j
        np.ldexp(F, (rs.uniform(129) * 200 - 100).astype(int)),
        np.array([0.5, 1.0, 2.0, np.nextafter(2.0, 0.0), np.nextafter(1.0, 0.0), np.nextafter(1.0, 2.0),
                  np.finfo(np.float64).tiny, np.finfo(np.float64).max]),
    ])
    x = np.concatenate([x, hm.log_arguments(30)])
    ref = np.log(x.astype(np.longdouble))
    y = gpu_lib.nll_diag_math(4, x)
    ok = ref != 0
    assert np.all(y[~ok] == 0.0)
    err = np.abs(y[ok].astype(np.longdouble) - ref[ok]) / np.spacing(np.abs(ref[ok]).astype(np.float64)).astype(np.longdouble)
    assert float(err.max()) < 0.51, (float(err.max()), x[ok][np.argmax(err)])
    # integer arithmetic throughout: the device reproduces the host build bit for bit
    host = hm.host_math(hm.host_math_binary(tmp_path), "log", x, tmp_path)
    np.testing.assert_array_equal(y.view(np.int64), host.view(np.int64))


def test_reciprocal_correction_order(gpu_lib):
    """Why a reciprocal refinement keeps the e^2 term: a hardware approximation alone
    (rcp.approx.ftz.f64 here) is good to about 2^-20, so one Newton step (error e^2) leaves
    about 2^-40 (1e-12, which would enter every gradient term); the kernels' refinement
    y0 (1 + e + e^2) has error e^3 and rounds to within 0.51 ulp (test_reciprocal_accuracy)."""
    rs = synth.Stream(24, 0)
    x = np.concatenate([np.exp((2 * rs.uniform(400000) - 1) * 600.0), 1.0 + rs.uniform(200000)])
    xl = x.astype(np.longdouble)
    e_approx = np.abs(gpu_lib.nll_diag_math(5, x).astype(np.longdouble) * xl - 1)
    e_newton = np.abs(gpu_lib.nll_diag_math(6, x).astype(np.longdouble) * xl - 1)
    assert 2.0 ** -24 < float(e_approx.max()) < 2.0 ** -18, float(e_approx.max())
    assert float(e_newton.max()) <= 4.0 * float(e_approx.max()) ** 2 + 2.0 ** -52
    assert float(e_newton.max()) > 2.0 ** -46  # far from the 2^-53 of the cubic correction
