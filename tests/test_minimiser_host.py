"""Host logic of the library's quasi-Newton minimiser, run on CPU objectives (no GPU).

The objective for the likelihood checks is the oracle NLL; the library's minimiser must
reach the same minimum as the oracle's independent Newton fit."""
import math

import numpy as np
import pytest

import oracle
from oracle import fit as ofit
from paper_2505_12414_gb300 import synth


@pytest.fixture(scope="module")
def g():
    import paper_2505_12414_gb300 as g
    from paper_2505_12414_gb300 import build

    build.build()
    g.load()
    return g


def test_quadratic_minimum_and_covariance(g):
    rs = synth.Stream(1, 1)
    n = 6
    M = rs.uniform(n * n).reshape(n, n) - 0.5
    H = M @ M.T + n * np.eye(n)
    x0 = rs.uniform(n)

    def f(x):
        d = x - x0
        return 0.5 * d @ H @ d + 3.0, H @ d

    for strategy in (0, 1):
        r = g.fit_minimise_fcn(f, np.zeros(n), tol_edm=1e-20, strategy=strategy, hessian=1)
        assert r["status"] == 0
        np.testing.assert_allclose(r["theta"], x0, rtol=0, atol=1e-9)
        np.testing.assert_allclose(r["cov"], np.linalg.inv(H), rtol=1e-6, atol=1e-9)


def test_rosenbrock(g):
    def f(x):
        a, b = x
        return (1 - a) ** 2 + 100 * (b - a * a) ** 2, np.array([-2 * (1 - a) - 400 * a * (b - a * a),
                                                               200 * (b - a * a)])

    r = g.fit_minimise_fcn(f, [-1.2, 1.0], step=[0.1, 0.1], tol_edm=1e-18, strategy=0, hessian=0, max_iter=2000)
    assert r["status"] == 0
    np.testing.assert_allclose(r["theta"], [1.0, 1.0], atol=1e-6)


def test_bounds_and_fixed_parameters(g):
    # minimum of (x-3)^2 + (y+1)^2 with x bounded in [0, 2] sits on the bound x -> 2
    def f(x):
        return (x[0] - 3) ** 2 + (x[1] + 1) ** 2 + (x[2] - 5) ** 2, np.array(
            [2 * (x[0] - 3), 2 * (x[1] + 1), 2 * (x[2] - 5)])

    r = g.fit_minimise_fcn(f, [1.0, 0.0, 0.7], lo=[0.0, 0.0, 0.0], hi=[2.0, 0.0, 0.0], fixed=[0, 0, 1],
                           tol_edm=1e-14, strategy=0, hessian=0)
    assert abs(r["theta"][0] - 2.0) < 1e-4
    assert abs(r["theta"][1] + 1.0) < 1e-6
    assert r["theta"][2] == 0.7 and r["err"][2] == 0.0


def test_rejected_points_are_avoided(g):
    # objective undefined for x < 0.5: the line search must back off
    def f(x):
        if x[0] < 0.5:
            raise ValueError
        return (x[0] - 0.6) ** 2, np.array([2 * (x[0] - 0.6)])

    r = g.fit_minimise_fcn(f, [3.0], step=[5.0], tol_edm=1e-16, strategy=0, hessian=0)
    assert r["status"] == 0 and abs(r["theta"][0] - 0.6) < 1e-7


@pytest.mark.parametrize("kind", [oracle.MASS1D, oracle.KSTAR4D])
def test_oracle_likelihood_minimum_matches_oracle_newton(g, kind):
    if kind == oracle.MASS1D:
        cols, ranges, truth = synth.mass1d(10000, stream=31), synth.RANGES_1D, synth.TRUTH_1D
        lo = np.array([5200.0, 5.0, -0.02, 0.0])
        hi = np.array([5400.0, 60.0, 0.02, 1.0])
    else:
        cols, ranges, truth = synth.kstar4d(3000, stream=32), synth.RANGES_4D, synth.TRUTH_4D
        lo = np.zeros(18)
        hi = np.zeros(18)
        lo[17], hi[17] = 0.0, 1.0
    step = np.maximum(np.abs(truth) * 1e-2, 1e-2)
    step[[0, 1]] = [1.0, 1.0]
    if kind == oracle.MASS1D:
        step[2] = 2e-4

    def f(t):
        nll, gr, _, st = oracle.nll_grad(kind, ranges, cols, t)
        if st != 0:
            raise ValueError
        return nll, gr

    start = truth + 0.3 * step
    r = g.fit_minimise_fcn(f, start, lo=lo, hi=hi, step=step, tol_edm=1e-14, strategy=1, hessian=1)
    ref = ofit.fit(kind, ranges, cols, truth, tol_edm=1e-18, h0=step * 1e-2)
    assert r["status"] == 0, r
    assert ref["converged"]
    pull = (r["theta"] - ref["theta"]) / ref["err"]
    assert np.max(np.abs(pull)) < 1e-6, pull
    np.testing.assert_allclose(r["err"], ref["err"], rtol=1e-3)


def test_analytic_hessian_options_need_a_model(g):
    # strategy 2 and hessian 2/3 take second derivatives from a model; a host callback has none
    def f(x):
        return float(np.sum(x ** 2)), 2.0 * x

    for strategy, hessian in ((2, 0), (0, 2), (1, 3)):
        r = g.fit_minimise_fcn(f, [1.0, 2.0], strategy=strategy, hessian=hessian)
        assert r["status"] == g.NLL_ERR_ARG
