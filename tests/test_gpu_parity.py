"""Parity of the CUDA path (through the C ABI) with the oracle, on the same seeded inputs.

Tolerances (fixed for this path):
  NLL:        |nll_gpu - nll_orc| <= 1e-12 * sum_i |w_i ln P_i|       (= 1e-12 |NLL| when
              all log-densities share a sign, as in the MeV configurations)
  gradient:   |g_gpu - g_orc| <= 1e-9 |g_orc| + 1e-13 S_k,  S_k = sum_i |w_i dln P_i/dtheta_k|
              (the second term covers components that cancel near a minimum)
  fits:       fitted parameters agree to 1e-6 of their uncertainty.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import fit as ofit
from paper_2505_12414_gb300 import synth

pytestmark = pytest.mark.gpu

M1, M4 = oracle.MASS1D, oracle.KSTAR4D
NTHREADS = 8

_cache = {}


def data(kind, n, stream=0, weighted=False):
    key = (kind, n, stream, weighted)
    if key not in _cache:
        cols = synth.mass1d(n, stream=stream) if kind == M1 else synth.kstar4d(n, stream=stream)
        w = synth.weights(n, stream=1000003 + stream) if weighted else None
        _cache[key] = (cols, w)
    return _cache[key]


def ranges_of(kind):
    return synth.RANGES_1D if kind == M1 else synth.RANGES_4D


def truth_of(kind):
    return synth.TRUTH_1D if kind == M1 else synth.TRUTH_4D


def scale_of(kind):
    if kind == M1:
        return np.array([2.0, 1.0, 2e-4, 0.02])
    return np.array([1.0, 1.0] + [0.03] * 8 + [2e-4] + [0.03] * 6 + [0.02])


def thetas(kind, k=3):
    out = [truth_of(kind)]
    for j in range(k):
        out.append(synth.perturb(truth_of(kind), scale_of(kind), k=j))
    return out


def assert_parity(kind, cols, w, theta, nll, grad, ranges=None):
    ranges = ranges_of(kind) if ranges is None else ranges
    rn, rg, rs, st = oracle.nll_grad(kind, ranges, cols, theta, w=w, nthreads=NTHREADS)
    assert st == 0
    lp = np.log(oracle.pdf(kind, ranges, theta, cols))
    nscale = np.sum(np.abs(lp if w is None else w * lp))
    assert abs(nll - rn) <= 1e-12 * nscale, (nll, rn, (nll - rn) / nscale)
    if grad is not None:
        bad = np.abs(grad - rg) > 1e-9 * np.abs(rg) + 1e-13 * rs
        assert not bad.any(), list(zip(np.where(bad)[0], grad[bad], rg[bad], rs[bad]))


def make_model(g, kind, cols, w=None, precompute=True, ranges=None):
    m = g.Model(kind, ranges_of(kind) if ranges is None else ranges)
    m.load(cols, w, precompute)
    return m


# --------------------------------------------------------------------------------------
@pytest.mark.parametrize("n", [1, 2, 3, 63, 64, 65, 255, 256, 257, 1000, 10000, 100003])
def test_mass1d_parity(gpu_lib, n):
    cols, _ = data(M1, n, stream=n)
    m = make_model(gpu_lib, M1, cols)
    for th in thetas(M1):
        nll, gr = m.eval_grad(th)
        assert_parity(M1, cols, None, th, nll, gr)
        assert_parity(M1, cols, None, th, m.eval(th), None)
    m.close()


@pytest.mark.parametrize("n", [1, 1000, 65537])
def test_mass1d_weighted_parity(gpu_lib, n):
    cols, w = data(M1, n, stream=n, weighted=True)
    m = make_model(gpu_lib, M1, cols, w)
    for th in thetas(M1):
        nll, gr = m.eval_grad(th)
        assert_parity(M1, cols, w, th, nll, gr)
    m.close()


def test_mass1d_paper_gev_configuration(gpu_lib):
    cols = synth.mass1d(20000, theta=synth.TRUTH_1D_GEV, ranges=synth.RANGES_1D_GEV)
    m = make_model(gpu_lib, M1, cols, ranges=synth.RANGES_1D_GEV)
    for th in (synth.TRUTH_1D_GEV, synth.TRUTH_1D_GEV + [0.01, 0.005, 0.2, -0.05]):
        nll, gr = m.eval_grad(th)
        assert_parity(M1, cols, None, th, nll, gr, ranges=synth.RANGES_1D_GEV)
    m.close()


@pytest.mark.parametrize("variant", [1, 2])
@pytest.mark.parametrize("weighted", [False, True])
@pytest.mark.parametrize("n", [1, 2, 5, 511, 4097, 100003])
def test_kstar4d_parity(gpu_lib, variant, weighted, n):
    cols, w = data(M4, n, stream=n, weighted=weighted)
    m = make_model(gpu_lib, M4, cols, w, precompute=(variant == 1))
    gpu_lib.nll_set_launch(m.handle, 0, 0, variant)
    assert gpu_lib.nll_get_launch(m.handle)["variant"] == variant
    for th in thetas(M4):
        nll, gr = m.eval_grad(th)
        assert_parity(M4, cols, w, th, nll, gr)
        assert_parity(M4, cols, w, th, m.eval(th), None)
    m.close()


def test_kstar4d_full_size_bench_configuration(gpu_lib):
    """1M events, the launch shape the bench uses (autotuned), every output compared."""
    cols, _ = data(M4, 1_000_000, stream=0)
    m = make_model(gpu_lib, M4, cols)
    m.eval_grad(truth_of(M4))
    gpu_lib.nll_autotune(m.handle)
    for th in thetas(M4, 2):
        nll, gr = m.eval_grad(th)
        assert_parity(M4, cols, None, th, nll, gr)
    m.close()


@pytest.mark.slow
def test_kstar4d_weighted_10M(gpu_lib):
    """The adjoint-check scale: 1e7 weighted events."""
    n = 10_000_000
    cols = synth.kstar4d(n, stream=4)
    w = synth.weights(n, stream=1000007)
    m = make_model(gpu_lib, M4, cols, w)
    th = synth.perturb(truth_of(M4), scale_of(M4), k=11)
    nll, gr = m.eval_grad(th)
    rn, rg, rs, st = oracle.nll_grad(M4, synth.RANGES_4D, cols, th, w=w, nthreads=16)
    assert st == 0
    assert abs(nll - rn) <= 1e-12 * abs(rn)
    assert np.all(np.abs(gr - rg) <= 1e-9 * np.abs(rg) + 1e-13 * rs)
    m.close()


def test_precomputed_basis_matches_oracle_terms(gpu_lib):
    n = 20011
    cols, _ = data(M4, n, stream=5)
    m = make_model(gpu_lib, M4, cols)
    B = gpu_lib.nll_precomputed_basis(m.handle, n)
    f = oracle.angular_terms(cols[1], cols[2], cols[3])
    ref = np.empty((n, 13))
    ref[:, 0] = f[:, 0] + f[:, 2]
    ref[:, 1] = f[:, 1] - f[:, 0] - f[:, 2] - f[:, 3]
    ref[:, 2:9] = f[:, 4:11]
    ref[:, 9] = 2 * cols[1] ** 2 - 1
    ref[:, 10] = 2 * cols[2] ** 2 - 1
    ref[:, 11] = cols[3] / math.pi
    ref[:, 12] = 2 * ref[:, 11] ** 2 - 1
    # basis terms are O(0.1) and T2 = 2x^2 - 1 cancels near x^2 = 1/2: a few ulps of 1 absolute
    np.testing.assert_allclose(B, ref, rtol=1e-13, atol=2e-15)
    m.close()


def test_zero_events(gpu_lib):
    m = gpu_lib.Model(M4, synth.RANGES_4D)
    m.load([np.zeros(0)] * 4)
    nll, gr = m.eval_grad(synth.TRUTH_4D)
    assert nll == 0.0 and np.all(gr == 0.0)
    m.close()


def test_events_outside_ranges_are_rejected(gpu_lib):
    cols, _ = data(M4, 1000, stream=6)
    bad = [c.copy() for c in cols]
    bad[1][17] = 1.0000001
    m = gpu_lib.Model(M4, synth.RANGES_4D)
    with pytest.raises(gpu_lib.NLLError) as e:
        m.load(bad)
    assert e.value.status == gpu_lib.NLL_ERR_ARG
    bad = [c.copy() for c in cols]
    bad[0][3] = 5169.0
    with pytest.raises(gpu_lib.NLLError):
        m.load(bad)
    with pytest.raises(gpu_lib.NLLError) as e:
        m.eval(synth.TRUTH_4D)
    assert e.value.status == gpu_lib.NLL_ERR_STATE
    m.close()


def test_nonpositive_density_is_reported(gpu_lib):
    cols, _ = data(M4, 2000, stream=14)
    m = make_model(gpu_lib, M4, cols)
    th = synth.TRUTH_4D.copy()
    th[6] = 3.0
    th[17] = 0.999
    nll, gr, st = gpu_lib.nll_eval_grad(m.handle, th, check=False)
    assert st == gpu_lib.NLL_ERR_NONPOSITIVE_PDF and nll == math.inf
    m.close()


def test_invalid_parameters_are_rejected(gpu_lib):
    cols, _ = data(M1, 1000, stream=7)
    m = make_model(gpu_lib, M1, cols)
    for th in ([5279.6, -1.0, -0.002, 0.3], [5279.6, 20.0, -0.002, 1.2], [np.nan, 20.0, -0.002, 0.3]):
        _, st = gpu_lib.nll_eval(m.handle, th, check=False)
        assert st == gpu_lib.NLL_ERR_ARG
    # grad needs 0 < fsig < 1, plain NLL accepts the closed interval
    _, _, st = gpu_lib.nll_eval_grad(m.handle, [5279.6, 20.0, -0.002, 1.0], check=False)
    assert st == gpu_lib.NLL_ERR_ARG
    for f in (0.0, 1.0):
        th = [5279.6, 20.0, -0.002, f]
        assert_parity(M1, cols, None, th, m.eval(th), None)
    m.close()


def test_repeated_evaluations_are_bitwise_identical(gpu_lib):
    cols, _ = data(M4, 100003, stream=100003)
    m = make_model(gpu_lib, M4, cols)
    a = m.eval_grad(synth.TRUTH_4D)
    for _ in range(3):
        b = m.eval_grad(synth.TRUTH_4D)
        assert a[0] == b[0] and np.array_equal(a[1], b[1])
    m.close()


@pytest.mark.parametrize("shape", [(1, 64), (1, 256), (3, 192), (8, 128), (32, 256)])
def test_launch_shapes(gpu_lib, shape):
    cols, _ = data(M4, 100003, stream=100003)
    m = make_model(gpu_lib, M4, cols)
    gpu_lib.nll_set_launch(m.handle, shape[0], shape[1], 0)
    th = thetas(M4)[1]
    nll, gr = m.eval_grad(th)
    assert_parity(M4, cols, None, th, nll, gr)
    m.close()


def test_device_resident_inputs(gpu_lib):
    import torch

    cols, w = data(M4, 4097, stream=4097, weighted=True)
    host = make_model(gpu_lib, M4, cols, w)
    dev = gpu_lib.Model(M4, synth.RANGES_4D)
    dev.load([torch.tensor(c, device="cuda") for c in cols], torch.tensor(w, device="cuda"))
    a, b = host.eval_grad(synth.TRUTH_4D), dev.eval_grad(synth.TRUTH_4D)
    assert a[0] == b[0] and np.array_equal(a[1], b[1])
    host.close()
    dev.close()


def test_torch_stream(gpu_lib):
    import torch

    s = torch.cuda.Stream()
    cols, _ = data(M1, 10000, stream=10000)
    m = gpu_lib.Model(M1, synth.RANGES_1D, stream=s.cuda_stream)
    m.load(cols)
    nll, gr = m.eval_grad(synth.TRUTH_1D)
    assert_parity(M1, cols, None, synth.TRUTH_1D, nll, gr)
    m.close()


# --------------------------------------------------------------------------------------
# fits: GPU minimiser vs the oracle's Newton fit, to 1e-6 of the uncertainty
# --------------------------------------------------------------------------------------
def _bounds(kind):
    n = 4 if kind == M1 else 18
    lo, hi = np.zeros(n), np.zeros(n)
    lo[-1], hi[-1] = 0.0, 1.0
    return lo, hi


@pytest.mark.parametrize("kind,n", [(M1, 10000), (M4, 20000)])
def test_fit_parity(gpu_lib, kind, n):
    cols, _ = data(kind, n, stream=21)
    m = make_model(gpu_lib, kind, cols)
    truth = truth_of(kind)
    step = scale_of(kind)
    lo, hi = _bounds(kind)
    r = m.fit(truth + 0.5 * step, lo=lo, hi=hi, step=step, tol_edm=1e-14, strategy=1, hessian=1)
    ref = ofit.fit(kind, ranges_of(kind), cols, truth, tol_edm=1e-18, nthreads=NTHREADS, h0=step * 1e-2)
    assert r["status"] == 0, r["status"]
    assert ref["converged"]
    pull = (r["theta"] - ref["theta"]) / ref["err"]
    assert np.max(np.abs(pull)) < 1e-6, pull
    np.testing.assert_allclose(r["err"], ref["err"], rtol=1e-3)
    m.close()
