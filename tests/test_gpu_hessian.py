"""Analytic Hessian and squared-weight score matrix on the GPU against the oracle (paper
Sec. 2.1: analytic Hessian for the HESSE uncertainties, Fisher information for weighted
fits), and the fits that use them."""
import numpy as np
import pytest

import oracle
from paper_2505_12414_gb300 import synth

pytestmark = pytest.mark.gpu

M1, M4 = oracle.MASS1D, oracle.KSTAR4D


def case(kind, n, stream, weighted):
    if kind == M1:
        cols, ranges, theta = synth.mass1d(n, stream=stream), synth.RANGES_1D, np.array([5283.0, 22.0, -0.0017, 0.35])
    else:
        cols, ranges, theta = synth.kstar4d(n, stream=stream), synth.RANGES_4D, synth.TRUTH_4D + 0.01
    w = synth.weights(n, stream=stream + 1) if weighted else None
    return cols, ranges, theta, w


def check_against_oracle(kind, cols, ranges, theta, w, nll, g, H, W, nthreads=1):
    ref = oracle.nll_hess(kind, ranges, cols, theta, w=w, nthreads=nthreads)
    assert ref["status"] == 0
    _, rg, rs, _ = oracle.nll_grad(kind, ranges, cols, theta, w=w, nthreads=nthreads)
    lp = np.log(oracle.pdf(kind, ranges, theta, cols))
    nscale = np.sum(np.abs(lp if w is None else w * lp))
    # tolerances: NLL and gradient as the gradient kernel; H within 1e-9 relative or 1e-12 of
    # the size of the terms the oracle subtracts per event (its own rounding bound: the plain
    # form cancels where one component dominates an event, the kernel's split does not);
    # W within 1e-12 of sqrt(W_aa W_bb) (its Cauchy-Schwarz bound)
    assert abs(nll - ref["nll"]) <= 1e-12 * nscale
    assert np.all(np.abs(g - rg) <= 1e-9 * np.abs(rg) + 1e-13 * rs), (g, rg)
    dH = np.abs(H - ref["hess"])
    assert np.all(dH <= 1e-9 * np.abs(ref["hess"]) + 1e-12 * ref["hscale"]), np.unravel_index(
        np.argmax(dH / (1e-9 * np.abs(ref["hess"]) + 1e-12 * ref["hscale"])), dH.shape)
    assert np.array_equal(H, H.T)
    if W is not None:
        d = np.sqrt(np.outer(np.diag(ref["w2"]), np.diag(ref["w2"])))
        assert np.all(np.abs(W - ref["w2"]) <= 1e-9 * np.abs(ref["w2"]) + 1e-12 * d)


@pytest.mark.parametrize("n", [1, 2, 127, 128, 129, 1000, 4099])
@pytest.mark.parametrize("kind,weighted,precompute",
                         [(M1, False, True), (M1, True, True), (M4, False, True), (M4, True, True),
                          (M4, False, False), (M4, True, False)])
def test_hessian_parity(gpu_lib, kind, weighted, precompute, n):
    cols, ranges, theta, w = case(kind, n, 300 + n, weighted)
    m = gpu_lib.Model(kind, ranges).load(cols, w, precompute=precompute)
    nll, g, H, W = m.eval_hess(theta, w2=True)
    check_against_oracle(kind, cols, ranges, theta, w, nll, g, H, W)
    # without W the Hessian is the same number
    nll2, g2, H2 = m.eval_hess(theta)
    assert nll2 == nll and np.array_equal(g2, g) and np.array_equal(H2, H)
    m.close()


def test_hessian_full_size_weighted(gpu_lib):
    # the bench workload size: 10^6 4D events, weighted, against the threaded oracle
    cols, ranges, theta, w = case(M4, 1_000_000, 310, True)
    m = gpu_lib.Model(M4, ranges).load(cols, w)
    nll, g, H, W = m.eval_hess(theta, w2=True)
    check_against_oracle(M4, cols, ranges, theta, w, nll, g, H, W, nthreads=16)
    # deterministic: the same bits on a second call
    again = m.eval_hess(theta, w2=True)
    assert again[0] == nll and np.array_equal(again[2], H) and np.array_equal(again[3], W)
    # the NLL and gradient of the Hessian pass agree with the fused gradient kernel
    n2, g2 = m.eval_grad(theta)
    _, _, rs, _ = oracle.nll_grad(M4, ranges, cols, theta, w=w, nthreads=16)
    assert abs(n2 - nll) <= 1e-12 * abs(nll)
    assert np.all(np.abs(g2 - g) <= 2e-9 * np.abs(g) + 2e-13 * rs)
    m.close()


def test_hessian_error_cases(gpu_lib):
    cols, ranges, theta, _ = case(M4, 500, 320, False)
    m = gpu_lib.Model(M4, ranges)
    with pytest.raises(gpu_lib.NLLError) as e:
        m.eval_hess(theta)
    assert e.value.status == gpu_lib.NLL_ERR_STATE
    m.load(cols)
    bad = theta.copy()
    bad[17] = 1.0
    with pytest.raises(gpu_lib.NLLError) as e:
        m.eval_hess(bad)
    assert e.value.status == gpu_lib.NLL_ERR_ARG
    neg = theta.copy()
    neg[6] = 3.0  # AFB far outside the physical region: negative rate somewhere
    neg[17] = 0.999
    nll, g, H, st = gpu_lib.nll_eval_hess(m.handle, neg, check=False)
    assert st == gpu_lib.NLL_ERR_NONPOSITIVE_PDF and nll == np.inf and np.all(np.isnan(H))
    m.load([c[:0] for c in cols])
    nll, g, H = m.eval_hess(theta)
    assert nll == 0.0 and np.all(g == 0.0) and np.all(H == 0.0)
    m.close()


def close_cov(C, ref):
    # 1e-6 relative, or 1e-9 of sqrt(C_aa C_bb) for entries near zero
    d = np.sqrt(np.outer(np.diag(ref), np.diag(ref)))
    assert np.all(np.abs(C - ref) <= 1e-6 * np.abs(ref) + 1e-9 * d), np.max(np.abs(C - ref) / d)


def _bounds(kind):
    n = 4 if kind == M1 else 18
    lo, hi = np.zeros(n), np.zeros(n)
    lo[-1], hi[-1] = 0.0, 1.0
    return lo, hi


def _step(kind):
    if kind == M1:
        return np.array([2.0, 1.0, 2e-4, 0.02])
    return np.array([1.0, 1.0] + [0.03] * 8 + [2e-4] + [0.03] * 6 + [0.02])


@pytest.mark.parametrize("kind,n", [(M1, 5000), (M4, 5000)])
def test_fits_with_analytic_hessian(gpu_lib, kind, n):
    cols = synth.mass1d(n, stream=330) if kind == M1 else synth.kstar4d(n, stream=331)
    ranges, truth = (synth.RANGES_1D, synth.TRUTH_1D) if kind == M1 else (synth.RANGES_4D, synth.TRUTH_4D)
    lo, hi = _bounds(kind)
    m = gpu_lib.Model(kind, ranges).load(cols)
    start = truth + 0.5 * _step(kind)
    fd = m.fit(start, lo=lo, hi=hi, step=_step(kind), tol_edm=1e-14, strategy=1, hessian=1)
    an = m.fit(start, lo=lo, hi=hi, step=_step(kind), tol_edm=1e-14, strategy=2, hessian=2)
    assert fd["status"] == 0 and an["status"] == 0
    assert np.max(np.abs((an["theta"] - fd["theta"]) / fd["err"])) < 1e-6
    np.testing.assert_allclose(an["err"], fd["err"], rtol=1e-4)
    assert an["n_eval"] < fd["n_eval"]
    # the covariance is the inverse of the oracle's Hessian at the fitted point
    ref = oracle.nll_hess(kind, ranges, cols, an["theta"])
    close_cov(an["cov"], np.linalg.inv(ref["hess"]))
    m.close()


def test_weighted_fit_sandwich_covariance(gpu_lib):
    # constant weights c: H scales with c and W with c^2, so H^-1 W H^-1 does not depend on c
    # while the inverse Hessian shrinks as 1/c; with varying weights the sandwich is
    # H^-1 W H^-1 of the oracle's matrices at the fitted point
    n = 20000
    cols = synth.mass1d(n, stream=340)
    lo, hi = _bounds(M1)
    kw = dict(lo=lo, hi=hi, step=_step(M1), tol_edm=1e-14, strategy=2)
    errs = {}
    for c in (1.0, 0.25):
        m = gpu_lib.Model(M1, synth.RANGES_1D).load(cols, np.full(n, c))
        errs[c, 2] = m.fit(synth.TRUTH_1D, hessian=2, **kw)
        errs[c, 3] = m.fit(synth.TRUTH_1D, hessian=3, **kw)
        m.close()
    for key, r in errs.items():
        assert r["status"] == 0, key
    np.testing.assert_allclose(errs[0.25, 2]["err"], 2.0 * errs[1.0, 2]["err"], rtol=1e-6)
    np.testing.assert_allclose(errs[0.25, 3]["err"], errs[1.0, 3]["err"], rtol=1e-6)
    # w = 1: sandwich and inverse Hessian estimate the same covariance
    np.testing.assert_allclose(errs[1.0, 3]["err"], errs[1.0, 2]["err"], rtol=0.05)

    w = synth.weights(n, stream=341)
    m = gpu_lib.Model(M1, synth.RANGES_1D).load(cols, w)
    r = m.fit(synth.TRUTH_1D, hessian=3, **kw)
    assert r["status"] == 0
    ref = oracle.nll_hess(M1, synth.RANGES_1D, cols, r["theta"], w=w)
    Hi = np.linalg.inv(ref["hess"])
    close_cov(r["cov"], Hi @ ref["w2"] @ Hi)
    m.close()


def test_host_callback_minimiser_rejects_analytic_options(gpu_lib):
    # a host objective has no second derivatives; batched and served fits take the options
    for strategy, hessian in ((2, 1), (1, 2), (0, 3)):
        r = gpu_lib.fit_minimise_fcn(lambda x: (float(np.sum(x ** 2)), 2 * x), [1.0, 2.0], strategy=strategy,
                                     hessian=hessian)
        assert r["status"] == gpu_lib.NLL_ERR_ARG


# --------------------------------------------------------------------------------------
# batched: per-toy Hessians in one device pass, and device-resident fits that use them
# --------------------------------------------------------------------------------------
RAGGED = [0, 1, 2, 127, 128, 129, 4095, 4096, 4097, 9000, 0, 3]


def ragged(kind, sizes, stream0, weighted):
    off = np.zeros(len(sizes) + 1, dtype=np.int64)
    off[1:] = np.cumsum(sizes)
    parts = [synth.mass1d(n, stream=stream0 + t) if kind == M1 else synth.kstar4d(n, stream=stream0 + t)
             for t, n in enumerate(sizes)]
    ndim = 1 if kind == M1 else 4
    cols = [np.concatenate([p[d] for p in parts]) for d in range(ndim)]
    w = synth.weights(int(off[-1]), stream=stream0 + 999) if weighted else None
    return off, cols, w


@pytest.mark.parametrize("kind,weighted,precompute",
                         [(M1, False, True), (M1, True, True), (M4, False, True), (M4, True, False)])
def test_batch_hessian_parity(gpu_lib, kind, weighted, precompute):
    off, cols, w = ragged(kind, RAGGED, 3600, weighted)
    ranges = synth.RANGES_1D if kind == M1 else synth.RANGES_4D
    base = np.array([5283.0, 22.0, -0.0017, 0.35]) if kind == M1 else synth.TRUTH_4D + 0.01
    scale = np.array([2.0, 1.0, 2e-4, 0.02]) if kind == M1 else np.array([1.0, 1.0] + [0.03] * 8 + [2e-4] + [0.03] * 6 + [0.02])
    thetas = np.array([synth.perturb(base, scale, k=t) for t in range(len(RAGGED))])
    b = gpu_lib.Batch(kind, ranges).load(off, cols, w, precompute=precompute)
    nll, g, H, W, st = b.eval_hess(thetas, w2=True)
    for t in range(len(RAGGED)):
        sl = slice(off[t], off[t + 1])
        ct = [c[sl] for c in cols]
        wt = w[sl] if w is not None else None
        assert st[t] == 0
        if off[t + 1] == off[t]:
            assert nll[t] == 0.0 and np.all(g[t] == 0.0) and np.all(H[t] == 0.0)
            continue
        check_against_oracle(kind, ct, ranges, thetas[t], wt, nll[t], g[t], H[t], W[t])
    # the single-sample pass on one toy gives the same numbers within rounding
    t = 8
    sl = slice(off[t], off[t + 1])
    m = gpu_lib.Model(kind, ranges).load([c[sl] for c in cols], w[sl] if w is not None else None,
                                         precompute=precompute)
    n1, g1, H1, W1 = m.eval_hess(thetas[t], w2=True)
    assert abs(n1 - nll[t]) <= 1e-13 * abs(n1)
    d = np.sqrt(np.outer(np.diag(np.abs(H1)), np.diag(np.abs(H1))))
    assert np.all(np.abs(H1 - H[t]) <= 1e-12 * d + 1e-12 * np.abs(H1))
    m.close()
    b.close()


def test_batch_hessian_reports_bad_points(gpu_lib):
    off, cols, _ = ragged(M4, [500, 600, 700], 3700, False)
    b = gpu_lib.Batch(M4, synth.RANGES_4D).load(off, cols)
    th = np.array([synth.TRUTH_4D] * 3)
    th[1, 17] = 1.0   # fsig outside (0, 1): invalid parameter point
    th[2, 6] = 3.0    # AFB far outside the physical region: negative rate somewhere
    th[2, 17] = 0.999
    nll, g, H, st = b.eval_hess(th)
    assert st[0] == 0 and np.isfinite(nll[0])
    assert st[1] == gpu_lib.NLL_ERR_ARG and np.isinf(nll[1]) and np.all(np.isnan(H[1]))
    assert st[2] == gpu_lib.NLL_ERR_NONPOSITIVE_PDF and np.isinf(nll[2])
    b.close()


@pytest.mark.parametrize("kind,nev,ntoy", [(M1, 3000, 8), (M4, 3000, 4)])
def test_batch_fits_with_analytic_hessian(gpu_lib, kind, nev, ntoy):
    off, cols, _ = ragged(kind, [nev] * ntoy, 3800, False)
    ranges = synth.RANGES_1D if kind == M1 else synth.RANGES_4D
    truth = synth.TRUTH_1D if kind == M1 else synth.TRUTH_4D
    lo, hi = _bounds(kind)
    step = _step(kind)
    start = truth + 0.5 * step
    b = gpu_lib.Batch(kind, ranges).load(off, cols)
    an = b.fit(start, lo=lo, hi=hi, step=step, tol_edm=1e-14, strategy=2, hessian=2)
    fd = b.fit(start, lo=lo, hi=hi, step=step, tol_edm=1e-14, strategy=1, hessian=1)
    assert np.all(an["status"] == 0) and np.all(fd["status"] == 0)
    assert np.all(an["n_eval"] < fd["n_eval"])
    for t in range(ntoy):
        sl = slice(off[t], off[t + 1])
        m = gpu_lib.Model(kind, ranges).load([c[sl] for c in cols])
        s = m.fit(start, lo=lo, hi=hi, step=step, tol_edm=1e-14, strategy=2, hessian=2)
        assert s["status"] == 0
        assert np.max(np.abs((an["theta"][t] - s["theta"]) / s["err"])) < 1e-6
        np.testing.assert_allclose(an["err"][t], s["err"], rtol=1e-5)
        np.testing.assert_allclose(an["err"][t], fd["err"][t], rtol=1e-3)
        # the covariance is the inverse of the oracle's Hessian at the toy's minimum
        ref = oracle.nll_hess(kind, ranges, [c[sl] for c in cols], an["theta"][t])
        close_cov(an["cov"][t], np.linalg.inv(ref["hess"]))
        m.close()
    b.close()


def test_batch_weighted_sandwich(gpu_lib):
    off, cols, w = ragged(M1, [20000, 15000, 25000], 3900, True)
    lo, hi = _bounds(M1)
    b = gpu_lib.Batch(M1, synth.RANGES_1D).load(off, cols, w)
    r = b.fit(synth.TRUTH_1D, lo=lo, hi=hi, step=_step(M1), tol_edm=1e-14, strategy=2, hessian=3)
    assert np.all(r["status"] == 0)
    for t in range(3):
        sl = slice(off[t], off[t + 1])
        ref = oracle.nll_hess(M1, synth.RANGES_1D, [cols[0][sl]], r["theta"][t], w=w[sl])
        Hi = np.linalg.inv(ref["hess"])
        close_cov(r["cov"][t], Hi @ ref["w2"] @ Hi)
    b.close()


def test_batched_weighted_pulls_with_the_sandwich(gpu_lib):
    # 1000 weighted toys (weights 0.2 or 2, unrelated to the data): pulls with the sandwich
    # covariance (hessian 3) have unit width; with the plain inverse Hessian (hessian 2) the
    # spread is underestimated by sqrt(E[w^2] / E[w]) = 1.36
    import math

    ntoy, nev = 1000, 2000
    off, cols = synth.toys1d(ntoy, nev, fixed_size=True)
    w = np.where(synth.Stream(synth.BASE_SEED, 830000).uniform(int(off[-1])) < 0.5, 0.2, 2.0)
    lo, hi = _bounds(M1)
    b = gpu_lib.Batch(M1, synth.RANGES_1D).load(off, cols, w)
    widths = {}
    for hessian in (3, 2):
        r = b.fit(synth.TRUTH_1D, lo=lo, hi=hi, step=_step(M1), tol_edm=1e-10, strategy=2, hessian=hessian)
        assert np.mean(r["status"] == 0) > 0.995
        ok = r["status"] == 0
        pulls = (r["theta"][ok] - synth.TRUTH_1D) / r["err"][ok]
        widths[hessian] = pulls.std(axis=0)
        assert np.all(np.abs(pulls.mean(axis=0)) < 4.0 / math.sqrt(ntoy) * widths[hessian] + 0.02)
    assert np.all(np.abs(widths[3] - 1.0) < 4.0 / math.sqrt(2 * ntoy) + 0.02), widths[3]
    assert np.all(widths[2] > 1.2), widths[2]
    b.close()


@pytest.mark.parametrize("kind,n", [(M1, 10000), (M4, 20000)])
def test_newton_route_matches_the_oracle_fit_in_fewer_passes(gpu_lib, kind, n):
    """strategy 4 (Newton steps with the analytic Hessian at every iterate) reaches the oracle's
    minimum to 1e-6 of the uncertainty, with its covariance, in fewer passes than the
    quasi-Newton route with analytic start matrix and polish (strategy 2, hessian 2)."""
    from oracle import fit as ofit

    cols = synth.mass1d(n, stream=21) if kind == M1 else synth.kstar4d(n, stream=21)
    ranges = synth.RANGES_1D if kind == M1 else synth.RANGES_4D
    truth = synth.TRUTH_1D if kind == M1 else synth.TRUTH_4D
    step = np.array([2.0, 1.0, 2e-4, 0.02]) if kind == M1 else np.array([1.0, 1.0] + [0.03] * 8 + [2e-4] + [0.03] * 6 + [0.02])
    npar = len(truth)
    lo, hi = np.zeros(npar), np.zeros(npar)
    hi[-1] = 1.0
    m = gpu_lib.Model(kind, ranges).load(cols)
    r4 = m.fit(truth + 0.5 * step, lo=lo, hi=hi, step=step, tol_edm=1e-14, strategy=4, hessian=2)
    r2 = m.fit(truth + 0.5 * step, lo=lo, hi=hi, step=step, tol_edm=1e-14, strategy=2, hessian=2)
    m.close()
    ref = ofit.fit(kind, ranges, cols, truth, tol_edm=1e-18, nthreads=8, h0=step * 1e-2)
    assert r4["status"] == 0 and r2["status"] == 0 and ref["converged"]
    assert np.max(np.abs((r4["theta"] - ref["theta"]) / ref["err"])) < 1e-6
    np.testing.assert_allclose(r4["err"], ref["err"], rtol=1e-3)
    assert r4["n_eval"] < r2["n_eval"]
