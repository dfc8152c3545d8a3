"""Parity with the oracle at the edges of the method, through every entry point of the C ABI.

Parameter points where the hoisted parameter-only terms switch branches (Sec. 2.4.1, Eq. 2):
  * alpha == 0 exactly: the exponential's normalisation is the window width (the paper's
    alpha == 0 branch), its log-derivative the window's midpoint;
  * |alpha (mb - ma)| <= 1e-3: d ln N2 / d alpha from its series;
  * |alpha (mb - ma)| < 1/2: d^2 ln N2 / d alpha^2 (the analytic Hessian) from its series;
  * the Gaussian mean on the window's lower edge, and outside it on either side;
  * a width small enough that, for events on the window's upper edge, the Gaussian factor
    drops below exp(-704): the kernels' exponential returns 0 there, the oracle's a
    subnormal; and a narrow width where most events have a vanishing Gaussian factor.
Events on the boundary of the observable box (Sec. 2.4.2, Eq. 3): cos theta_l and
cos theta_K = +-1 (sin = 0; at the four corners both the S- and P-wave terms of A vanish and
only the background remains), phi = +-pi (the sine/cosine table index wraps), m = ma, m = mb.

Entry points: nll_eval_grad and nll_eval (4D: precomputed and direct angular variants,
weighted and unweighted), an in-place sample (on_device = 2), nll_eval_hess, the batched
nll_batch_eval_grad (both schedules) and nll_batch_eval_hess with one toy per parameter
point (device-side hoisting), nll_eval_grad_4d_noalloc, and served fits (device-side
hoisting inside the fit loop) against the oracle's own fits.  The exponent-range guard of
the kernels' factored exponential returns NLL_ERR_ARG on every entry point.

Tolerances as everywhere: NLL 1e-12 of sum |w ln P|; gradient 1e-9 relative + 1e-13 of the
term scale S_k; Hessian 1e-9 relative + 1e-12 of the size of the two terms the oracle
subtracts per event; fitted parameters 1e-6 of their uncertainty.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import fit as ofit
from paper_2505_12414_gb300 import synth

pytestmark = pytest.mark.gpu

M1, M4 = oracle.MASS1D, oracle.KSTAR4D
MA, MB = synth.RANGES_1D[0], synth.RANGES_1D[1]
D = MB - MA

# parameter points: (name, {index in the mass-model order: value}); the 4D model takes the
# same mass parameters (mu -> 0, sigma -> 1, alpha -> 10)
EDGE_POINTS = [
    ("alpha_zero", {2: 0.0}),
    ("alpha_series", {2: 1e-4 / D}),            # |alpha D| = 1e-4 < 1e-3
    ("alpha_series_neg", {2: -8e-4 / D}),       # |alpha D| = 8e-4
    ("alpha_coth_series", {2: -0.3 / D}),       # |alpha D| = 0.3 < 1/2
    ("mu_on_lower_edge", {0: MA}),
    ("mu_below_window", {0: MA - 10.0}),
    ("mu_above_window", {0: MB + 10.0}),
    ("sigma_upper_edge_underflow", {1: 18.3}),  # (mb - mu)^2 / 2 sigma^2 = 712 > 704
    ("sigma_narrow", {1: 3.0}),
]
NAMES = [p[0] for p in EDGE_POINTS]
MAP4D = {0: 0, 1: 1, 2: 10, 3: 17}


def theta_of(kind, name):
    mods = dict(EDGE_POINTS)[name]
    th = (synth.TRUTH_1D if kind == M1 else synth.TRUTH_4D).copy()
    for k, v in mods.items():
        th[k if kind == M1 else MAP4D[k]] = v
    return th


def ranges_of(kind):
    return synth.RANGES_1D if kind == M1 else synth.RANGES_4D


def edge_events(kind, n_base=4099, stream=8800):
    """A seeded sample with events on every face, edge and corner of the observable box
    spliced in at several positions (both halves of a 128-bit pair, and the ragged tail)."""
    if kind == M1:
        base = synth.mass1d(n_base, stream=stream)[0]
        edges = np.array([MA, MB, MA, MB, MB, MA, MB])
        cols = [np.concatenate([base[:1000], edges, base[1000:3001], edges[::-1], base[3001:], [MB]])]
        return cols
    base = synth.kstar4d(n_base, stream=stream)
    rs = synth.Stream(synth.BASE_SEED, stream + 1)
    pick = rs.uniform(4 * 81)
    mvals = [MA, MB, None]
    lvals = [-1.0, 1.0, None]
    pvals = [-math.pi, math.pi, None]
    rows = []
    i = 0
    for m in mvals:
        for cl in lvals:
            for ck in lvals:
                for ph in pvals:
                    row = [m if m is not None else MA + D * pick[i],
                           cl if cl is not None else 2.0 * pick[i + 1] - 1.0,
                           ck if ck is not None else 2.0 * pick[i + 2] - 1.0,
                           ph if ph is not None else math.pi * (2.0 * pick[i + 3] - 1.0)]
                    rows.append(row)
                    i += 4
    e = np.array(rows).T  # 81 events
    cols = []
    for c in range(4):
        cols.append(np.concatenate([base[c][:1000], e[c][:40], base[c][1000:3001], e[c][40:], base[c][3001:],
                                    e[c][:1]]))
    return cols


_data = {}


def data(kind, weighted):
    key = (kind, weighted)
    if key not in _data:
        cols = edge_events(kind)
        w = synth.weights(len(cols[0]), stream=8900) if weighted else None
        _data[key] = (cols, w)
    return _data[key]


def assert_parity(kind, cols, w, th, nll, grad):
    rn, rg, rs, st = oracle.nll_grad(kind, ranges_of(kind), cols, th, w=w, nthreads=8)
    assert st == 0
    lp = np.log(oracle.pdf(kind, ranges_of(kind), th, cols))
    nscale = np.sum(np.abs(lp if w is None else w * lp))
    assert abs(nll - rn) <= 1e-12 * nscale, (nll, rn, (nll - rn) / nscale)
    if grad is not None:
        bad = np.abs(grad - rg) > 1e-9 * np.abs(rg) + 1e-13 * rs
        assert not bad.any(), list(zip(np.where(bad)[0], grad[bad], rg[bad], rs[bad]))


def assert_hess_parity(kind, cols, w, th, nll, g, H, W):
    ranges = ranges_of(kind)
    ref = oracle.nll_hess(kind, ranges, cols, th, w=w, nthreads=8)
    assert ref["status"] == 0
    assert_parity(kind, cols, w, th, nll, g)
    dH = np.abs(H - ref["hess"])
    tol = 1e-9 * np.abs(ref["hess"]) + 1e-12 * ref["hscale"]
    assert np.all(dH <= tol), np.unravel_index(np.argmax(dH / tol), dH.shape)
    if W is not None:
        d = np.sqrt(np.outer(np.diag(ref["w2"]), np.diag(ref["w2"])))
        assert np.all(np.abs(W - ref["w2"]) <= 1e-9 * np.abs(ref["w2"]) + 1e-12 * d)


def test_edge_sample_lies_on_the_box():
    cols = edge_events(M4)
    assert np.sum(np.abs(cols[1]) == 1.0) >= 54 and np.sum(np.abs(cols[2]) == 1.0) >= 54
    assert np.sum((np.abs(cols[1]) == 1.0) & (np.abs(cols[2]) == 1.0)) >= 36  # the four A = 0 corners
    assert np.sum(np.abs(cols[3]) == math.pi) >= 54
    assert np.sum(cols[0] == MA) >= 27 and np.sum(cols[0] == MB) >= 27
    # the Gaussian factor of the upper-edge events underflows the kernels' exponential range
    th = theta_of(M1, "sigma_upper_edge_underflow")
    assert (MB - th[0]) ** 2 / (2 * th[1] ** 2) > 704.0


# --------------------------------------------------------------------------------------
# single-sample entry points
# --------------------------------------------------------------------------------------
@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("weighted", [False, True])
def test_mass_model_edges(gpu_lib, name, weighted):
    cols, w = data(M1, weighted)
    th = theta_of(M1, name)
    m = gpu_lib.Model(M1, synth.RANGES_1D).load(cols, w)
    nll, g = m.eval_grad(th)
    assert_parity(M1, cols, w, th, nll, g)
    assert_parity(M1, cols, w, th, m.eval(th), None)
    m.close()


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("variant", [1, 2])
@pytest.mark.parametrize("weighted", [False, True])
def test_4d_model_edges(gpu_lib, name, variant, weighted):
    cols, w = data(M4, weighted)
    th = theta_of(M4, name)
    m = gpu_lib.Model(M4, synth.RANGES_4D).load(cols, w, precompute=(variant == 1))
    gpu_lib.nll_set_launch(m.handle, 0, 0, variant)
    nll, g = m.eval_grad(th)
    assert_parity(M4, cols, w, th, nll, g)
    assert_parity(M4, cols, w, th, m.eval(th), None)
    m.close()


@pytest.mark.parametrize("kind", [M1, M4])
@pytest.mark.parametrize("weighted", [False, True])
def test_in_place_edges(gpu_lib, kind, weighted):
    import torch

    cols, w = data(kind, weighted)
    dev = [torch.from_numpy(c).to("cuda") for c in cols]
    wd = torch.from_numpy(w).to("cuda") if w is not None else None
    torch.cuda.synchronize()
    m = gpu_lib.Model(kind, ranges_of(kind)).load(dev, wd, in_place=True)
    for name in NAMES:
        th = theta_of(kind, name)
        nll, g = m.eval_grad(th)
        assert_parity(kind, cols, w, th, nll, g)
    m.close()


@pytest.mark.parametrize("kind", [M1, M4])
@pytest.mark.parametrize("weighted", [False, True])
def test_hessian_edges(gpu_lib, kind, weighted):
    cols, w = data(kind, weighted)
    m = gpu_lib.Model(kind, ranges_of(kind)).load(cols, w)
    for name in NAMES:
        th = theta_of(kind, name)
        nll, g, H, W = m.eval_hess(th, w2=True)
        assert_hess_parity(kind, cols, w, th, nll, g, H, W)
    m.close()


@pytest.mark.parametrize("weighted", [False, True])
def test_noalloc_edges(gpu_lib, weighted):
    import torch

    cols, w = data(M4, weighted)
    dev = [torch.from_numpy(c).to("cuda") for c in cols]
    wd = torch.from_numpy(w).to("cuda") if w is not None else None
    torch.cuda.synchronize()
    for name in NAMES:
        th = theta_of(M4, name)
        nll, g = gpu_lib.nll_eval_grad_4d_noalloc(synth.RANGES_4D, dev, th, dev_weights=wd)
        assert_parity(M4, cols, w, th, nll, g)


# --------------------------------------------------------------------------------------
# batched entry points: one toy per parameter point, hoisted on the device
# --------------------------------------------------------------------------------------
def _batch(g, kind, cols, w, ntoy, precompute=True):
    n = len(cols[0])
    off = np.arange(ntoy + 1, dtype=np.int64) * n
    tiled = [np.tile(c, ntoy) for c in cols]
    wt = np.tile(w, ntoy) if w is not None else None
    return g.Batch(kind, ranges_of(kind)).load(off, tiled, wt, precompute=precompute)


@pytest.mark.parametrize("kind", [M1, M4])
@pytest.mark.parametrize("weighted", [False, True])
@pytest.mark.parametrize("tile", [0, 256])
def test_batch_edges(gpu_lib, kind, weighted, tile):
    cols, w = data(kind, weighted)
    thetas = np.array([theta_of(kind, nm) for nm in NAMES])
    b = _batch(gpu_lib, kind, cols, w, len(NAMES))
    b.set_schedule(tile, 0)
    nll, g, st = b.eval_grad(thetas)
    assert np.all(st == 0), st
    for i, th in enumerate(thetas):
        assert_parity(kind, cols, w, th, nll[i], g[i])
    b.close()


@pytest.mark.parametrize("kind", [M1, M4])
@pytest.mark.parametrize("weighted", [False, True])
def test_batch_hessian_edges(gpu_lib, kind, weighted):
    cols, w = data(kind, weighted)
    thetas = np.array([theta_of(kind, nm) for nm in NAMES])
    b = _batch(gpu_lib, kind, cols, w, len(NAMES))
    nll, g, H, W, st = b.eval_hess(thetas, w2=True)
    assert np.all(st == 0), st
    for i, th in enumerate(thetas):
        assert_hess_parity(kind, cols, w, th, nll[i], g[i], H[i], W[i])
    b.close()


@pytest.mark.parametrize("kind", [M1, M4])
@pytest.mark.parametrize("weighted,precompute", [(False, True), (True, False)])
def test_estimated_start_matrix_fits_on_edges(gpu_lib, kind, weighted, precompute):
    """Batched fits of the edge sample (events on every face, edge and corner of the box) whose
    start matrices come from the single-precision pass (strategy 5) or a subsample (strategy
    3): the single-precision staging meets cos = +-1 (a zero basis column), phi = +-pi and the
    window edges, and the fits reach the minima of strategy 2."""
    cols, w = data(kind, weighted)
    b = _batch(gpu_lib, kind, cols, w, 4, precompute=precompute)
    step = np.array([2.0, 1.0, 2e-4, 0.02]) if kind == M1 else np.array([1.0, 1.0] + [0.03] * 8 + [2e-4] + [0.03] * 6 + [0.02])
    lo, hi = np.zeros(len(step)), np.zeros(len(step))
    hi[-1] = 1.0
    th0 = (synth.TRUTH_1D if kind == M1 else synth.TRUTH_4D) + 0.3 * step
    r = {st: b.fit(th0, lo=lo, hi=hi, step=step, tol_edm=1e-14, strategy=st, hessian=2) for st in (2, 3, 5)}
    b.close()
    for st in (3, 5):
        assert np.all(r[st]["status"] == 0) and np.all(r[2]["status"] == 0)
        assert np.max(np.abs(r[st]["theta"] - r[2]["theta"]) / r[2]["err"]) < 1e-6
        np.testing.assert_allclose(r[st]["err"], r[2]["err"], rtol=1e-6)


# --------------------------------------------------------------------------------------
# served fits (device-side hoisting at every step of the fit) against the oracle's fits
# --------------------------------------------------------------------------------------
@pytest.mark.parametrize("alpha_fixed", [0.0, 1e-4 / D, None])
def test_served_fit_edges(gpu_lib, alpha_fixed):
    """Mass-model fits of a sample with a flat background (alpha = 0): with alpha fixed at 0
    (the alpha == 0 branch at every step), fixed inside the series branch, and free (the fit
    ends at |alpha D| well below 1/2, the series branch of the analytic Hessian).  Strategy 2
    and hessian 2: analytic start matrix at admission, Newton polish at poll."""
    from paper_2505_12414_gb300.serve import Request, serve

    truth = np.array([5279.6, 20.0, 0.0, 0.3])
    cols = synth.mass1d(10000, stream=8950, theta=truth)
    fixed = np.zeros(4, dtype=np.int32)
    th0 = truth + np.array([1.0, 0.5, 0.0, 0.01])
    if alpha_fixed is not None:
        fixed[2] = 1
        th0[2] = alpha_fixed
    else:
        th0[2] = 1e-5
    lo, hi = np.zeros(4), np.zeros(4)
    hi[3] = 1.0
    step = np.array([2.0, 1.0, 2e-4, 0.02])
    srv = gpu_lib.Server(M1, synth.RANGES_1D, 2, 20000, 1024, lo=lo, hi=hi, step=step, fixed=fixed,
                         tol_edm=1e-14, strategy=2, hessian=2)
    req = Request(0, M1, cols, th0, 0.0)
    serve({M1: srv}, [req], realtime=False)
    srv.close()
    r = req.result
    assert r["status"] == 0
    ref = ofit.fit(M1, synth.RANGES_1D, cols, th0, tol_edm=1e-18, nthreads=8, h0=step * 1e-2, fixed=fixed)
    assert ref["converged"]
    free = fixed == 0
    pull = (r["theta"][free] - ref["theta"][free]) / ref["err"][free]
    assert np.max(np.abs(pull)) < 1e-6, pull
    np.testing.assert_allclose(r["err"][free], ref["err"][free], rtol=1e-4)
    if alpha_fixed is not None:
        assert r["theta"][2] == alpha_fixed and r["err"][2] == 0.0
    else:
        assert abs(r["theta"][2] * D) < 0.5


# --------------------------------------------------------------------------------------
# the exponent-range guard: |alpha| (mb - ma) + max(ln b1, 0) > 700 is rejected
# --------------------------------------------------------------------------------------
def test_exponent_range_guard(gpu_lib):
    import torch

    for kind in (M1, M4):
        cols, _ = data(kind, False)
        th = theta_of(kind, "alpha_zero")
        th[2 if kind == M1 else 10] = 701.0 / D
        m = gpu_lib.Model(kind, ranges_of(kind)).load(cols)
        nll, g, st = gpu_lib.nll_eval_grad(m.handle, th, check=False)
        assert st == gpu_lib.NLL_ERR_ARG
        _, st = gpu_lib.nll_eval(m.handle, th, check=False)
        assert st == gpu_lib.NLL_ERR_ARG
        with pytest.raises(gpu_lib.NLLError) as e:
            m.eval_hess(th)
        assert e.value.status == gpu_lib.NLL_ERR_ARG
        # just inside the range the point is evaluated (the plain form of the oracle overflows
        # exp(alpha m) there, the kernels' factored form does not)
        ok = th.copy()
        ok[2 if kind == M1 else 10] = 690.0 / D
        nll, g, st = gpu_lib.nll_eval_grad(m.handle, ok, check=False)
        assert st == gpu_lib.NLL_OK and np.isfinite(nll) and np.all(np.isfinite(g))
        m.close()
        b = _batch(gpu_lib, kind, cols, None, 2)
        _, _, st = b.eval_grad(np.array([th, theta_of(kind, "alpha_zero")]))
        assert st[0] == gpu_lib.NLL_ERR_ARG and st[1] == gpu_lib.NLL_OK
        b.close()
    cols, _ = data(M4, False)
    dev = [torch.from_numpy(c).to("cuda") for c in cols]
    th = theta_of(M4, "alpha_zero")
    th[10] = -701.0 / D
    _, _, st = gpu_lib.nll_eval_grad_4d_noalloc(synth.RANGES_4D, dev, th, check=False)
    assert st == gpu_lib.NLL_ERR_ARG
