"""Pins of the oracle against what the paper and the mathematics fix (CPU only).

Each test checks the oracle against something other than itself: printed constants of
the paper, a second form of the same quantity that the paper states (hoisted terms,
the exponential-only kernel), a library routine for a special case, brute-force
quadrature, high-precision arithmetic, or a closed-form maximum-likelihood solution.
"""
import math
import os

import mpmath as mp
import numpy as np
import pytest
from numpy.polynomial.legendre import leggauss

import oracle
from oracle import fit as ofit
from paper_2505_12414_gb300 import synth

M1, M4 = oracle.MASS1D, oracle.KSTAR4D
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def gl_panels(lo, hi, panels, order):
    x, w = leggauss(order)
    edges = np.linspace(lo, hi, panels + 1)
    xs, ws = [], []
    for a, b in zip(edges[:-1], edges[1:]):
        xs.append(0.5 * (b - a) * x + 0.5 * (a + b))
        ws.append(0.5 * (b - a) * w)
    return np.concatenate(xs), np.concatenate(ws)


MASS_THETAS = [
    synth.TRUTH_1D,
    np.array([5300.0, 35.0, 0.0, 0.6]),          # alpha == 0 branch
    np.array([5180.0, 12.0, 0.003, 0.5]),        # Gaussian cut by the lower edge, rising exponential
    np.array([5900.0, 60.0, -0.006, 0.1]),       # Gaussian near the upper edge
]


# --------------------------------------------------------------------------------------
# normalisation (paper Eq. 2: N1 and N2 normalise each component over the window)
# --------------------------------------------------------------------------------------
@pytest.mark.parametrize("theta", MASS_THETAS)
def test_mass_density_integrates_to_one(theta):
    x, w = gl_panels(5170.0, 5970.0, 200, 16)
    p = oracle.pdf(M1, synth.RANGES_1D, theta, [x])
    assert abs(np.dot(w, p) - 1.0) < 1e-12


def test_mass_density_integrates_to_one_gev_paper_set():
    x, w = gl_panels(5.0, 7.0, 200, 16)
    p = oracle.pdf(M1, synth.RANGES_1D_GEV, synth.TRUTH_1D_GEV, [x])
    assert abs(np.dot(w, p) - 1.0) < 1e-12


# --------------------------------------------------------------------------------------
# special cases reducing to library routines (catches swapped fsig / 1 - fsig, signs)
# --------------------------------------------------------------------------------------
def test_pure_components_match_scipy():
    from scipy import stats

    ma, mb = synth.MASS_WINDOW
    m = np.linspace(ma, mb, 1001)
    mu, sig = 5279.6, 20.0
    # fsig = 1: truncated normal
    p = oracle.pdf(M1, synth.RANGES_1D, [mu, sig, -0.002, 1.0], [m])
    ref = stats.truncnorm.pdf(m, (ma - mu) / sig, (mb - mu) / sig, loc=mu, scale=sig)
    np.testing.assert_allclose(p, ref, rtol=1e-11, atol=0)
    # fsig = 0, falling exponential: truncated exponential from ma
    al = -0.002
    p = oracle.pdf(M1, synth.RANGES_1D, [mu, sig, al, 0.0], [m])
    ref = stats.truncexpon.pdf(m, b=-al * (mb - ma), loc=ma, scale=-1.0 / al)
    np.testing.assert_allclose(p, ref, rtol=1e-11, atol=0)
    # fsig = 0, rising exponential: mirror image about mb
    al = 0.004
    p = oracle.pdf(M1, synth.RANGES_1D, [mu, sig, al, 0.0], [m])
    ref = stats.truncexpon.pdf(mb - m, b=al * (mb - ma), loc=0.0, scale=1.0 / al)
    np.testing.assert_allclose(p, ref, rtol=1e-11, atol=0)
    # fsig = 0, alpha = 0: uniform
    p = oracle.pdf(M1, synth.RANGES_1D, [mu, sig, 0.0, 0.0], [m])
    np.testing.assert_allclose(p, 1.0 / (mb - ma), rtol=1e-15)
    # mixture is linear in fsig
    pa = oracle.pdf(M1, synth.RANGES_1D, [mu, sig, -0.002, 1.0], [m])
    pb = oracle.pdf(M1, synth.RANGES_1D, [mu, sig, -0.002, 0.0], [m])
    pm = oracle.pdf(M1, synth.RANGES_1D, [mu, sig, -0.002, 0.3], [m])
    np.testing.assert_allclose(pm, 0.3 * pa + 0.7 * pb, rtol=1e-14)


# --------------------------------------------------------------------------------------
# the paper's exponential-only kernel (Sec. 2.3.1 listing): window [5, 7], alpha == 0
# branch with the printed normalisation 2.0
# --------------------------------------------------------------------------------------
@pytest.mark.parametrize("alpha", [-1.0, 0.0, 0.37, -0.05])
def test_exponential_kernel_listing_gev(alpha):
    m = np.linspace(5.0, 7.0, 257)
    p = oracle.pdf(M1, [5.0, 7.0], [5.28, 0.06, alpha, 0.0], [m])
    if alpha == 0.0:
        norm = 2.0  # printed constant of the alpha == 0 branch
    else:
        norm = (math.exp(7.0 * alpha) - math.exp(5.0 * alpha)) / alpha
    ref = alpha * m - math.log(norm)
    np.testing.assert_allclose(np.log(p), ref, rtol=0, atol=2e-14)


@pytest.mark.parametrize("alpha", [-1e-9, 3e-13, -2e-6])
def test_exponential_normalisation_small_slope_40_digits(alpha):
    # the printed form (e^{7a} - e^{5a})/a cancels for tiny |a|; the integral itself does not
    m = np.linspace(5.0, 7.0, 33)
    p = oracle.pdf(M1, [5.0, 7.0], [5.28, 0.06, alpha, 0.0], [m])
    with mp.workdps(40):
        a = mp.mpf(alpha)
        ref = [float(mp.exp(a * mp.mpf(float(x))) * a / (mp.exp(7 * a) - mp.exp(5 * a))) for x in m]
    np.testing.assert_allclose(p, ref, rtol=4e-16)


def test_alpha_zero_branch_is_continuous():
    ma, mb = synth.MASS_WINDOW
    D = mb - ma
    z = oracle.mass_norms(ma, mb, 5279.6, 20.0, 0.0)
    assert z["N2"] == D
    assert z["dlnN2_dalpha"] == 0.5 * (ma + mb)
    for a in (1e-12, -1e-12, 1e-7, -1e-7):
        n = oracle.mass_norms(ma, mb, 5279.6, 20.0, a)
        t = a * D
        assert abs(n["N2"] / (math.exp(a * ma) * D * (1 + t / 2 + t * t / 6 + t ** 3 / 24)) - 1.0) < 1e-14
    # across the switch between the closed form and the series (|alpha D| = 1e-3)
    for t in (1e-3 * (1 - 1e-9), 1e-3 * (1 + 1e-9)):
        a = t / D
        n = oracle.mass_norms(ma, mb, 5279.6, 20.0, a)
        with mp.workdps(50):
            am = mp.mpf(a)
            ref = ma + D * mp.e ** (am * D) / (mp.e ** (am * D) - 1) - 1 / am
        assert abs(n["dlnN2_dalpha"] - float(ref)) < 1e-12 * abs(float(ref))


# --------------------------------------------------------------------------------------
# hoisted form of Sec. 2.4.1 (b0, b1, b2 and the optimised kernel) equals the plain P
# --------------------------------------------------------------------------------------
@pytest.mark.parametrize("theta", MASS_THETAS)
def test_hoisted_terms_reproduce_density(theta):
    mu, sig, al, f = theta
    ma, mb = synth.MASS_WINDOW
    b0 = 1.0 / (2.0 * sig ** 2)
    b1 = f / (math.sqrt(2 * math.pi) * sig) / (
        0.5 * (math.erf((mu - ma) / (math.sqrt(2) * sig)) - math.erf((mu - mb) / (math.sqrt(2) * sig))))
    b2 = (1.0 - f) / ((mb - ma) if al == 0.0 else (math.exp(al * mb) - math.exp(al * ma)) / al)
    m = synth.mass1d(2000, theta=theta)[0]
    lnp_hoisted = np.log(np.exp(-((m - mu) ** 2) * b0) * b1 + np.exp(m * al) * b2)
    lnp = np.log(oracle.pdf(M1, synth.RANGES_1D, theta, [m]))
    np.testing.assert_allclose(lnp, lnp_hoisted, rtol=2e-14, atol=0)


# --------------------------------------------------------------------------------------
# angular basis: the printed prefactors of the paper's precompute kernel
# --------------------------------------------------------------------------------------
def _read_golden_basis():
    rows = []
    with open(os.path.join(GOLDEN, "angular_basis_prefactors.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            col, mono, pref, coef = line.split()
            rows.append((int(col), mono, float(pref), coef))
    return rows


def _monomial(name, ctl, ctk, phi):
    sl, sk = np.sqrt(1 - ctl ** 2), np.sqrt(1 - ctk ** 2)
    return {
        "s2phi_sl2_sk2": np.sin(2 * phi) * (1 - ctl ** 2) * (1 - ctk ** 2),
        "sphi_ctksk_ctlsl": np.sin(phi) * ctk * sk * ctl * sl,
        "sphi_sl_ctksk": np.sin(phi) * sl * ctk * sk,
        "ctl_sk2": ctl * (1 - ctk ** 2),
        "cphi_sl_ctksk": np.cos(phi) * sl * ctk * sk,
        "cphi_ctksk_ctlsl": np.cos(phi) * ctk * sk * ctl * sl,
        "c2phi_sl2_sk2": np.cos(2 * phi) * (1 - ctl ** 2) * (1 - ctk ** 2),
        "c2l_ck2": (2 * ctl ** 2 - 1) * ctk ** 2,
        "c2l_sk2": (2 * ctl ** 2 - 1) * (1 - ctk ** 2),
        "sk2": 1 - ctk ** 2,
        "ck2": ctk ** 2,
    }[name]


def _coef(expr, FL, S3, S4, S5, AFB, S7, S8, S9):
    return {"S9": S9, "S8": S8, "S7": S7, "AFB": AFB, "S5": S5, "S4": S4, "S3": S3,
            "-FL": -FL, "1-FL": 1 - FL, "FL": FL}[expr]


def test_printed_prefactors_are_nine_over_32pi_multiples():
    c = 9.0 / (32.0 * math.pi)
    mult = {"s2phi_sl2_sk2": 1, "sphi_ctksk_ctlsl": 4, "sphi_sl_ctksk": 2, "ctl_sk2": 4 / 3,
            "cphi_sl_ctksk": 2, "cphi_ctksk_ctlsl": 4, "c2phi_sl2_sk2": 1, "c2l_ck2": 1,
            "c2l_sk2": 0.25, "sk2": 0.75, "ck2": 1}
    for _, mono, pref, _ in _read_golden_basis():
        assert abs(pref / (mult[mono] * c) - 1.0) < 2e-15


def test_angular_rate_matches_printed_basis():
    rs = synth.Stream(11, 0)
    n = 5000
    ctl, ctk = 2 * rs.uniform(n) - 1, 2 * rs.uniform(n) - 1
    phi = math.pi * (2 * rs.uniform(n) - 1)
    rows = _read_golden_basis()
    for trial in range(5):
        pars = (rs.uniform(8) - 0.5) * 0.4
        pars[0] = 0.2 + 0.6 * rs.uniform(1)[0]  # FL
        theta = synth.TRUTH_4D.copy()
        theta[2:10] = pars
        # A via the printed columns and pairing
        A_printed = sum(pref * _monomial(mono, ctl, ctk, phi) * _coef(coef, *pars) for _, mono, pref, coef in rows)
        # A via the oracle: fsig = 1 density divided by the (angle-independent) Gaussian
        m = np.full(n, 5279.6)
        p4 = oracle.pdf(M4, synth.RANGES_4D, np.concatenate([theta[:17], [1.0]]), [m, ctl, ctk, phi])
        g = oracle.pdf(M1, synth.RANGES_1D, [theta[0], theta[1], theta[10], 1.0], [m])
        np.testing.assert_allclose(p4 / g, A_printed, rtol=1e-13, atol=1e-16)
        # and term by term: the oracle's eleven terms against the printed columns
    terms = oracle.angular_terms(ctl, ctk, phi)
    by_mono = {mono: pref * _monomial(mono, ctl, ctk, phi) for _, mono, pref, _ in rows}
    np.testing.assert_allclose(terms[:, 0], by_mono["sk2"], rtol=1e-14, atol=1e-17)
    np.testing.assert_allclose(terms[:, 1], by_mono["ck2"], rtol=1e-14, atol=1e-17)
    np.testing.assert_allclose(terms[:, 2], by_mono["c2l_sk2"], rtol=1e-14, atol=1e-17)
    np.testing.assert_allclose(terms[:, 3], by_mono["c2l_ck2"], rtol=1e-14, atol=1e-17)
    for k, mono in enumerate(["c2phi_sl2_sk2", "cphi_ctksk_ctlsl", "cphi_sl_ctksk", "ctl_sk2",
                              "sphi_sl_ctksk", "sphi_ctksk_ctlsl", "s2phi_sl2_sk2"]):
        np.testing.assert_allclose(terms[:, 4 + k], by_mono[mono], rtol=1e-13, atol=1e-17)


def test_angular_rate_integrates_to_one_for_any_coefficients():
    xl, wl = leggauss(24)
    xp, wp = gl_panels(-math.pi, math.pi, 8, 12)
    L, K, P = np.meshgrid(xl, xl, xp, indexing="ij")
    W = (wl[:, None, None] * wl[None, :, None] * wp[None, None, :]).ravel()
    ctl, ctk, phi = L.ravel(), K.ravel(), P.ravel()
    rs = synth.Stream(5, 1)
    for _ in range(4):
        th = synth.TRUTH_4D.copy()
        th[2:10] = rs.uniform(8) - 0.5
        th[17] = 1.0
        m = np.full(len(ctl), th[0])
        g = oracle.pdf(M1, synth.RANGES_1D, [th[0], th[1], th[10], 1.0], m[:1])[0]
        p = oracle.pdf(M4, synth.RANGES_4D, th, [m, ctl, ctk, phi]) / g
        assert abs(np.dot(W, p) - 1.0) < 1e-13


def test_angular_terms_integrals_closed_form():
    # f1..f4 integrate to 9/8, 3/4, -1/8, -1/4 (so that A integrates to 1); f5..f11 to 0
    xl, wl = leggauss(24)
    xp, wp = gl_panels(-math.pi, math.pi, 8, 12)
    L, K, P = np.meshgrid(xl, xl, xp, indexing="ij")
    W = (wl[:, None, None] * wl[None, :, None] * wp[None, None, :]).ravel()
    t = oracle.angular_terms(L.ravel(), K.ravel(), P.ravel())
    ints = W @ t
    np.testing.assert_allclose(ints[:4], [9 / 8, 3 / 4, -1 / 8, -1 / 4], rtol=1e-13)
    np.testing.assert_allclose(ints[4:], 0.0, atol=1e-14)


def test_chebyshev_background_matches_numpy():
    from numpy.polynomial import chebyshev as C

    rs = synth.Stream(3, 2)
    n = 3000
    x1, x2 = 2 * rs.uniform(n) - 1, 2 * rs.uniform(n) - 1
    phi = math.pi * (2 * rs.uniform(n) - 1)
    m = 5170 + 800 * rs.uniform(n)
    th = synth.TRUTH_4D.copy()
    th[11:17] = [0.3, -0.2, -0.15, 0.25, 0.1, 0.05]
    th[17] = 0.0
    p4 = oracle.pdf(M4, synth.RANGES_4D, th, [m, x1, x2, phi])
    e = oracle.pdf(M1, synth.RANGES_1D, [th[0], th[1], th[10], 0.0], [m])
    ref = np.ones(n)
    for j, x in enumerate([x1, x2, phi / math.pi]):
        coef = [1.0, th[11 + 2 * j], th[12 + 2 * j]]
        # normalise by Gauss-Legendre quadrature of the Chebyshev series over the observable
        xq, wq = leggauss(8)
        nrm = np.dot(wq, C.chebval(xq, coef)) * (math.pi if j == 2 else 1.0)
        ref *= C.chebval(x, coef) / nrm
    np.testing.assert_allclose(p4 / e, ref, rtol=1e-13)


def test_4d_density_integrates_to_one():
    xm, wm = gl_panels(5170.0, 5970.0, 100, 8)
    xl, wl = leggauss(10)
    xp, wp = gl_panels(-math.pi, math.pi, 4, 10)
    M, L, K, P = np.meshgrid(xm, xl, xl, xp, indexing="ij")
    W = (wm[:, None, None, None] * wl[None, :, None, None] * wl[None, None, :, None]
         * wp[None, None, None, :]).ravel()
    p = oracle.pdf(M4, synth.RANGES_4D, synth.TRUTH_4D, [M.ravel(), L.ravel(), K.ravel(), P.ravel()])
    assert abs(np.dot(W, p) - 1.0) < 1e-11


# --------------------------------------------------------------------------------------
# accept-reject bound (paper appendix, get_max of the angular PDF) and positivity at truth
# --------------------------------------------------------------------------------------
def test_angular_rate_below_paper_bound_and_nonnegative_at_truth():
    g = np.linspace(-1, 1, 64)
    gp = np.linspace(-math.pi, math.pi, 64)
    L, K, P = np.meshgrid(g, g, gp, indexing="ij")
    ctl, ctk, phi = L.ravel(), K.ravel(), P.ravel()
    t = oracle.angular_terms(ctl, ctk, phi)
    rs = synth.Stream(9, 3)
    for trial in range(6):
        pars = synth.TRUTH_4D[2:10] if trial == 0 else (rs.uniform(8) - 0.5) * 0.6
        FL, S3, S4, S5, AFB, S7, S8, S9 = pars
        S = np.array([1 - FL, FL, 1 - FL, -FL, S3, S4, S5, AFB, S7, S8, S9])
        A = t @ S
        bound = 9 / (32 * math.pi) * (4 + abs(S3) + abs(S4) + abs(S5) + 4 / 3 * abs(AFB) + abs(S7) + abs(S8)
                                      + abs(S9))
        assert A.max() <= bound
        if trial == 0:
            assert A.min() >= -1e-15


# --------------------------------------------------------------------------------------
# high-precision references: the NLL of a few events at 40 digits, and its derivatives
# by numerical differentiation at that precision
# --------------------------------------------------------------------------------------
def _mp_nll(kind, ranges, cols, theta):
    """NLL at the caller's mpmath precision (set mp.mp.dps before calling)."""
    ma, mb = mp.mpf(ranges[0]), mp.mpf(ranges[1])
    th = [t if isinstance(t, mp.mpf) else mp.mpf(float(t)) for t in theta]

    def gauss(m, mu, s):
        n1 = (mp.erf((mu - ma) / (mp.sqrt(2) * s)) - mp.erf((mu - mb) / (mp.sqrt(2) * s))) / 2
        return mp.exp(-(m - mu) ** 2 / (2 * s ** 2)) / (mp.sqrt(2 * mp.pi) * s * n1)

    def expo(m, a):
        n2 = (mb - ma) if a == 0 else (mp.exp(a * mb) - mp.exp(a * ma)) / a
        return mp.exp(a * m) / n2

    tot = mp.mpf(0)
    for i in range(len(cols[0])):
        m = mp.mpf(float(cols[0][i]))
        if kind == M1:
            mu, s, a, f = th
            p = f * gauss(m, mu, s) + (1 - f) * expo(m, a)
        else:
            mu, s, FL, S3, S4, S5, AFB, S7, S8, S9, a, c1l, c2l, c1k, c2k, c1p, c2p, f = th
            cl, ck, ph = (mp.mpf(float(cols[d][i])) for d in (1, 2, 3))
            sl, sk = mp.sqrt(1 - cl ** 2), mp.sqrt(1 - ck ** 2)
            cos2l = 2 * cl ** 2 - 1
            s2l, s2k = 2 * sl * cl, 2 * sk * ck
            A = 9 / (32 * mp.pi) * (
                (1 - FL) * mp.mpf(3) / 4 * sk ** 2 + FL * ck ** 2 + (1 - FL) / 4 * sk ** 2 * cos2l
                - FL * ck ** 2 * cos2l + S3 * sk ** 2 * sl ** 2 * mp.cos(2 * ph) + S4 * s2k * s2l * mp.cos(ph)
                + S5 * s2k * sl * mp.cos(ph) + AFB * mp.mpf(4) / 3 * sk ** 2 * cl + S7 * s2k * sl * mp.sin(ph)
                + S8 * s2k * s2l * mp.sin(ph) + S9 * sk ** 2 * sl ** 2 * mp.sin(2 * ph))
            B = mp.mpf(1)
            for x, c1, c2, sc in ((cl, c1l, c2l, 1), (ck, c1k, c2k, 1), (ph / mp.pi, c1p, c2p, mp.pi)):
                B *= (1 + c1 * x + c2 * (2 * x ** 2 - 1)) / (sc * (2 - mp.mpf(2) / 3 * c2))
            p = f * gauss(m, mu, s) * A + (1 - f) * expo(m, a) * B
        tot -= mp.log(p)
    return tot


@pytest.mark.parametrize("kind,n", [(M1, 1), (M1, 7), (M1, 16), (M4, 1), (M4, 5), (M4, 16)])
def test_tiny_n_against_40_digit_arithmetic(kind, n):
    if kind == M1:
        cols, ranges, theta = synth.mass1d(n, stream=40 + n), synth.RANGES_1D, synth.TRUTH_1D
    else:
        cols, ranges, theta = synth.kstar4d(n, stream=40 + n), synth.RANGES_4D, synth.TRUTH_4D
    nll, g, _, st = oracle.nll_grad(kind, ranges, cols, theta)
    assert st == 0
    mp.mp.dps = 40
    ref = _mp_nll(kind, ranges, cols, theta)
    assert abs(nll - float(ref)) <= 4e-15 * abs(float(ref))


@pytest.mark.parametrize("kind", [M1, M4])
def test_gradient_against_40_digit_differentiation(kind):
    n = 12
    if kind == M1:
        cols, ranges = synth.mass1d(n, stream=77), synth.RANGES_1D
        theta = np.array([5283.0, 22.0, -0.0017, 0.35])
    else:
        cols, ranges = synth.kstar4d(n, stream=78), synth.RANGES_4D
        theta = synth.TRUTH_4D + 0.01
    _, g, sc, st = oracle.nll_grad(kind, ranges, cols, theta)
    assert st == 0
    for k in range(len(theta)):
        def f(x, k=k):
            t = [mp.mpf(float(v)) for v in theta]
            t[k] = x
            return _mp_nll(kind, ranges, cols, t)
        mp.mp.dps = 40
        ref = float(mp.diff(f, mp.mpf(float(theta[k]))))
        assert abs(g[k] - ref) <= 1e-12 * abs(ref) + 1e-14 * sc[k], (k, g[k], ref)


@pytest.mark.parametrize("kind", [M1, M4])
def test_gradient_against_central_differences(kind):
    if kind == M1:
        cols, ranges, theta = synth.mass1d(3000, stream=5), synth.RANGES_1D, synth.TRUTH_1D
    else:
        cols, ranges, theta = synth.kstar4d(3000, stream=6), synth.RANGES_4D, synth.TRUTH_4D
    _, g, sc, _ = oracle.nll_grad(kind, ranges, cols, theta)
    for k in range(len(theta)):
        h = 1e-6 * max(abs(theta[k]), 1e-2)
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        fd = (oracle.nll_grad(kind, ranges, cols, tp, grad=False)[0]
              - oracle.nll_grad(kind, ranges, cols, tm, grad=False)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * abs(g[k]) + 1e-7 * sc[k], (k, fd, g[k])


# --------------------------------------------------------------------------------------
# closed-form maximum-likelihood solutions
# --------------------------------------------------------------------------------------
def test_pure_gaussian_mle_is_sample_mean_and_std():
    # window 40 sigma wide on both sides: the truncation is below double precision, so
    # the MLE of (mu, sigma) is the sample mean and the 1/N standard deviation.
    mu0, s0 = 5500.0, 5.0
    ranges = [mu0 - 200.0, mu0 + 200.0]
    m = synth.mass1d(5000, stream=9, theta=[mu0, s0, 0.0, 1.0], ranges=ranges)[0]
    mhat, shat = m.mean(), m.std()
    _, g, sc, _ = oracle.nll_grad(M1, ranges, [m], [mhat, shat, 0.0, 1.0])
    assert abs(g[0]) < 1e-12 * sc[0]
    assert abs(g[1]) < 1e-12 * sc[1]


def test_pure_exponential_mle_matches_quadrature_moment():
    from scipy import integrate, optimize

    ma, mb = synth.MASS_WINDOW
    m = synth.mass1d(20000, stream=10, theta=[5279.6, 20.0, -0.0025, 0.0])[0]
    mbar = m.mean()

    def mean_of(alpha):  # mean of exp(alpha m) on the window, by adaptive quadrature
        num = integrate.quad(lambda x: x * math.exp(alpha * (x - ma)), ma, mb, epsabs=0, epsrel=1e-13)[0]
        den = integrate.quad(lambda x: math.exp(alpha * (x - ma)), ma, mb, epsabs=0, epsrel=1e-13)[0]
        return num / den

    ahat = optimize.brentq(lambda a: mean_of(a) - mbar, -0.01, 0.01, xtol=1e-16, rtol=1e-15)
    _, g, sc, _ = oracle.nll_grad(M1, synth.RANGES_1D, [m], [5279.6, 20.0, ahat, 0.0])
    assert abs(g[2]) < 1e-9 * sc[2]


# --------------------------------------------------------------------------------------
# summation: thread count does not change the result beyond Kahan rounding; repeatable
# --------------------------------------------------------------------------------------
def test_threads_and_repeatability():
    cols = synth.kstar4d(40000, stream=12)
    a = oracle.nll_grad(M4, synth.RANGES_4D, cols, synth.TRUTH_4D, nthreads=1)
    b = oracle.nll_grad(M4, synth.RANGES_4D, cols, synth.TRUTH_4D, nthreads=8)
    c = oracle.nll_grad(M4, synth.RANGES_4D, cols, synth.TRUTH_4D, nthreads=8)
    assert abs(a[0] - b[0]) <= 1e-15 * abs(a[0])
    np.testing.assert_allclose(a[1], b[1], rtol=1e-13, atol=1e-15 * a[2].max())
    assert b[0] == c[0] and np.array_equal(b[1], c[1])


def test_weights_enter_linearly():
    cols = synth.mass1d(5000, stream=13)
    w = synth.weights(5000)
    a = oracle.nll_grad(M1, synth.RANGES_1D, cols, synth.TRUTH_1D, w=w)
    b = oracle.nll_grad(M1, synth.RANGES_1D, cols, synth.TRUTH_1D, w=2.0 * w)
    assert abs(b[0] - 2 * a[0]) <= 1e-15 * abs(b[0])
    lp = np.log(oracle.pdf(M1, synth.RANGES_1D, synth.TRUTH_1D, cols))
    assert abs(a[0] + np.dot(w, lp)) <= 1e-12 * abs(a[0])


def test_nonpositive_density_is_flagged():
    cols = synth.kstar4d(2000, stream=14)
    th = synth.TRUTH_4D.copy()
    th[6] = 3.0  # AFB far outside the physical region makes A negative somewhere
    th[17] = 0.999
    nll, _, _, st = oracle.nll_grad(M4, synth.RANGES_4D, cols, th)
    assert st == oracle.ERR_NONPOSITIVE and nll == math.inf


# --------------------------------------------------------------------------------------
# statistical pin: pulls of fitted parameters over pseudo-experiments (paper Sec. 2.5 /
# Sec. 3.1 validate fits this way): mean 0 and width 1
# --------------------------------------------------------------------------------------
@pytest.mark.slow
def test_pulls_mass_model():
    ntoy, nev = 1000, 1000
    truth = synth.TRUTH_1D
    pulls = []
    for t in range(ntoy):
        m = synth.mass1d(nev, stream=500000 + t)
        r = ofit.fit(M1, synth.RANGES_1D, m, truth, tol_edm=1e-10, h0=[0.5, 0.5, 2e-5, 0.02])
        assert r["converged"]
        pulls.append((r["theta"] - truth) / r["err"])
    pulls = np.array(pulls)
    mean, width = pulls.mean(axis=0), pulls.std(axis=0)
    # 4 sigma statistical bands for 600 toys
    assert np.all(np.abs(mean) < 4.0 / math.sqrt(ntoy) + 0.02), mean
    assert np.all(np.abs(width - 1.0) < 4.0 / math.sqrt(2 * ntoy) + 0.02), width


@pytest.mark.slow
def test_pulls_4d_model():
    ntoy, nev = 200, 2000
    truth = synth.TRUTH_4D
    h0 = np.maximum(np.abs(truth), 0.05) * 1e-3
    pulls = []
    for t in range(ntoy):
        cols = synth.kstar4d(nev, stream=600000 + t)
        r = ofit.fit(M4, synth.RANGES_4D, cols, truth, tol_edm=1e-10, h0=h0)
        assert r["converged"]
        pulls.append((r["theta"] - truth) / r["err"])
    pulls = np.array(pulls)
    mean, width = pulls.mean(axis=0), pulls.std(axis=0)
    assert np.all(np.abs(mean) < 4.0 / math.sqrt(ntoy)), mean
    assert np.all(np.abs(width - 1.0) < 4.0 / math.sqrt(2 * ntoy)), width


# --------------------------------------------------------------------------------------
# second derivatives: the Hessian of the NLL (HESSE uncertainties) and the squared-weight
# score matrix W = sum w^2 s s^T of the weighted-fit sandwich covariance
# --------------------------------------------------------------------------------------
def _hess_case(kind, n, stream):
    if kind == M1:
        return synth.mass1d(n, stream=stream), synth.RANGES_1D, np.array([5283.0, 22.0, -0.0017, 0.35])
    return synth.kstar4d(n, stream=stream), synth.RANGES_4D, synth.TRUTH_4D + 0.01


@pytest.mark.parametrize("kind,n", [(M1, 6), (M4, 3)])
def test_hessian_against_40_digit_differentiation(kind, n):
    cols, ranges, theta = _hess_case(kind, n, 90 + kind)
    r = oracle.nll_hess(kind, ranges, cols, theta)
    assert r["status"] == 0
    H, hs = r["hess"], r["hscale"]
    npar = len(theta)
    mp.mp.dps = 40
    t0 = [mp.mpf(float(v)) for v in theta]
    for a in range(npar):
        for b in range(a, npar):
            if a == b:
                def f1(x, a=a):
                    t = list(t0)
                    t[a] = x
                    return _mp_nll(kind, ranges, cols, t)
                ref = mp.diff(f1, t0[a], 2)
            else:
                def f2(x, y, a=a, b=b):
                    t = list(t0)
                    t[a], t[b] = x, y
                    return _mp_nll(kind, ranges, cols, t)
                ref = mp.diff(f2, (t0[a], t0[b]), (1, 1))
            ref = float(ref)
            assert abs(H[a, b] - ref) <= 1e-11 * abs(ref) + 1e-13 * hs[a, b], (a, b, H[a, b], ref)
            assert H[a, b] == H[b, a]


@pytest.mark.parametrize("mu,sigma", [(5279.6, 20.0), (5180.0, 12.0), (5900.0, 60.0), (5570.0, 300.0)])
def test_gaussian_normalisation_second_derivatives_40_digits(mu, sigma):
    ma, mb = synth.RANGES_1D
    mp.mp.dps = 40

    def lnN1(x, y):
        return mp.log((mp.erf((x - ma) / (mp.sqrt(2) * y)) - mp.erf((x - mb) / (mp.sqrt(2) * y))) / 2)

    r = oracle.mass_norms2(ma, mb, mu, sigma, 0.0)
    x0, y0 = mp.mpf(mu), mp.mpf(sigma)
    refs = [mp.diff(lnN1, (x0, y0), (2, 0)), mp.diff(lnN1, (x0, y0), (1, 1)), mp.diff(lnN1, (x0, y0), (0, 2))]
    got = [r["d2lnN1_mumu"], r["d2lnN1_musigma"], r["d2lnN1_sigmasigma"]]
    for g, ref in zip(got, refs):
        # the first-order terms carry the erf difference's relative rounding (~1e-16 / N1)
        assert abs(g - float(ref)) <= 1e-11 * abs(float(ref)) + 1e-20, (g, ref)


@pytest.mark.parametrize("alpha", [-0.002, 0.003, -5e-5, 1e-4, -1.3e-4, 6.1e-4, -6.2e-4, 6.3e-4, 0.0, 1e-9, 0.9])
def test_exponential_normalisation_second_derivative_is_the_variance(alpha):
    # d^2 ln N2 / d alpha^2 is the variance of m under exp(alpha m) on the window
    # (cumulant generating function); at alpha = 0 it is the uniform variance (mb-ma)^2/12.
    ma, mb = synth.RANGES_1D
    r = oracle.mass_norms2(ma, mb, 5279.6, 20.0, alpha)["d2lnN2_alpha"]
    mp.mp.dps = 40
    a = mp.mpf(alpha)
    w = lambda x: mp.exp(a * (x - ma))
    z = mp.quad(w, [ma, mb])
    m1 = mp.quad(lambda x: x * w(x), [ma, mb]) / z
    m2 = mp.quad(lambda x: (x - m1) ** 2 * w(x), [ma, mb]) / z
    assert abs(r - float(m2)) <= 1e-13 * float(m2), (alpha, r, m2)
    if alpha == 0.0:
        assert abs(r - (mb - ma) ** 2 / 12) <= 1e-15 * r


def test_hessian_pure_gaussian_closed_form():
    # f = 1 and a window 40 sigma wide: N1 = 1 exactly, so the (mu, sigma) block is the
    # textbook Gaussian one: sum 1/s^2, sum 2 d/s^3, sum (3 d^2/s^4 - 1/s^2).
    mu0, s0 = 5500.0, 5.0
    ranges = [mu0 - 200.0, mu0 + 200.0]
    m = synth.mass1d(4000, stream=91, theta=[mu0, s0, 0.0, 1.0], ranges=ranges)[0]
    th = [5501.0, 5.3, 0.0, 1.0]
    r = oracle.nll_hess(M1, ranges, [m], th)
    d = m - th[0]
    s = th[1]
    assert abs(r["hess"][0, 0] - len(m) / s ** 2) <= 1e-13 * len(m) / s ** 2
    ref01 = math.fsum(2 * d / s ** 3)
    assert abs(r["hess"][0, 1] - ref01) <= 1e-12 * math.fsum(abs(2 * d / s ** 3))
    ref11 = math.fsum(3 * d ** 2 / s ** 4 - 1 / s ** 2)
    assert abs(r["hess"][1, 1] - ref11) <= 1e-12 * math.fsum(3 * d ** 2 / s ** 4 + 1 / s ** 2)


def test_hessian_pure_exponential_is_n_times_variance():
    # f = 0: the alpha-alpha entry is N Var(m) under the fitted exponential, for any data
    for alpha in (-0.0025, 0.0, 2e-5):
        m = synth.mass1d(3000, stream=92, theta=[5279.6, 20.0, -0.0025, 0.0])[0]
        r = oracle.nll_hess(M1, synth.RANGES_1D, [m], [5279.6, 20.0, alpha, 0.0])
        v = oracle.mass_norms2(*synth.RANGES_1D, 5279.6, 20.0, alpha)["d2lnN2_alpha"]
        assert abs(r["hess"][2, 2] - len(m) * v) <= 1e-13 * len(m) * v


@pytest.mark.parametrize("kind", [M1, M4])
def test_hessian_against_central_differences_of_gradient(kind):
    cols, ranges, theta = _hess_case(kind, 3000, 93)
    r = oracle.nll_hess(kind, ranges, cols, theta)
    H, hs = r["hess"], r["hscale"]
    for k in range(len(theta)):
        h = 1e-5 * max(abs(theta[k]), 1e-2)
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        fd = (oracle.nll_grad(kind, ranges, cols, tp)[1] - oracle.nll_grad(kind, ranges, cols, tm)[1]) / (2 * h)
        assert np.all(np.abs(fd - H[:, k]) <= 1e-4 * np.abs(H[:, k]) + 1e-6 * hs[:, k]), (k, fd, H[:, k])


@pytest.mark.parametrize("kind", [M1, M4])
def test_score_matrix_and_weights(kind):
    cols, ranges, theta = _hess_case(kind, 2000, 94)
    w = synth.weights(2000, stream=95)
    r = oracle.nll_hess(kind, ranges, cols, theta, w=w)
    # W from the per-event scores (gradient code, pinned above) and the weights
    s = oracle.dlogpdf(kind, ranges, theta, cols)
    ref = (w[:, None] * s).T @ (w[:, None] * s)
    scale = np.sqrt(np.outer(np.diag(ref), np.diag(ref)))
    assert np.all(np.abs(r["w2"] - ref) <= 1e-12 * scale)
    # H and the per-event second derivatives
    d2 = oracle.d2logpdf(kind, ranges, theta, [c[:50] for c in cols])
    r50 = oracle.nll_hess(kind, ranges, [c[:50] for c in cols], theta, w=w[:50])
    assert np.all(np.abs(r50["hess"] + np.einsum("i,iab->ab", w[:50], d2)) <= 1e-13 * r50["hscale"])
    # weights enter H linearly and W quadratically; both symmetric
    r2 = oracle.nll_hess(kind, ranges, cols, theta, w=2.0 * w)
    assert np.array_equal(r2["hess"], 2.0 * r["hess"]) and np.array_equal(r2["w2"], 4.0 * r["w2"])
    assert np.array_equal(r["hess"], r["hess"].T) and np.array_equal(r["w2"], r["w2"].T)
    # the gradient returned with the Hessian is the one of nll_grad
    _, g, _, _ = oracle.nll_grad(kind, ranges, cols, theta, w=w)
    assert np.array_equal(r["grad"], g)


@pytest.mark.parametrize("kind,n", [(M1, 200000), (M4, 100000)])
def test_information_equality_at_the_truth(kind, n):
    # For a sample drawn from the model at the true parameters, E[-d^2 ln P] = E[s s^T]
    # (Bartlett's second identity), so H and W (w = 1) agree up to O(1/sqrt(n)) fluctuations.
    cols = synth.mass1d(n, stream=96) if kind == M1 else synth.kstar4d(n, stream=97)
    ranges, truth = (synth.RANGES_1D, synth.TRUTH_1D) if kind == M1 else (synth.RANGES_4D, synth.TRUTH_4D)
    r = oracle.nll_hess(kind, ranges, cols, truth, nthreads=8)
    H, W = r["hess"], r["w2"]
    eH = np.sqrt(np.diag(np.linalg.inv(H)))
    eW = np.sqrt(np.diag(np.linalg.inv(W)))
    assert np.all(np.abs(eH / eW - 1.0) < 0.03), eH / eW
    # off-diagonal structure too: correlations agree
    cH = np.linalg.inv(H) / np.outer(eH, eH)
    cW = np.linalg.inv(W) / np.outer(eW, eW)
    assert np.max(np.abs(cH - cW)) < 0.03


def test_hessian_scale_bounds_the_plain_form_cancellation():
    # two events deep in the background tail: the (fsig, alpha) entry is O(ps) while the two
    # terms of the plain form are O(1); 40-digit differentiation shows the oracle's error
    # stays within 1e-13 of the reported scale
    cols = synth.mass1d(2, stream=302)
    th = np.array([5283.0, 22.0, -0.0017, 0.35])
    r = oracle.nll_hess(M1, synth.RANGES_1D, cols, th)
    mp.mp.dps = 40
    t0 = [mp.mpf(float(v)) for v in th]

    def f2(x, y):
        t = list(t0)
        t[2], t[3] = x, y
        return _mp_nll(M1, synth.RANGES_1D, cols, t)

    ref = float(mp.diff(f2, (t0[2], t0[3]), (1, 1)))
    err = abs(r["hess"][2, 3] - ref)
    assert err > 1e-9 * abs(ref)  # the cancellation is real ...
    assert err <= 1e-13 * r["hscale"][2, 3]  # ... and the scale accounts for it


def two_valued_weights(n, stream):
    # weights independent of the events, 0.2 or 2 with equal probability:
    # E[w] = 1.1, E[w^2] = 2.02, so the weighted estimator's spread exceeds the inverse
    # Hessian's prediction by sqrt(E[w^2] / E[w]) = 1.36
    return np.where(synth.Stream(synth.BASE_SEED, stream).uniform(n) < 0.5, 0.2, 2.0)


def test_sandwich_covariance_matches_the_spread_of_weighted_fits():
    # statistical pin of reading "weighted-fit covariance": over pseudo-experiments with
    # weights unrelated to the data, the sandwich H^-1 W H^-1 predicts the spread of the fitted
    # values; the plain inverse Hessian does not
    ntoy, nev = 300, 2000
    fitted, sand, naive = [], [], []
    for t in range(ntoy):
        m = synth.mass1d(nev, stream=810000 + t)
        w = two_valued_weights(nev, 820000 + t)
        r = ofit.fit(M1, synth.RANGES_1D, m, synth.TRUTH_1D, w=w, tol_edm=1e-12, h0=[0.5, 0.5, 2e-5, 0.02])
        assert r["converged"]
        h = oracle.nll_hess(M1, synth.RANGES_1D, m, r["theta"], w=w)
        Hi = np.linalg.inv(h["hess"])
        fitted.append(r["theta"])
        sand.append(np.sqrt(np.diag(Hi @ h["w2"] @ Hi)))
        naive.append(np.sqrt(np.diag(Hi)))
    spread = np.std(np.array(fitted), axis=0)
    ratio_sand = spread / np.mean(np.array(sand), axis=0)
    ratio_naive = spread / np.mean(np.array(naive), axis=0)
    # the standard deviation of 300 values is known to ~4 %; 4 sigma bands
    assert np.all(np.abs(ratio_sand - 1.0) < 0.17), ratio_sand
    assert np.all(ratio_naive > 1.2), ratio_naive
