"""On-device generation (paper Sec. 2.5) against the oracle's density: binned goodness of fit.

The paper generates its pseudo-experiments on the accelerator by accept-reject, with every
parameter fixed so that parameter-only terms fold into constants (Sec. 2.5; the bound is the
appendix's get_max of the angular PDF).  Here 10^7 events are generated on the device at a
parameter point and histogrammed; each bin's probability is the integral of the oracle's
normalised density over the bin (composite Gauss-Legendre quadrature over the full
observable box, the other observables integrated out), and Pearson's chi^2 with
(bins - 1) degrees of freedom must have a p-value above 1e-3 (fixed seeds).

Histograms: 100 mass bins; for the 4D model also 50 bins in each angle and the 10 x 10 x 10
grid of (cos theta_l, cos theta_K, phi).  Points: the mass model at its truth, with alpha = 0
(flat background: the generator's uniform branch) and with |alpha (mb - ma)| small (the
generator's log1p branch); the 4D model at its truth, at alpha = 0, and at the paper's
angular point FL = 0.6 with the other coefficients 0 (Sec. 3.3, generated by the folded
kernel without phi or sin theta terms).  A planted mistake in the hypothesis (the oracle's
c2 of cos theta_l off by 0.02, a 2 % change of the background shape in that observable)
must fail the same test decisively, which shows it can see shape errors of that size.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2505_12414_gb300 import synth

pytestmark = pytest.mark.gpu

M1, M4 = oracle.MASS1D, oracle.KSTAR4D
N_EVENTS = 10_000_000
SEED = 20250518


def _axis(lo, hi, nbins, k):
    """Gauss-Legendre nodes and weights, k per bin, over nbins equal bins of [lo, hi]."""
    x, w = np.polynomial.legendre.leggauss(k)
    e = np.linspace(lo, hi, nbins + 1)
    a, b = e[:-1, None], e[1:, None]
    return (0.5 * (b - a) * x + 0.5 * (a + b)).ravel(), (0.5 * (b - a) * w).ravel()


def bin_probabilities(kind, theta, spec):
    """Integral of the oracle's density over the bins of the observables marked `keep`, the
    others integrated over their whole range.  spec[d] = (nbins, k, keep) per observable d
    (m; cos theta_l, cos theta_K, phi).  Returns an array of shape (nbins of kept axes)."""
    ranges = synth.RANGES_1D if kind == M1 else synth.RANGES_4D
    axes = [_axis(ranges[2 * d], ranges[2 * d + 1], nb, k) for d, (nb, k, _) in enumerate(spec)]
    out_shape = [nb for nb, _, keep in spec if keep]
    out = np.zeros(out_shape)
    x0, w0 = axes[0]
    k0 = spec[0][1]
    for b0 in range(spec[0][0]):  # one bin (k0 nodes) of the first observable at a time
        sl = slice(b0 * k0, (b0 + 1) * k0)
        grids = np.meshgrid(x0[sl], *[a[0] for a in axes[1:]], indexing="ij")
        wts = np.ones(grids[0].shape)
        for d, wgrid in enumerate(np.meshgrid(w0[sl], *[a[1] for a in axes[1:]], indexing="ij")):
            wts *= wgrid
        p = oracle.pdf(kind, ranges, theta, [g.ravel() for g in grids]).reshape(grids[0].shape) * wts
        # reduce: sum the k nodes of each bin of a kept axis, the whole of an integrated axis
        for d in range(len(spec) - 1, 0, -1):
            nb, k, keep = spec[d]
            shape = p.shape[:d] + ((nb, k) if keep else (nb * k,)) + p.shape[d + 1:]
            p = p.reshape(shape).sum(axis=d + 1 if keep else d)
        p = p.sum(axis=0)  # the k0 nodes of this bin of the first observable
        if spec[0][2]:
            out[b0] += p
        else:
            out += p
    return out


def chi2_pvalue(counts, probs):
    from scipy.stats import chi2

    n = counts.sum()
    expect = n * probs
    assert expect.min() > 20.0, expect.min()
    x2 = float(np.sum((counts - expect) ** 2 / expect))
    dof = counts.size - 1
    return x2, dof, float(chi2.sf(x2, dof))


PTS = {
    "mass_truth": (M1, synth.TRUTH_1D),
    "mass_alpha_zero": (M1, np.array([5279.6, 20.0, 0.0, 0.3])),
    "mass_alpha_log1p": (M1, np.array([5279.6, 20.0, -5e-5, 0.3])),
    "4d_truth": (M4, synth.TRUTH_4D),
    "4d_alpha_zero": (M4, np.concatenate([synth.TRUTH_4D[:10], [0.0], synth.TRUTH_4D[11:]])),
    "4d_paper_angular": (M4, np.concatenate([synth.TRUTH_4D[:2], [0.6] + [0.0] * 7, synth.TRUTH_4D[10:]])),
}

_samples = {}


def sample(g, name):
    if name not in _samples:
        kind, th = PTS[name]
        ranges = synth.RANGES_1D if kind == M1 else synth.RANGES_4D
        cols = g.nll_generate(kind, ranges, th, N_EVENTS, seed=SEED, stream=list(PTS).index(name))
        _samples.clear()  # keep one 10^7-event sample on the host at a time
        _samples[name] = [c.cpu().numpy() for c in cols]
        del cols
    return _samples[name]


def _hist(x, lo, hi, nb):
    return np.histogram(x, bins=np.linspace(lo, hi, nb + 1))[0].astype(np.float64)


HISTS_1D = ["mass"]
HISTS_4D = ["mass", "ctl", "ctk", "phi", "angular_grid"]
CASES = [(nm, h) for nm in PTS for h in (HISTS_1D if PTS[nm][0] == M1 else HISTS_4D)]


def counts_and_probs(g, name, hist, theta=None):
    kind, th = PTS[name]
    th = th if theta is None else theta
    cols = sample(g, name)
    ma, mb = synth.RANGES_1D
    if hist == "mass":
        counts = _hist(cols[0], ma, mb, 100)
        spec = [(100, 4, True)] + ([(2, 8, False), (2, 8, False), (2, 8, False)] if kind == M4 else [])
        return counts, bin_probabilities(kind, th, spec)
    m_int = (20, 8, False)  # mass integrated: 20 panels of 40 MeV, 8 nodes each
    if hist in ("ctl", "ctk", "phi"):
        d = {"ctl": 1, "ctk": 2, "phi": 3}[hist]
        lo, hi = (-math.pi, math.pi) if d == 3 else (-1.0, 1.0)
        counts = _hist(cols[d], lo, hi, 50)
        spec = [m_int] + [(50, 4, True) if j == d else (2, 8, False) for j in (1, 2, 3)]
        return counts, bin_probabilities(kind, th, spec)
    edges = [np.linspace(-1, 1, 11), np.linspace(-1, 1, 11), np.linspace(-math.pi, math.pi, 11)]
    counts = np.histogramdd(np.stack(cols[1:], axis=1), bins=edges)[0]
    spec = [m_int, (10, 4, True), (10, 4, True), (10, 4, True)]
    return counts, bin_probabilities(kind, th, spec)


@pytest.mark.parametrize("name,hist", CASES)
def test_generated_histogram_matches_the_oracle_density(gpu_lib, name, hist):
    counts, probs = counts_and_probs(gpu_lib, name, hist)
    assert counts.sum() == N_EVENTS  # every event inside the box
    assert abs(probs.sum() - 1.0) < 1e-9, probs.sum()  # the quadrature covers the whole density
    x2, dof, p = chi2_pvalue(counts.ravel(), probs.ravel())
    assert p > 1e-3, (name, hist, x2, dof, p)


def test_planted_shape_error_in_the_hypothesis_fails(gpu_lib):
    th = PTS["4d_truth"][1].copy()
    th[12] += 0.02  # c2 of cos theta_l in the oracle's hypothesis only
    counts, probs = counts_and_probs(gpu_lib, "4d_truth", "ctl", theta=th)
    x2, dof, p = chi2_pvalue(counts, probs)
    assert p < 1e-12, (x2, dof, p)
