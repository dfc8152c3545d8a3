"""Oracle minimiser: damped Newton on a finite-difference Hessian of the oracle's gradient.

TEST INFRASTRUCTURE ONLY (see the package docstring).  It is deliberately a different
algorithm from the library's quasi-Newton minimiser so the two share nothing but the
objective's definition.  The paper minimises with Minuit's Migrad and takes uncertainties
from the inverse Hessian (HESSE), Sec. 2.1 and Sec. 3.1; this is the plain Newton form of
the same minimum and covariance.
"""
import numpy as np

from . import nll_grad


def fd_hessian(kind, ranges, cols, theta, h, w=None, nthreads=1, free=None):
    """Central differences of the analytic gradient, symmetrised; restricted to the parameters
    listed in `free` (all when None)."""
    free = np.arange(len(theta)) if free is None else np.asarray(free)
    n = len(free)
    H = np.zeros((n, n))
    for j, k in enumerate(free):
        tp = np.array(theta, dtype=float)
        tm = np.array(theta, dtype=float)
        tp[k] += h[k]
        tm[k] -= h[k]
        _, gp, _, sp = nll_grad(kind, ranges, cols, tp, w, nthreads)
        _, gm, _, sm = nll_grad(kind, ranges, cols, tm, w, nthreads)
        if sp != 0 or sm != 0:
            raise FloatingPointError("non-positive density inside the Hessian stencil")
        H[:, j] = (gp[free] - gm[free]) / (2.0 * h[k])
    return 0.5 * (H + H.T)


def fit(kind, ranges, cols, theta0, w=None, tol_edm=1e-15, max_iter=60, nthreads=1, h0=None, fixed=None):
    """Minimise the oracle NLL from theta0; parameters with fixed[k] != 0 stay at theta0[k].

    Returns dict(theta, cov, err, nll, edm, n_iter, converged); cov and err are zero in the
    rows and columns of fixed parameters."""
    theta = np.array(theta0, dtype=float)
    n = len(theta)
    free = np.arange(n) if fixed is None else np.flatnonzero(np.asarray(fixed) == 0)
    if h0 is None:
        h = 1e-4 * np.maximum(np.abs(theta), 1e-2)
    else:
        h = np.array(h0, dtype=float)
    nll, g, _, st = nll_grad(kind, ranges, cols, theta, w, nthreads)
    if st != 0:
        raise FloatingPointError("non-positive density at the start point")
    g = g[free]
    edm = np.inf
    cov = None
    it = 0
    for it in range(1, max_iter + 1):
        H = fd_hessian(kind, ranges, cols, theta, h, w, nthreads, free)
        try:
            cov = np.linalg.inv(H)
        except np.linalg.LinAlgError:
            cov = None
        if cov is None or np.any(np.diag(cov) <= 0):
            # not positive definite: fall back to a scaled gradient step
            step = -g * (h[free] * h[free]) * 1e2
        else:
            step = -cov @ g
        edm = 0.5 * float(g @ cov @ g) if cov is not None else np.inf
        if edm < tol_edm:
            break
        lam = 1.0
        while True:
            trial = theta.copy()
            trial[free] += lam * step
            nll_t, g_t, _, st_t = nll_grad(kind, ranges, cols, trial, w, nthreads)
            if st_t == 0 and nll_t <= nll + 1e-12 * abs(nll):
                break
            lam *= 0.5
            if lam < 1e-10:
                raise RuntimeError("oracle Newton line search failed")
        theta, nll, g = trial, nll_t, g_t[free]
        if cov is not None and np.all(np.diag(cov) > 0):
            h[free] = 1e-3 * np.sqrt(np.diag(cov))
    full = None
    if cov is not None:
        full = np.zeros((n, n))
        full[np.ix_(free, free)] = cov
    err = np.sqrt(np.diag(full)) if full is not None else None
    return dict(theta=theta, cov=full, err=err, nll=nll, edm=edm, n_iter=it, converged=bool(edm < tol_edm))
