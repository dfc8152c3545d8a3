"""Oracle: plain CPU FP64 reference for the unbinned NLL of arXiv 2505.12414, its gradient
and its Hessian.

TEST INFRASTRUCTURE ONLY.  Only tests/, ``__graft_entry__.smoke()`` and bench.py's
CPU-baseline leg may import this package.  The product path (the CUDA library and its
Python binding) never imports it, and this package never imports the product path.

The arithmetic lives in ``oracle.c`` (plain C, Kahan summation, paper Sec. 2.1 Eq. 1,
Sec. 2.4.1 Eq. 2, Sec. 2.4.2 Eq. 3); this module only marshals arguments via ctypes.
"""
import ctypes
import os

import numpy as np

from . import build as _build

MASS1D = 1
KSTAR4D = 2
NPAR = {MASS1D: 4, KSTAR4D: 18}
NDIM = {MASS1D: 1, KSTAR4D: 4}

OK = 0
ERR_NONPOSITIVE = 4

_lib = None


def lib():
    """Load (building first if needed) the oracle shared library."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        dpp = ctypes.POINTER(dp)
        L.oracle_nll_grad.argtypes = [ctypes.c_int, dp, dpp, dp, ctypes.c_int64, dp, ctypes.c_int, dp, dp, dp]
        L.oracle_nll_grad.restype = ctypes.c_int
        L.oracle_pdf.argtypes = [ctypes.c_int, dp, dp, dpp, ctypes.c_int64, dp]
        L.oracle_pdf.restype = ctypes.c_int
        L.oracle_dlogpdf.argtypes = [ctypes.c_int, dp, dp, dpp, ctypes.c_int64, dp]
        L.oracle_dlogpdf.restype = ctypes.c_int
        L.oracle_angular_terms.argtypes = [dp, dp, dp, ctypes.c_int64, dp]
        L.oracle_angular_terms.restype = None
        L.oracle_mass_norms.argtypes = [ctypes.c_double] * 5 + [dp]
        L.oracle_mass_norms.restype = None
        L.oracle_nll_hess.argtypes = [ctypes.c_int, dp, dpp, dp, ctypes.c_int64, dp, ctypes.c_int, dp, dp, dp, dp,
                                      dp]
        L.oracle_nll_hess.restype = ctypes.c_int
        L.oracle_mass_norms2.argtypes = [ctypes.c_double] * 5 + [dp]
        L.oracle_mass_norms2.restype = None
        L.oracle_d2logpdf.argtypes = [ctypes.c_int, dp, dp, dpp, ctypes.c_int64, dp]
        L.oracle_d2logpdf.restype = ctypes.c_int
        _lib = L
    return _lib


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _cols(cols):
    arrs = [_f64(c) for c in cols]
    ptrs = (ctypes.POINTER(ctypes.c_double) * len(arrs))(*[_dptr(a) for a in arrs])
    return arrs, ptrs


def nll_grad(kind, ranges, cols, theta, w=None, nthreads=1, grad=True):
    """Return (nll, grad, scale, status).  grad/scale are None when grad=False.

    ``scale[k]`` is sum_i |w_i d ln P_i / d theta_k|, the size of the terms that make up
    gradient component k (used by the tolerance rule for cancelling sums)."""
    L = lib()
    arrs, ptrs = _cols(cols)
    n = len(arrs[0])
    rng = _f64(ranges)
    th = _f64(theta)
    wa = _f64(w) if w is not None else None
    out = np.zeros(1)
    g = np.zeros(NPAR[kind]) if grad else None
    s = np.zeros(NPAR[kind]) if grad else None
    st = L.oracle_nll_grad(
        kind, _dptr(rng), ptrs, _dptr(wa) if wa is not None else None, n, _dptr(th), int(nthreads),
        _dptr(out), _dptr(g) if grad else None, _dptr(s) if grad else None,
    )
    return float(out[0]), g, s, st


def pdf(kind, ranges, theta, cols):
    """Per-event normalised density P_i."""
    L = lib()
    arrs, ptrs = _cols(cols)
    out = np.zeros(len(arrs[0]))
    st = L.oracle_pdf(kind, _dptr(_f64(ranges)), _dptr(_f64(theta)), ptrs, len(arrs[0]), _dptr(out))
    assert st == OK
    return out


def dlogpdf(kind, ranges, theta, cols):
    """Per-event d ln P_i / d theta, shape (n, npar)."""
    L = lib()
    arrs, ptrs = _cols(cols)
    n = len(arrs[0])
    out = np.zeros((n, NPAR[kind]))
    st = L.oracle_dlogpdf(kind, _dptr(_f64(ranges)), _dptr(_f64(theta)), ptrs, n, _dptr(out))
    assert st == OK
    return out


def angular_terms(ctl, ctk, phi):
    """The eleven terms f_i of paper Eq. 3 per event (9/(32 pi) included), shape (n, 11)."""
    L = lib()
    a, b, c = _f64(ctl), _f64(ctk), _f64(phi)
    out = np.zeros((len(a), 11))
    L.oracle_angular_terms(_dptr(a), _dptr(b), _dptr(c), len(a), _dptr(out))
    return out


def mass_norms(ma, mb, mu, sigma, alpha):
    """dict with N1, dlnN1_dmu, dlnN1_dsigma, N2, dlnN2_dalpha (paper Eq. 2)."""
    out = np.zeros(5)
    lib().oracle_mass_norms(ma, mb, mu, sigma, alpha, _dptr(out))
    return dict(N1=out[0], dlnN1_dmu=out[1], dlnN1_dsigma=out[2], N2=out[3], dlnN2_dalpha=out[4])


def nll_hess(kind, ranges, cols, theta, w=None, nthreads=1):
    """Return dict(nll, grad, hess, w2, hscale, status).

    ``hess`` is the Hessian of the NLL, ``w2`` = sum_i w_i^2 s_i s_i^T with s_i = d ln P_i/dtheta
    (the middle of the weighted-fit sandwich covariance), ``hscale[a, b]`` = sum_i
    |w_i| (|P_ab/P| + |P_a P_b/P^2|), the size of the two terms whose difference makes up
    each event's share of hess[a, b] (it bounds this plain form's rounding error)."""
    L = lib()
    arrs, ptrs = _cols(cols)
    n = len(arrs[0])
    npar = NPAR[kind]
    wa = _f64(w) if w is not None else None
    out = np.zeros(1)
    g = np.zeros(npar)
    h = np.zeros((npar, npar))
    q = np.zeros((npar, npar))
    hs = np.zeros((npar, npar))
    st = L.oracle_nll_hess(kind, _dptr(_f64(ranges)), ptrs, _dptr(wa) if wa is not None else None, n,
                           _dptr(_f64(theta)), int(nthreads), _dptr(out), _dptr(g), _dptr(h), _dptr(q), _dptr(hs))
    return dict(nll=float(out[0]), grad=g, hess=h, w2=q, hscale=hs, status=st)


def mass_norms2(ma, mb, mu, sigma, alpha):
    """dict with the second derivatives d2lnN1_mumu, d2lnN1_musigma, d2lnN1_sigmasigma, d2lnN2_alpha."""
    out = np.zeros(4)
    lib().oracle_mass_norms2(ma, mb, mu, sigma, alpha, _dptr(out))
    return dict(d2lnN1_mumu=out[0], d2lnN1_musigma=out[1], d2lnN1_sigmasigma=out[2], d2lnN2_alpha=out[3])


def d2logpdf(kind, ranges, theta, cols):
    """Per-event d^2 ln P_i / dtheta dtheta^T, shape (n, npar, npar)."""
    L = lib()
    arrs, ptrs = _cols(cols)
    n = len(arrs[0])
    npar = NPAR[kind]
    out = np.zeros((n, npar, npar))
    st = L.oracle_d2logpdf(kind, _dptr(_f64(ranges)), _dptr(_f64(theta)), ptrs, n, _dptr(out))
    assert st == OK
    return out
