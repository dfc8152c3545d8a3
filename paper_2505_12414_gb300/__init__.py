"""Python binding of libgbnll: the GB300 unbinned-NLL hot path (arXiv 2505.12414).

Argument marshalling only.  Every evaluation runs in the CUDA library's kernels; there is
no CPU fallback: if the library is not built, or no CUDA device is present, the calls
raise.  Function names match the C ABI in include/gbnll.h.

Inputs may be numpy arrays (host memory, copied by the library) or CUDA torch tensors
(device memory on the model's device, copied device-to-device).  Streams: pass
``torch.cuda.current_stream().cuda_stream`` (0, CUDA's default stream, is the default).
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libgbnll.so")

NLL_OK = 0
NLL_ERR_ARG = 1
NLL_ERR_CUDA = 2
NLL_ERR_OOM = 3
NLL_ERR_NONPOSITIVE_PDF = 4
NLL_ERR_NOT_CONVERGED = 5
NLL_ERR_TIMEOUT = 6
NLL_ERR_STATE = 7

NLL_MODEL_MASS1D = 1
NLL_MODEL_KSTARMUMU4D = 2

NLL_VARIANT_AUTO = 0
NLL_VARIANT_PRECOMPUTE = 1
NLL_VARIANT_DIRECT = 2

FIT_MAXPAR = 32

_lib = None


class NLLError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("gbnll status %d: %s" % (status, message))
        self.status = status


class fit_options(ctypes.Structure):
    _fields_ = [("tol_edm", ctypes.c_double), ("max_iter", ctypes.c_int), ("strategy", ctypes.c_int),
                ("hessian", ctypes.c_int)]


class fit_result(ctypes.Structure):
    _fields_ = [("theta", ctypes.c_double * FIT_MAXPAR), ("err", ctypes.c_double * FIT_MAXPAR),
                ("cov", ctypes.c_double * (FIT_MAXPAR * FIT_MAXPAR)), ("nll", ctypes.c_double),
                ("edm", ctypes.c_double), ("n_eval", ctypes.c_int), ("n_iter", ctypes.c_int),
                ("status", ctypes.c_int)]


_FIT_RESULT_DTYPE = np.dtype(fit_result)  # the same layout as a numpy record


def _results_of(res, n, **extra):
    """Per-fit arrays from a record array of fit_result (n parameters)."""
    out = dict(theta=res["theta"][:, :n].copy(), err=res["err"][:, :n].copy(), nll=res["nll"].copy(),
               edm=res["edm"].copy(), n_eval=res["n_eval"].copy(), n_iter=res["n_iter"].copy(),
               status=res["status"].copy(), cov=res["cov"][:, : n * n].reshape(-1, n, n).copy())
    out.update(extra)
    return out


FIT_FCN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                           ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double))

_DP = ctypes.POINTER(ctypes.c_double)


def load(path=None):
    """Load libgbnll.so (built by __graft_entry__.build()); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError("libgbnll.so is not built (%s); run __graft_entry__.build()" % p)
    L = ctypes.CDLL(p)
    vp = ctypes.c_void_p
    L.nll_create_model.argtypes = [ctypes.c_int, _DP, ctypes.c_int, ctypes.c_size_t, ctypes.POINTER(vp)]
    L.nll_load_events.argtypes = [vp, ctypes.POINTER(vp), vp, ctypes.c_int64, ctypes.c_int, ctypes.c_int]
    L.nll_eval.argtypes = [vp, _DP, ctypes.c_int, _DP]
    L.nll_eval_grad.argtypes = [vp, _DP, ctypes.c_int, _DP, _DP]
    L.nll_eval_hess.argtypes = [vp, _DP, ctypes.c_int, _DP, _DP, _DP, _DP]
    L.nll_hess_num_slots.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
    L.fit_minimise.argtypes = [vp, _DP, _DP, _DP, _DP, ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                               ctypes.POINTER(fit_options), ctypes.POINTER(fit_result)]
    L.fit_minimise_fcn.argtypes = [FIT_FCN, vp, _DP, _DP, _DP, _DP, ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                   ctypes.POINTER(fit_options), ctypes.POINTER(fit_result)]
    L.nll_num_params.argtypes = [vp]
    L.nll_param_name.argtypes = [vp, ctypes.c_int]
    L.nll_param_name.restype = ctypes.c_char_p
    L.nll_last_error.argtypes = [vp]
    L.nll_last_error.restype = ctypes.c_char_p
    L.nll_destroy.argtypes = [vp]
    L.nll_destroy.restype = None
    L.nll_set_launch.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    L.nll_get_launch.argtypes = [vp] + [ctypes.POINTER(ctypes.c_int)] * 4
    L.nll_autotune.argtypes = [vp]
    L.nll_set_profiling.argtypes = [vp, ctypes.c_int]
    L.nll_last_kernel_ms.argtypes = [vp, _DP]
    L.nll_precomputed_basis.argtypes = [vp, _DP]
    L.nll_calibrate_fp64.argtypes = [ctypes.c_int, _DP]
    L.nll_diag_math.argtypes = [ctypes.c_int, ctypes.c_int, _DP, _DP, ctypes.c_int64]
    L.nll_batch_create.argtypes = [ctypes.c_int, _DP, ctypes.c_int, ctypes.c_size_t, ctypes.POINTER(vp)]
    L.nll_batch_load.argtypes = [vp, ctypes.POINTER(ctypes.c_int64), ctypes.c_int, ctypes.POINTER(vp), vp, ctypes.c_int]
    L.nll_batch_eval_grad.argtypes = [vp, _DP, _DP, _DP, ctypes.POINTER(ctypes.c_int)]
    L.nll_batch_eval_hess.argtypes = [vp, _DP, ctypes.c_int, _DP, _DP, _DP, _DP, ctypes.POINTER(ctypes.c_int)]
    L.nll_batch_fit.argtypes = [vp, _DP, ctypes.c_int, _DP, _DP, _DP, ctypes.POINTER(ctypes.c_int),
                                ctypes.POINTER(fit_options), ctypes.POINTER(fit_result), ctypes.POINTER(ctypes.c_int)]
    _IPp = ctypes.POINTER(ctypes.c_int)
    L.nll_batch_fit_arrays.argtypes = [vp, _DP, ctypes.c_int, _DP, _DP, _DP, _IPp, ctypes.POINTER(fit_options),
                                       _DP, _DP, _DP, _DP, _DP, _IPp, _IPp, _IPp, _IPp]
    L.nll_batch_set_schedule.argtypes = [vp, ctypes.c_int, ctypes.c_int]
    L.nll_batch_get_schedule.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    L.nll_batch_autotune.argtypes = [vp]
    L.nll_batch_num_toys.argtypes = [vp]
    L.nll_batch_last_error.argtypes = [vp]
    L.nll_batch_last_error.restype = ctypes.c_char_p
    L.nll_batch_destroy.argtypes = [vp]
    L.nll_batch_destroy.restype = None
    L.nll_server_create.argtypes = [ctypes.c_int, _DP, ctypes.c_int, ctypes.c_int, ctypes.c_int64, ctypes.c_int,
                                    _DP, _DP, _DP, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(fit_options),
                                    ctypes.POINTER(vp)]
    L.nll_server_submit.argtypes = [vp, ctypes.POINTER(vp), vp, ctypes.c_int64, _DP, ctypes.POINTER(ctypes.c_int64)]
    L.nll_server_step.argtypes = [vp, ctypes.c_int]
    L.nll_server_sync.argtypes = [vp]
    L.nll_server_poll.argtypes = [vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(fit_result), ctypes.c_int,
                                  ctypes.POINTER(ctypes.c_int)]
    L.nll_server_status.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                    ctypes.POINTER(ctypes.c_int64)]
    L.nll_server_progress.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    L.nll_server_cancel.argtypes = [vp, ctypes.c_int64]
    L.nll_server_last_error.argtypes = [vp]
    L.nll_server_last_error.restype = ctypes.c_char_p
    L.nll_server_destroy.argtypes = [vp]
    L.nll_server_destroy.restype = None
    L.nll_batch_generate.argtypes = [vp, _DP, ctypes.POINTER(ctypes.c_int64), ctypes.c_int, ctypes.c_uint64,
                                     ctypes.c_int]
    L.nll_generate.argtypes = [ctypes.c_int, _DP, _DP, ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint64,
                               ctypes.c_int, ctypes.c_size_t, ctypes.POINTER(vp)]
    L.nll_diag_uniforms.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64, ctypes.c_int, _DP]
    L.nll_eval_grad_4d_noalloc.argtypes = [_DP, ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p, ctypes.c_int64,
                                           _DP, ctypes.c_int, ctypes.c_int, ctypes.c_size_t, _DP, _DP]
    _lib = L
    return L


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a):
    return a.ctypes.data_as(_DP)


def _is_cuda_tensor(x):
    return hasattr(x, "is_cuda") and hasattr(x, "data_ptr") and bool(x.is_cuda)


def _check(model, st):
    if st != NLL_OK:
        msg = load().nll_last_error(model).decode() if model else ""
        raise NLLError(st, msg)


def _err(model):
    return load().nll_last_error(model).decode()


# ------------------------------------------------------------------------------------
# functions with the C ABI's names
# ------------------------------------------------------------------------------------
def nll_create_model(kind, obs_ranges, device=0, stream=0):
    """Create a model; returns an opaque handle (int)."""
    L = load()
    r = _f64(obs_ranges)
    h = ctypes.c_void_p()
    st = L.nll_create_model(int(kind), _p(r), int(device), int(stream or 0), ctypes.byref(h))
    if st != NLL_OK:
        raise NLLError(st, "nll_create_model failed")
    return h.value


def _in_place_ptr(x, what):
    """Address of a float64 contiguous array or tensor, without a copy (in-place loads)."""
    if hasattr(x, "data_ptr"):
        import torch

        if x.dtype != torch.float64 or not x.is_contiguous():
            raise ValueError("%s: in-place loads need contiguous float64 tensors" % what)
        return x.data_ptr(), int(x.numel())
    a = np.asarray(x)
    if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
        raise ValueError("%s: in-place loads need contiguous float64 arrays" % what)
    return a.ctypes.data, len(a)


def nll_load_events(model, columns, weights=None, precompute=True, in_place=False):
    """Copy events (numpy arrays on the host, or CUDA tensors) into the model.

    With in_place=True nothing is copied: every evaluation reads these buffers (pinned host
    memory, device memory, or on a coherent CPU-GPU system any host memory; float64,
    contiguous, 16-byte aligned).  Returns the objects the model reads; keep them alive
    and unchanged until the next load (Model.load keeps them)."""
    L = load()
    cols = list(columns)
    if in_place:
        ptrs, ns = zip(*[_in_place_ptr(c, "column %d" % i) for i, c in enumerate(cols)])
        if len(set(ns)) != 1:
            raise ValueError("columns differ in length")
        wp = None
        if weights is not None:
            wp, nw = _in_place_ptr(weights, "weights")
            if nw != ns[0]:
                raise ValueError("weights differ in length from the columns")
        arr = (ctypes.c_void_p * len(ptrs))(*ptrs)
        st = L.nll_load_events(model, arr, wp, ns[0], 2, 0)
        _check(model, st)
        return cols + ([weights] if weights is not None else [])
    on_device = _is_cuda_tensor(cols[0])
    keep = []
    if on_device:
        import torch

        cols = [c.to(torch.float64).contiguous() for c in cols]
        keep.extend(cols)
        ptrs = [c.data_ptr() for c in cols]
        n = int(cols[0].numel())
        wp = None
        if weights is not None:
            w = weights.to(torch.float64).contiguous()
            keep.append(w)
            wp = w.data_ptr()
    else:
        cols = [_f64(c) for c in cols]
        keep.extend(cols)
        ptrs = [c.ctypes.data for c in cols]
        n = len(cols[0])
        wp = None
        if weights is not None:
            w = _f64(weights)
            keep.append(w)
            wp = w.ctypes.data
    arr = (ctypes.c_void_p * len(ptrs))(*ptrs)
    st = L.nll_load_events(model, arr, wp, n, 1 if on_device else 0, 1 if precompute else 0)
    _check(model, st)


def nll_eval(model, theta, check=True):
    """NLL at theta.  With check=False returns (nll, status) instead of raising."""
    L = load()
    th = _f64(theta)
    out = ctypes.c_double()
    st = L.nll_eval(model, _p(th), len(th), ctypes.byref(out))
    if not check:
        return out.value, st
    _check(model, st)
    return out.value


def nll_eval_grad(model, theta, check=True):
    """(NLL, gradient ndarray) at theta.  With check=False also returns the status."""
    L = load()
    th = _f64(theta)
    out = ctypes.c_double()
    g = np.zeros(len(th))
    st = L.nll_eval_grad(model, _p(th), len(th), ctypes.byref(out), _p(g))
    if not check:
        return out.value, g, st
    _check(model, st)
    return out.value, g


def nll_eval_hess(model, theta, w2=False, check=True):
    """(NLL, gradient, Hessian[, W]) at theta from one device pass.  W = sum w^2 s s^T is
    returned when w2 is true (the middle of the weighted-fit covariance H^-1 W H^-1).
    With check=False the status is appended instead of raising."""
    L = load()
    th = _f64(theta)
    n = len(th)
    out = ctypes.c_double()
    g = np.zeros(n)
    H = np.zeros((n, n))
    W = np.zeros((n, n)) if w2 else None
    st = L.nll_eval_hess(model, _p(th), n, ctypes.byref(out), _p(g), _p(H), _p(W) if w2 else None)
    res = (out.value, g, H) + ((W,) if w2 else ())
    if not check:
        return res + (st,)
    _check(model, st)
    return res


def nll_hess_num_slots(kind, weighted=False, w2=False):
    """Per-event FMA slots of the Hessian pass (its FP64 cost per event, besides staging)."""
    return load().nll_hess_num_slots(int(kind), 1 if weighted else 0, 1 if w2 else 0)


def _fit_args(theta0, lo, hi, step, fixed):
    th = _f64(theta0)
    n = len(th)
    lo = _f64(lo) if lo is not None else np.zeros(n)
    hi = _f64(hi) if hi is not None else np.zeros(n)
    step = _f64(step) if step is not None else np.maximum(1e-3 * np.abs(th), 1e-3)
    fx = np.ascontiguousarray(fixed, dtype=np.int32) if fixed is not None else np.zeros(n, dtype=np.int32)
    return th, lo, hi, step, fx


def _result_dict(res, n):
    # theta, err and cov lead the record as one run of doubles: one view, three slices
    a = np.frombuffer(res, dtype=np.float64, count=2 * FIT_MAXPAR + FIT_MAXPAR * FIT_MAXPAR)
    return dict(theta=a[:n].copy(), err=a[FIT_MAXPAR:FIT_MAXPAR + n].copy(),
                cov=a[2 * FIT_MAXPAR:2 * FIT_MAXPAR + n * n].reshape(n, n).copy(), nll=res.nll, edm=res.edm,
                n_eval=res.n_eval, n_iter=res.n_iter, status=res.status)


def fit_minimise(model, theta0, lo=None, hi=None, step=None, fixed=None, tol_edm=1e-8, max_iter=500,
                 strategy=1, hessian=1):
    """Minimise the model's NLL on the GPU; returns a dict (theta, err, cov, nll, edm, ...)."""
    L = load()
    th, lo, hi, step, fx = _fit_args(theta0, lo, hi, step, fixed)
    opt = fit_options(tol_edm, max_iter, strategy, hessian)
    res = fit_result()
    L.fit_minimise(model, _p(th), _p(lo), _p(hi), _p(step), fx.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                   len(th), ctypes.byref(opt), ctypes.byref(res))
    return _result_dict(res, len(th))


def fit_minimise_fcn(fcn, theta0, lo=None, hi=None, step=None, fixed=None, tol_edm=1e-8, max_iter=500,
                     strategy=1, hessian=1):
    """The library's minimiser on a Python objective fcn(theta) -> (f, grad)."""
    L = load()
    th, lo, hi, step, fx = _fit_args(theta0, lo, hi, step, fixed)
    n = len(th)

    def cb(user, tp, fp, gp):
        try:
            t = np.ctypeslib.as_array(tp, shape=(n,)).copy()
            f, g = fcn(t)
            fp[0] = float(f)
            for k in range(n):
                gp[k] = float(g[k])
            return 0
        except Exception:
            return 1

    cfun = FIT_FCN(cb)
    opt = fit_options(tol_edm, max_iter, strategy, hessian)
    res = fit_result()
    L.fit_minimise_fcn(cfun, None, _p(th), _p(lo), _p(hi), _p(step),
                       fx.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), n, ctypes.byref(opt), ctypes.byref(res))
    return _result_dict(res, n)


def nll_num_params(model):
    return load().nll_num_params(model)


def nll_param_name(model, i):
    return load().nll_param_name(model, int(i)).decode()


def nll_last_error(model):
    return _err(model)


def nll_destroy(model):
    if model:
        load().nll_destroy(model)


def nll_set_launch(model, blocks_per_sm=0, threads_per_block=0, variant=0):
    _check(model, load().nll_set_launch(model, int(blocks_per_sm), int(threads_per_block), int(variant)))


def nll_get_launch(model):
    v = [ctypes.c_int() for _ in range(4)]
    _check(model, load().nll_get_launch(model, *[ctypes.byref(x) for x in v]))
    return dict(blocks_per_sm=v[0].value, threads=v[1].value, variant=v[2].value, sm_count=v[3].value)


def nll_autotune(model):
    _check(model, load().nll_autotune(model))


def nll_set_profiling(model, on=True):
    _check(model, load().nll_set_profiling(model, 1 if on else 0))


def nll_last_kernel_ms(model):
    out = ctypes.c_double()
    _check(model, load().nll_last_kernel_ms(model, ctypes.byref(out)))
    return out.value


def nll_precomputed_basis(model, n_events):
    out = np.zeros((int(n_events), 13))
    _check(model, load().nll_precomputed_basis(model, _p(out)))
    return out


def nll_calibrate_fp64(device=0):
    """FP64 throughput of the device: dict of operations/s (see include/gbnll.h)."""
    r = np.zeros(6)
    st = load().nll_calibrate_fp64(int(device), _p(r))
    if st != NLL_OK:
        raise NLLError(st, "nll_calibrate_fp64 failed")
    keys = ["dfma", "cuda_exp", "cuda_div_plus_dadd", "cuda_log_plus_dadd", "lib_exp", "lib_rcp_plus_dadd"]
    return dict(zip(keys, r.tolist()))


def nll_diag_math(fn, x, device=0):
    """Evaluate the library's device exp (fn=0), reciprocal (fn=1), sin (fn=2), cos (fn=3), log
    (fn=4), the hardware reciprocal approximation alone (fn=5) or with one Newton step (fn=6) on
    host array x (see nll_diag_math in the C header for the argument conventions)."""
    xa = _f64(x)
    y = np.zeros_like(xa)
    st = load().nll_diag_math(int(device), int(fn), _p(xa), _p(y), len(xa))
    if st != NLL_OK:
        raise NLLError(st, "nll_diag_math failed")
    return y


NLL_NOALLOC_MAX_BLOCKS = 1024


def nll_generate(kind, obs_ranges, theta, n_events, seed, stream=0, device=0):
    """Generate n_events events on the device; returns a list of CUDA torch tensors."""
    import torch

    ndim = 1 if kind == NLL_MODEL_MASS1D else 4
    cols = [torch.empty(max(int(n_events), 1), dtype=torch.float64, device="cuda:%d" % device) for _ in range(ndim)]
    ptrs = (ctypes.c_void_p * ndim)(*[c.data_ptr() for c in cols])
    torch.cuda.synchronize(device)
    st = load().nll_generate(int(kind), _p(_f64(obs_ranges)), _p(_f64(theta)), int(n_events),
                             int(seed) & ((1 << 64) - 1), int(stream), int(device), 0, ptrs)
    if st != NLL_OK:
        raise NLLError(st, "nll_generate failed")
    return [c[: int(n_events)] for c in cols]


def nll_diag_uniforms(seed, stream, n, device=0):
    out = np.zeros(int(n))
    st = load().nll_diag_uniforms(int(seed) & ((1 << 64) - 1), int(stream), int(n), int(device), _p(out))
    if st != NLL_OK:
        raise NLLError(st, "nll_diag_uniforms failed")
    return out


def _noalloc_stream(stream, dev_columns):
    """The stream to run on: the given one, else torch's current stream when the columns are
    CUDA tensors (so that work queued on it, such as the columns' own writes, comes first),
    else CUDA's default stream."""
    if stream:
        return int(stream)
    if dev_columns and _is_cuda_tensor(dev_columns[0]):
        import torch

        return int(torch.cuda.current_stream(dev_columns[0].device).cuda_stream)
    return 0


def nll_eval_grad_4d_noalloc(obs_ranges, dev_columns, theta, dev_weights=None, blocks=0, stream=0, check=True,
                             n_events=None):
    """4D NLL and gradient on caller-owned device buffers, without any device allocation by the
    library.  dev_columns are four CUDA tensors (the event count is their length unless
    n_events says otherwise) or four raw device pointers (then n_events is required).  Returns
    (nll, grad) or, with check=False, (nll, grad, status)."""
    L = load()
    r = _f64(obs_ranges)
    if len(dev_columns) != 4:
        raise ValueError("four device columns (m, cos theta_l, cos theta_K, phi) expected")
    tensors = all(_is_cuda_tensor(c) for c in dev_columns)
    if n_events is None:
        if not tensors:
            raise ValueError("n_events is required when raw device pointers are passed")
        n_events = int(dev_columns[0].numel())
    if tensors:
        for c in dev_columns:
            if c.dtype != _torch_f64() or not c.is_contiguous() or c.numel() < n_events:
                raise ValueError("columns must be contiguous float64 CUDA tensors of at least n_events elements")
    ptrs = [c.data_ptr() if hasattr(c, "data_ptr") else int(c) for c in dev_columns]
    arr = (ctypes.c_void_p * 4)(*ptrs)
    return _noalloc_call(L, r, arr, dev_weights, n_events, theta, blocks, _noalloc_stream(stream, dev_columns), check)


def _torch_f64():
    import torch

    return torch.float64


def _noalloc_call(L, r, arr, dev_weights, n, theta, blocks, stream, check):
    th = _f64(theta)
    wp = None
    if dev_weights is not None:
        wp = dev_weights.data_ptr() if hasattr(dev_weights, "data_ptr") else int(dev_weights)
    out = ctypes.c_double()
    g = np.zeros(len(th))
    st = L.nll_eval_grad_4d_noalloc(_p(r), arr, wp, int(n), _p(th), len(th), int(blocks), int(stream or 0),
                                    ctypes.byref(out), _p(g))
    if not check:
        return out.value, g, st
    if st != NLL_OK:
        raise NLLError(st, "nll_eval_grad_4d_noalloc failed")
    return out.value, g


def nll_eval_grad_4d_noalloc_n(obs_ranges, dev_columns, n_events, theta, dev_weights=None, blocks=0, stream=0,
                               check=True):
    """As nll_eval_grad_4d_noalloc with an explicit event count (buffers may be longer)."""
    return nll_eval_grad_4d_noalloc(obs_ranges, dev_columns, theta, dev_weights=dev_weights, blocks=blocks,
                                    stream=stream, check=check, n_events=n_events)


class Model:
    """Owning wrapper around a model handle."""

    def __init__(self, kind, obs_ranges, device=0, stream=0):
        self.kind = kind
        self.handle = nll_create_model(kind, obs_ranges, device, stream)
        n = nll_num_params(self.handle)
        # preallocated argument buffers for the repeated-evaluation path
        self._n = n
        self._th = np.zeros(n)
        self._g = np.zeros(n)
        self._out = ctypes.c_double()
        self._thp = self._th.ctypes.data_as(_DP)
        self._gp = self._g.ctypes.data_as(_DP)
        self._outp = ctypes.byref(self._out)

    def load(self, columns, weights=None, precompute=True, in_place=False):
        kept = nll_load_events(self.handle, columns, weights, precompute, in_place)
        self._in_place_keep = kept if in_place else None  # the buffers the model reads
        return self

    def eval(self, theta):
        self._th[:] = theta
        st = load().nll_eval(self.handle, self._thp, self._n, self._outp)
        _check(self.handle, st)
        return self._out.value

    def eval_grad(self, theta):
        """(NLL, gradient); the gradient array is a fresh copy."""
        self._th[:] = theta
        st = load().nll_eval_grad(self.handle, self._thp, self._n, self._outp, self._gp)
        _check(self.handle, st)
        return self._out.value, self._g.copy()

    def eval_hess(self, theta, w2=False):
        """(NLL, gradient, Hessian[, W]); see nll_eval_hess."""
        return nll_eval_hess(self.handle, theta, w2)

    def fit(self, theta0, **kw):
        return fit_minimise(self.handle, theta0, **kw)

    @property
    def num_params(self):
        return nll_num_params(self.handle)

    def param_names(self):
        return [nll_param_name(self.handle, i) for i in range(self.num_params)]

    def close(self):
        if self.handle:
            nll_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------------------------
# batched pseudo-experiments
# ------------------------------------------------------------------------------------
def _bcheck(handle, st):
    if st != NLL_OK:
        raise NLLError(st, load().nll_batch_last_error(handle).decode())


class Batch:
    """Many toys of one model (CSR samples); batched evaluation and device-resident fits."""

    def __init__(self, kind, obs_ranges, device=0, stream=0):
        L = load()
        r = _f64(obs_ranges)
        h = ctypes.c_void_p()
        st = L.nll_batch_create(int(kind), _p(r), int(device), int(stream or 0), ctypes.byref(h))
        if st != NLL_OK:
            raise NLLError(st, "nll_batch_create failed")
        self.handle = h.value
        self.kind = kind
        self.npar = 4 if kind == NLL_MODEL_MASS1D else 18
        self.n_toys = 0

    def load(self, offsets, columns, weights=None, precompute=True):
        off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
        cols = [_f64(c) for c in columns]
        ptrs = (ctypes.c_void_p * len(cols))(*[c.ctypes.data for c in cols])
        w = _f64(weights) if weights is not None else None
        st = load().nll_batch_load(self.handle, off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), len(off) - 1,
                                   ptrs, w.ctypes.data if w is not None else None, 1 if precompute else 0)
        _bcheck(self.handle, st)
        self.n_toys = len(off) - 1
        return self

    def generate(self, theta, counts, seed, precompute=True):
        """Generate the toys on the device (counts[t] events for toy t) instead of loading them."""
        c = np.ascontiguousarray(np.asarray(counts, dtype=np.int64))
        th = _f64(theta)
        st = load().nll_batch_generate(self.handle, _p(th), c.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), len(c),
                                       int(seed) & ((1 << 64) - 1), 1 if precompute else 0)
        _bcheck(self.handle, st)
        self.n_toys = len(c)
        return self

    def eval_grad(self, thetas):
        """(nll[n], grad[n, npar], status[n]) at one parameter point per toy."""
        th = _f64(np.broadcast_to(np.asarray(thetas, dtype=np.float64), (self.n_toys, self.npar)))
        nll = np.zeros(self.n_toys)
        g = np.zeros((self.n_toys, self.npar))
        stv = np.zeros(self.n_toys, dtype=np.int32)
        load().nll_batch_eval_grad(self.handle, _p(th), _p(nll), _p(g), stv.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
        return nll, g, stv

    def eval_hess(self, thetas, w2=False):
        """Per-toy (nll [n], grad [n, np], H [n, np, np][, W], status [n]) in one device pass;
        thetas is [n, np] or one shared [np] point."""
        t = np.asarray(thetas, dtype=np.float64)
        shared = 1 if t.ndim == 1 else 0
        th = _f64(t)
        n, npar = self.n_toys, self.npar
        nll = np.zeros(max(n, 1))
        g = np.zeros((max(n, 1), npar))
        H = np.zeros((max(n, 1), npar, npar))
        W = np.zeros((max(n, 1), npar, npar)) if w2 else None
        st = np.zeros(max(n, 1), dtype=np.int32)
        r = load().nll_batch_eval_hess(self.handle, _p(th), shared, _p(nll), _p(g), _p(H), _p(W) if w2 else None,
                                       st.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
        if r not in (NLL_OK, NLL_ERR_NONPOSITIVE_PDF, NLL_ERR_ARG):
            _bcheck(self.handle, r)
        out = (nll[:n], g[:n], H[:n]) + ((W[:n],) if w2 else ()) + (st[:n],)
        return out

    def fit(self, theta0, lo=None, hi=None, step=None, fixed=None, tol_edm=1e-8, max_iter=500, strategy=1,
            hessian=1):
        """Fit every toy on the device; returns a dict of per-toy arrays and 'steps'."""
        t0 = np.asarray(theta0, dtype=np.float64)
        shared = 1 if t0.ndim == 1 else 0
        th, lo, hi, step, fx = _fit_args(t0.reshape(-1)[: self.npar] if shared else t0[0], lo, hi, step, fixed)
        th = _f64(t0)
        opt = fit_options(tol_edm, max_iter, strategy, hessian)
        n, npar = max(self.n_toys, 1), self.npar
        ip = ctypes.POINTER(ctypes.c_int)
        out = dict(theta=np.empty((n, npar)), err=np.empty((n, npar)), nll=np.empty(n), edm=np.empty(n),
                   n_eval=np.empty(n, dtype=np.int32), n_iter=np.empty(n, dtype=np.int32),
                   status=np.empty(n, dtype=np.int32), cov=np.empty((n, npar, npar)))
        steps = ctypes.c_int()
        st = load().nll_batch_fit_arrays(self.handle, _p(th), shared, _p(lo), _p(hi), _p(step), fx.ctypes.data_as(ip),
                                         ctypes.byref(opt), _p(out["theta"]), _p(out["err"]), _p(out["cov"]),
                                         _p(out["nll"]), _p(out["edm"]), out["n_eval"].ctypes.data_as(ip),
                                         out["n_iter"].ctypes.data_as(ip), out["status"].ctypes.data_as(ip),
                                         ctypes.byref(steps))
        if st not in (NLL_OK, NLL_ERR_NOT_CONVERGED):
            _bcheck(self.handle, st)
        res = {k: v[: self.n_toys] for k, v in out.items()}
        res["steps"] = steps.value
        return res

    def set_schedule(self, tile_events=0, blocks_per_sm=0):
        _bcheck(self.handle, load().nll_batch_set_schedule(self.handle, int(tile_events), int(blocks_per_sm)))

    def get_schedule(self):
        a, b = ctypes.c_int(), ctypes.c_int()
        _bcheck(self.handle, load().nll_batch_get_schedule(self.handle, ctypes.byref(a), ctypes.byref(b)))
        return dict(tile_events=a.value, blocks_per_sm=b.value)

    def autotune(self):
        _bcheck(self.handle, load().nll_batch_autotune(self.handle))

    def close(self):
        if getattr(self, "handle", None):
            load().nll_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------------------------
# serving
# ------------------------------------------------------------------------------------
def _scheck(handle, st):
    if st != NLL_OK:
        raise NLLError(st, load().nll_server_last_error(handle).decode())


class Server:
    """Continuous batching of fits of one model kind (see nll_server_* in include/gbnll.h)."""

    def __init__(self, kind, obs_ranges, max_slots, pool_events, tile_events=4096, lo=None, hi=None, step=None,
                 fixed=None, tol_edm=1e-8, max_iter=500, strategy=1, hessian=1, device=0):
        L = load()
        self.kind = kind
        self.npar = 4 if kind == NLL_MODEL_MASS1D else 18
        self.ndim = 1 if kind == NLL_MODEL_MASS1D else 4
        th, lo, hi, step, fx = _fit_args(np.zeros(self.npar), lo, hi, step, fixed)
        opt = fit_options(tol_edm, max_iter, strategy, hessian)
        h = ctypes.c_void_p()
        st = L.nll_server_create(int(kind), _p(_f64(obs_ranges)), int(device), int(max_slots), int(pool_events),
                                 int(tile_events), _p(lo), _p(hi), _p(step),
                                 fx.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), ctypes.byref(opt), ctypes.byref(h))
        if st != NLL_OK:
            raise NLLError(st, "nll_server_create failed")
        self.handle = h.value
        self.max_slots = max_slots
        self._res = (fit_result * max_slots)()
        self._ids = (ctypes.c_int64 * max_slots)()

    def submit(self, columns, theta0):
        """Admit a fit; returns its id, or None when no slot or pool range is free."""
        cols = [_f64(c) for c in columns]
        ptrs = (ctypes.c_void_p * len(cols))(*[c.ctypes.data for c in cols])
        th = _f64(theta0)
        rid = ctypes.c_int64()
        st = load().nll_server_submit(self.handle, ptrs, None, len(cols[0]), _p(th), ctypes.byref(rid))
        if st == NLL_ERR_STATE:
            return None
        _scheck(self.handle, st)
        return rid.value

    def step(self, n=1):
        _scheck(self.handle, load().nll_server_step(self.handle, int(n)))

    def sync(self):
        _scheck(self.handle, load().nll_server_sync(self.handle))

    def progress(self):
        """Non-blocking: (steps queued and not yet completed, fits finished and not yet polled)."""
        a, b = ctypes.c_int(), ctypes.c_int()
        _scheck(self.handle, load().nll_server_progress(self.handle, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def cancel(self, request_id):
        """Withdraw an admitted fit that has not been polled: its slot and pool range are freed."""
        _scheck(self.handle, load().nll_server_cancel(self.handle, int(request_id)))

    def poll(self):
        """Finished fits as a list of (id, result dict); empty when none has finished (no wait)."""
        n = ctypes.c_int()
        _scheck(self.handle, load().nll_server_poll(self.handle, self._ids, self._res, self.max_slots, ctypes.byref(n)))
        return [(self._ids[i], _result_dict(self._res[i], self.npar)) for i in range(n.value)]

    def status(self):
        a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int64()
        _scheck(self.handle, load().nll_server_status(self.handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return dict(busy=a.value, free_slots=b.value, free_events=c.value)

    def close(self):
        if getattr(self, "handle", None):
            load().nll_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
