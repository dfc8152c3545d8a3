"""In-place samples (nll_load_events with on_device = 2): the kernels read the caller's
buffers -- pinned host memory over the CPU-GPU link, device memory, or pageable host memory
where the device reads it -- and match the oracle and the copying path."""
import numpy as np
import pytest
import torch

import oracle
from paper_2505_12414_gb300 import synth

pytestmark = pytest.mark.gpu

M1, M4 = oracle.MASS1D, oracle.KSTAR4D


def sample(kind, n, stream, weighted):
    cols = synth.mass1d(n, stream=stream) if kind == M1 else synth.kstar4d(n, stream=stream)
    ranges = synth.RANGES_1D if kind == M1 else synth.RANGES_4D
    theta = np.array([5283.0, 22.0, -0.0017, 0.35]) if kind == M1 else synth.TRUTH_4D + 0.01
    w = synth.weights(n, stream=stream + 1) if weighted else None
    return cols, ranges, theta, w


def pinned(a):
    t = torch.empty(len(a), dtype=torch.float64, pin_memory=True)
    t.numpy()[:] = a
    return t


def placed(arrays, where):
    if where == "pinned":
        return [pinned(a) for a in arrays]
    if where == "device":
        return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrays]
    return [np.ascontiguousarray(a) for a in arrays]  # pageable host memory


@pytest.mark.parametrize("n", [1, 3, 128, 129, 4097, 100001])
@pytest.mark.parametrize("kind,weighted", [(M1, False), (M1, True), (M4, False), (M4, True)])
@pytest.mark.parametrize("where", ["pinned", "device", "pageable"])
def test_in_place_parity(gpu_lib, kind, weighted, n, where):
    cols, ranges, theta, w = sample(kind, n, 400 + n, weighted)
    arrs = placed(list(cols) + ([w] if weighted else []), where)
    m = gpu_lib.Model(kind, ranges)
    try:
        m.load(arrs[: len(cols)], arrs[len(cols)] if weighted else None, in_place=True)
    except gpu_lib.NLLError as e:
        # the library refuses pageable memory where the device cannot read it
        if where == "pageable" and e.status == gpu_lib.NLL_ERR_ARG:
            pytest.skip("device does not read pageable host memory")
        raise
    nll, g = m.eval_grad(theta)
    rn, rg, rs, rst = oracle.nll_grad(kind, ranges, cols, theta, w=w)
    assert rst == 0
    lp = np.log(oracle.pdf(kind, ranges, theta, cols))
    nscale = np.sum(np.abs(lp if w is None else w * lp))
    assert abs(nll - rn) <= 1e-12 * nscale
    assert np.all(np.abs(g - rg) <= 1e-9 * np.abs(rg) + 1e-13 * rs)
    # the copying path, direct variant, same launch shape: the same gradient bits
    c = gpu_lib.Model(kind, ranges).load(cols, w, precompute=False)
    launch = gpu_lib.nll_get_launch(m.handle)
    gpu_lib.nll_set_launch(c.handle, launch["blocks_per_sm"], launch["threads"], 0)
    n2, g2 = c.eval_grad(theta)
    assert np.array_equal(g, g2)
    assert abs(nll - n2) <= 1e-14 * nscale
    m.close()
    c.close()


def test_in_place_rejects_events_outside_and_bad_weights(gpu_lib):
    cols, ranges, theta, w = sample(M4, 1001, 420, True)
    cols = [c.copy() for c in cols]
    cols[1][500] = 1.5  # cos theta_l outside [-1, 1]
    m = gpu_lib.Model(M4, ranges).load([pinned(c) for c in cols], pinned(w), in_place=True)
    nll, g, st = gpu_lib.nll_eval_grad(m.handle, theta, check=False)
    assert st == gpu_lib.NLL_ERR_ARG and nll == np.inf
    cols[1][500] = 0.5
    w = w.copy()
    w[7] = -1.0
    m.load([pinned(c) for c in cols], pinned(w), in_place=True)
    nll, g, st = gpu_lib.nll_eval_grad(m.handle, theta, check=False)
    assert st == gpu_lib.NLL_ERR_ARG
    w[7] = 1.0
    m.load([pinned(c) for c in cols], pinned(w), in_place=True)
    nll, g = m.eval_grad(theta)
    assert np.isfinite(nll)
    m.close()


def test_in_place_rejects_misaligned_buffers(gpu_lib):
    cols, ranges, theta, _ = sample(M1, 1000, 430, False)
    buf = pinned(np.concatenate([[0.0], cols[0]]))
    m = gpu_lib.Model(M1, ranges)
    with pytest.raises(gpu_lib.NLLError) as e:
        m.load([buf[1:]], in_place=True)  # 8-byte offset: not 16-byte aligned
    assert e.value.status == gpu_lib.NLL_ERR_ARG
    m.close()


def test_in_place_hessian_and_fit(gpu_lib):
    cols, ranges, theta, w = sample(M4, 20001, 440, True)
    m = gpu_lib.Model(M4, ranges).load([pinned(c) for c in cols], pinned(w), in_place=True)
    c = gpu_lib.Model(M4, ranges).load(cols, w, precompute=False)
    a = m.eval_hess(theta, w2=True)
    b = c.eval_hess(theta, w2=True)
    assert abs(a[0] - b[0]) <= 1e-13 * abs(b[0])
    assert np.array_equal(a[2], b[2]) and np.array_equal(a[3], b[3])
    lo, hi = np.zeros(18), np.zeros(18)
    hi[-1] = 1.0
    step = np.array([1.0, 1.0] + [0.03] * 8 + [2e-4] + [0.03] * 6 + [0.02])
    ra = m.fit(synth.TRUTH_4D, lo=lo, hi=hi, step=step, tol_edm=1e-12, strategy=2, hessian=3)
    rb = c.fit(synth.TRUTH_4D, lo=lo, hi=hi, step=step, tol_edm=1e-12, strategy=2, hessian=3)
    assert ra["status"] == 0 and rb["status"] == 0
    assert np.max(np.abs((ra["theta"] - rb["theta"]) / rb["err"])) < 1e-6
    np.testing.assert_allclose(ra["err"], rb["err"], rtol=1e-6)
    m.close()
    c.close()


@pytest.mark.parametrize("n", [1, 129, 100001])
@pytest.mark.parametrize("kind,weighted", [(M1, True), (M4, False), (M4, True)])
def test_copying_load_reads_pinned_and_pageable_alike(gpu_lib, kind, weighted, n):
    # load() stores host columns through its statistics kernel (pinned memory, and pageable
    # memory where the device reads it) or by cudaMemcpyAsync: every route stores the same
    # events, so the evaluations agree bit for bit, and out-of-range events are still refused
    cols, ranges, theta, w = sample(kind, n, 470 + n, weighted)
    res = []
    for where in ("pageable", "pinned", "device"):
        arrs = placed(list(cols) + ([w] if weighted else []), where)
        m = gpu_lib.Model(kind, ranges).load(arrs[:len(cols)], arrs[len(cols)] if weighted else None)
        res.append(m.eval_grad(theta))
        m.close()
    for f, g in res[1:]:
        assert f == res[0][0] and np.array_equal(g, res[0][1])
    bad = [c.copy() for c in cols]
    bad[0][n // 2] = ranges[1] + 1.0  # one event above the mass window
    m = gpu_lib.Model(kind, ranges)
    with pytest.raises(gpu_lib.NLLError) as e:
        m.load([pinned(c) for c in bad], pinned(w) if weighted else None)
    assert e.value.status == gpu_lib.NLL_ERR_ARG
    m.close()
