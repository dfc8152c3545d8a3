"""The no-allocation entry point (nll_eval_grad_4d_noalloc) against the oracle and against the
model entry point.

Some callers cannot call cudaMalloc: their device memory belongs to another allocator (a
framework that has reserved the device in its own pool), or they cannot accept cudaMalloc's
device-wide synchronisation.  They keep the sample in their own device buffers and call
nll_eval_grad_4d_noalloc, which uses a static device array as scratch.  Two calls in a row
must give the oracle's NLL and gradient within the parity tolerances used throughout the
tests (NLL 1e-12 of sum |w ln P|; gradient 1e-9 relative + 1e-13 of the term scale), and
what nll_eval_grad gives on the same events within the same tolerances.
"""
import numpy as np
import pytest

import oracle
from paper_2505_12414_gb300 import synth

pytestmark = pytest.mark.gpu


def _device_columns(cols, w):
    """Exactly-sized CUDA tensors (no padding: the entry point reads n_events doubles)."""
    import torch

    dev = [torch.from_numpy(np.ascontiguousarray(c)).to("cuda") for c in cols]
    wd = None if w is None else torch.from_numpy(np.ascontiguousarray(w)).to("cuda")
    torch.cuda.synchronize()
    return dev, wd


def _assert_oracle_parity(cols, w, th, nll, g):
    rn, rg, rs, st = oracle.nll_grad(oracle.KSTAR4D, synth.RANGES_4D, cols, th, w=w, nthreads=8)
    assert st == 0
    lp = np.log(oracle.pdf(oracle.KSTAR4D, synth.RANGES_4D, th, cols))
    nscale = np.sum(np.abs(lp if w is None else w * lp))
    assert abs(nll - rn) <= 1e-12 * nscale, (nll, rn)
    bad = np.abs(g - rg) > 1e-9 * np.abs(rg) + 1e-13 * rs
    assert not bad.any(), list(zip(np.where(bad)[0], g[bad], rg[bad]))
    return rs


@pytest.mark.parametrize("weighted", [False, True])
@pytest.mark.parametrize("n", [1, 3, 100003])
def test_noalloc_matches_oracle_and_model_two_calls(gpu_lib, weighted, n):
    cols = synth.kstar4d(n, stream=55)
    w = synth.weights(n, stream=56) if weighted else None
    dev, wd = _device_columns(cols, w)
    model = gpu_lib.Model(gpu_lib.NLL_MODEL_KSTARMUMU4D, synth.RANGES_4D)
    model.load(cols, w, precompute=False)
    scale = np.array([1.0, 1.0] + [0.03] * 8 + [2e-4] + [0.03] * 6 + [0.02])
    thetas = [synth.TRUTH_4D, synth.perturb(synth.TRUTH_4D, scale, k=3)]
    for th in thetas:  # two calls in a row share (and reuse) the static scratch
        nll, g = gpu_lib.nll_eval_grad_4d_noalloc(synth.RANGES_4D, dev, th, dev_weights=wd)
        rs = _assert_oracle_parity(cols, w, th, nll, g)
        ref_nll, ref_g = model.eval_grad(th)
        assert abs(nll - ref_nll) <= 1e-12 * abs(ref_nll)
        assert np.all(np.abs(g - ref_g) <= 1e-9 * np.abs(ref_g) + 1e-13 * rs)
    model.close()


def test_noalloc_on_a_side_stream(gpu_lib):
    import torch

    n = 20001
    cols = synth.kstar4d(n, stream=58)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):  # the columns are written on the side stream ...
        dev = [torch.from_numpy(c).to("cuda", non_blocking=False) * 1.0 for c in cols]
        # ... and the binding runs the call on the current (side) stream, after those writes
        nll, g = gpu_lib.nll_eval_grad_4d_noalloc(synth.RANGES_4D, dev, synth.TRUTH_4D)
    _assert_oracle_parity(cols, None, synth.TRUTH_4D, nll, g)
    nll2, g2 = gpu_lib.nll_eval_grad_4d_noalloc(synth.RANGES_4D, dev, synth.TRUTH_4D, stream=s.cuda_stream)
    assert nll2 == nll and np.array_equal(g2, g)


def test_noalloc_rejects_events_outside_the_ranges(gpu_lib):
    cols = [c.copy() for c in synth.kstar4d(1001, stream=59)]
    cols[2][1000] = 1.0000001  # the last event (a ragged tail pair)
    dev, _ = _device_columns(cols, None)
    nll, g, st = gpu_lib.nll_eval_grad_4d_noalloc(synth.RANGES_4D, dev, synth.TRUTH_4D, check=False)
    assert st == gpu_lib.NLL_ERR_ARG and nll == np.inf and np.all(np.isnan(g))
    w = synth.weights(1001, stream=60)
    w[7] = -0.5
    cols[2][1000] = 0.5
    dev, wd = _device_columns(cols, w)
    _, _, st = gpu_lib.nll_eval_grad_4d_noalloc(synth.RANGES_4D, dev, synth.TRUTH_4D, dev_weights=wd, check=False)
    assert st == gpu_lib.NLL_ERR_ARG


def test_noalloc_rejects_misaligned_columns_and_raw_pointers_without_a_count(gpu_lib):
    import torch

    cols = synth.kstar4d(1000, stream=61)
    dev, _ = _device_columns(cols, None)
    longer = torch.from_numpy(np.concatenate([[0.0], cols[2]])).to("cuda")
    shifted = [dev[0], dev[1], longer[1:], dev[3]]  # 8-byte offset: not 16-byte aligned
    _, _, st = gpu_lib.nll_eval_grad_4d_noalloc(synth.RANGES_4D, shifted, synth.TRUTH_4D, check=False)
    assert st == gpu_lib.NLL_ERR_ARG
    raw = [t.data_ptr() for t in dev]
    with pytest.raises(ValueError):
        gpu_lib.nll_eval_grad_4d_noalloc(synth.RANGES_4D, raw, synth.TRUTH_4D)
    nll, g = gpu_lib.nll_eval_grad_4d_noalloc(synth.RANGES_4D, raw, synth.TRUTH_4D, n_events=1000,
                                              stream=torch.cuda.current_stream().cuda_stream)
    _assert_oracle_parity(cols, None, synth.TRUTH_4D, nll, g)


def test_noalloc_rejects_sizes_beyond_the_static_scratch(gpu_lib):
    cols = synth.kstar4d(1000, stream=57)
    dev, _ = _device_columns(cols, None)
    _, _, st = gpu_lib.nll_eval_grad_4d_noalloc(synth.RANGES_4D, dev, synth.TRUTH_4D,
                                                blocks=gpu_lib.NLL_NOALLOC_MAX_BLOCKS + 1, check=False)
    assert st == gpu_lib.NLL_ERR_ARG
    nll, g, st = gpu_lib.nll_eval_grad_4d_noalloc(synth.RANGES_4D, dev, synth.TRUTH_4D,
                                                  blocks=gpu_lib.NLL_NOALLOC_MAX_BLOCKS, check=False)
    assert st == gpu_lib.NLL_OK
    _assert_oracle_parity(cols, None, synth.TRUTH_4D, nll, g)
