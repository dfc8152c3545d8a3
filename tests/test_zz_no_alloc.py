"""The no-allocation entry point (nll_eval_grad_4d_noalloc) against the model entry point.

Some callers cannot call cudaMalloc: their device memory belongs to another allocator (a
framework that has reserved the device in its own pool), or they cannot accept cudaMalloc's
device-wide synchronisation.  They keep the sample in their own device buffers and call
nll_eval_grad_4d_noalloc, which uses a static device array as scratch.  Two calls in a row
must give what nll_eval_grad gives on the same events, within the parity tolerances used
throughout the tests (NLL 1e-12 relative; gradient 1e-9 relative + 1e-13 of the term scale).
"""
import numpy as np
import pytest

import oracle
from paper_2505_12414_gb300 import synth

pytestmark = pytest.mark.gpu


def _device_columns(cols, w):
    import torch

    n = len(cols[0])
    npad = n + (n & 1)  # readable for an even count of doubles (pairs of events per load)
    dev = []
    for c in cols:
        t = torch.zeros(npad, dtype=torch.float64, device="cuda")
        t[:n] = torch.from_numpy(c)
        dev.append(t)
    wd = None
    if w is not None:
        wd = torch.zeros(npad, dtype=torch.float64, device="cuda")
        wd[:n] = torch.from_numpy(w)
    torch.cuda.synchronize()
    return dev, wd


@pytest.mark.parametrize("weighted", [False, True])
def test_noalloc_matches_model_entry_point_two_calls(gpu_lib, weighted):
    n = 100003
    cols = synth.kstar4d(n, stream=55)
    w = synth.weights(n, stream=56) if weighted else None
    dev, wd = _device_columns(cols, w)
    model = gpu_lib.Model(gpu_lib.NLL_MODEL_KSTARMUMU4D, synth.RANGES_4D)
    model.load(cols, w, precompute=False)
    scale = np.array([1.0, 1.0] + [0.03] * 8 + [2e-4] + [0.03] * 6 + [0.02])
    thetas = [synth.TRUTH_4D, synth.perturb(synth.TRUTH_4D, scale, k=3)]
    for th in thetas:  # two calls in a row share (and reuse) the static scratch
        ref_nll, ref_g = model.eval_grad(th)
        nll, g = gpu_lib.nll_eval_grad_4d_noalloc_n(synth.RANGES_4D, dev, n, th, dev_weights=wd)
        _, _, s, st = oracle.nll_grad(oracle.KSTAR4D, synth.RANGES_4D, cols, th, w=w, nthreads=8)
        assert st == 0
        assert abs(nll - ref_nll) <= 1e-12 * abs(ref_nll)
        assert np.all(np.abs(g - ref_g) <= 1e-9 * np.abs(ref_g) + 1e-13 * s)
    model.close()


def test_noalloc_rejects_sizes_beyond_the_static_scratch(gpu_lib):
    cols = synth.kstar4d(1000, stream=57)
    dev, _ = _device_columns(cols, None)
    _, _, st = gpu_lib.nll_eval_grad_4d_noalloc_n(synth.RANGES_4D, dev, 1000, synth.TRUTH_4D,
                                                  blocks=gpu_lib.NLL_NOALLOC_MAX_BLOCKS + 1, check=False)
    assert st == gpu_lib.NLL_ERR_ARG
    nll, _, st = gpu_lib.nll_eval_grad_4d_noalloc_n(synth.RANGES_4D, dev, 1000, synth.TRUTH_4D,
                                                    blocks=gpu_lib.NLL_NOALLOC_MAX_BLOCKS, check=False)
    assert st == gpu_lib.NLL_OK and np.isfinite(nll)
