"""On-device generation (paper Sec. 2.5): the counter-based stream equals the host
generator's, generation is deterministic, and device-generated toys fitted at the generation
point give unbiased pulls of unit width."""
import math

import numpy as np
import pytest

import oracle
from paper_2505_12414_gb300 import synth

pytestmark = pytest.mark.gpu

M1, M4 = oracle.MASS1D, oracle.KSTAR4D


def test_device_stream_equals_host_splitmix64(gpu_lib):
    for seed, stream in ((synth.BASE_SEED, 0), (12345, 77), (2 ** 63 + 5, 3)):
        dev = gpu_lib.nll_diag_uniforms(seed, stream, 4099)
        host = synth.Stream(seed, stream).uniform(4099)
        assert np.array_equal(dev, host)


def test_generation_is_deterministic_and_in_range(gpu_lib):
    th = synth.TRUTH_4D
    a = gpu_lib.nll_generate(M4, synth.RANGES_4D, th, 50001, seed=11, stream=3)
    b = gpu_lib.nll_generate(M4, synth.RANGES_4D, th, 50001, seed=11, stream=3)
    c = gpu_lib.nll_generate(M4, synth.RANGES_4D, th, 50001, seed=11, stream=4)
    for x, y in zip(a, b):
        assert bool((x == y).all())
    assert not bool((a[0] == c[0]).all())
    m, ctl, ctk, phi = (t.cpu().numpy() for t in a)
    assert m.min() >= 5170 and m.max() <= 5970
    assert np.abs(ctl).max() <= 1 and np.abs(ctk).max() <= 1 and np.abs(phi).max() <= math.pi
    # the signal fraction within +-3 sigma of the peak (signal is 0.5 of the events)
    sig = np.mean(np.abs(m - 5279.6) < 60.0)
    assert 0.5 < sig < 0.7


def test_batch_toys_equal_standalone_streams(gpu_lib):
    counts = [1000, 0, 1, 4097]
    b = gpu_lib.Batch(M1, synth.RANGES_1D).generate(synth.TRUTH_1D, counts, seed=99)
    th = np.tile(synth.TRUTH_1D, (4, 1))
    nll, _, st = b.eval_grad(th)
    for t, n in enumerate(counts):
        if n == 0:
            assert nll[t] == 0.0
            continue
        cols = gpu_lib.nll_generate(M1, synth.RANGES_1D, synth.TRUTH_1D, n, seed=99, stream=t)
        ref, _, _, _ = oracle.nll_grad(M1, synth.RANGES_1D, [cols[0].cpu().numpy()], synth.TRUTH_1D)
        assert abs(nll[t] - ref) <= 1e-12 * abs(ref)
    b.close()


def _bounds(n):
    lo, hi = np.zeros(n), np.zeros(n)
    hi[-1] = 1.0
    return lo, hi


@pytest.mark.parametrize("kind,ntoy,nev,truth", [
    (M1, 400, 1000, synth.TRUTH_1D),
    (M4, 200, 2000, synth.TRUTH_4D),
    # the paper's angular benchmark point (FL = 0.6, other coefficients 0): folded generation
    (M4, 200, 2000, np.concatenate([synth.TRUTH_4D[:2], [0.6] + [0.0] * 7, synth.TRUTH_4D[10:]])),
])
def test_device_generated_toys_give_unit_pulls(gpu_lib, kind, ntoy, nev, truth):
    ranges = synth.RANGES_1D if kind == M1 else synth.RANGES_4D
    b = gpu_lib.Batch(kind, ranges).generate(truth, [nev] * ntoy, seed=2024)
    lo, hi = _bounds(len(truth))
    step = np.array([2.0, 1.0, 2e-4, 0.02]) if kind == M1 else np.array([1.0, 1.0] + [0.03] * 8 + [2e-4] + [0.03] * 6 + [0.02])
    r = b.fit(truth, lo=lo, hi=hi, step=step, tol_edm=1e-10, strategy=1, hessian=1)
    assert np.mean(r["status"] == 0) > 0.99
    ok = r["status"] == 0
    pulls = (r["theta"][ok] - truth) / r["err"][ok]
    n = ok.sum()
    mean, width = pulls.mean(axis=0), pulls.std(axis=0)
    assert np.all(np.abs(mean) < 4.0 / math.sqrt(n) + 0.03), mean
    assert np.all(np.abs(width - 1.0) < 4.0 / math.sqrt(2 * n) + 0.03), width
    b.close()
