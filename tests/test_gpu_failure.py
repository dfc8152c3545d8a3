"""Failure paths provoked from the host (no GPU fault): running out of device memory through
the per-object allocation limit (GBNLL_DEVICE_ALLOC_LIMIT, read at creation), a cancelled
served fit, and requests that can never be admitted.  Every object stays usable or can be
destroyed, and destroying it returns all the device memory it held."""
import os

import numpy as np
import pytest

from paper_2505_12414_gb300 import synth

pytestmark = pytest.mark.gpu


class alloc_limit:
    """Set GBNLL_DEVICE_ALLOC_LIMIT for the objects created inside the block."""

    def __init__(self, nbytes):
        self.nbytes = nbytes

    def __enter__(self):
        self.old = os.environ.get("GBNLL_DEVICE_ALLOC_LIMIT")
        os.environ["GBNLL_DEVICE_ALLOC_LIMIT"] = str(int(self.nbytes))

    def __exit__(self, *exc):
        if self.old is None:
            del os.environ["GBNLL_DEVICE_ALLOC_LIMIT"]
        else:
            os.environ["GBNLL_DEVICE_ALLOC_LIMIT"] = self.old


def free_device_bytes():
    import torch

    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def test_model_load_beyond_the_limit_returns_oom_and_the_model_stays_usable(gpu_lib):
    base = free_device_bytes()
    with alloc_limit(16 << 20):
        m = gpu_lib.Model(gpu_lib.NLL_MODEL_KSTARMUMU4D, synth.RANGES_4D)
    big = synth.kstar4d(200_000, stream=61)  # 27 MB with the angular basis
    with pytest.raises(gpu_lib.NLLError) as e:
        m.load(big, precompute=True)
    assert e.value.status == gpu_lib.NLL_ERR_OOM
    with pytest.raises(gpu_lib.NLLError) as e:  # no sample kept
        m.eval(synth.TRUTH_4D)
    assert e.value.status == gpu_lib.NLL_ERR_STATE
    small = synth.kstar4d(20_000, stream=62)
    m.load(small, precompute=True)
    nll, g = m.eval_grad(synth.TRUTH_4D)
    assert np.isfinite(nll) and np.all(np.isfinite(g))
    # the Hessian scratch is allocated at the first Hessian call: past the limit it fails the
    # same way and the gradient path goes on working
    with alloc_limit(1 << 20):
        m2 = gpu_lib.Model(gpu_lib.NLL_MODEL_MASS1D, synth.RANGES_1D)
    with pytest.raises(gpu_lib.NLLError) as e:
        m2.load(synth.mass1d(200_000, stream=63))
    assert e.value.status == gpu_lib.NLL_ERR_OOM
    m2.load(synth.mass1d(1000, stream=63))
    with pytest.raises(gpu_lib.NLLError) as e:
        m2.eval_hess(synth.TRUTH_1D)
    assert e.value.status == gpu_lib.NLL_ERR_OOM
    assert np.isfinite(m2.eval_grad(synth.TRUTH_1D)[0])
    m.close()
    m2.close()
    assert abs(free_device_bytes() - base) < (4 << 20)


def test_batch_load_beyond_the_limit_returns_oom(gpu_lib):
    base = free_device_bytes()
    with alloc_limit(8 << 20):
        b = gpu_lib.Batch(gpu_lib.NLL_MODEL_MASS1D, synth.RANGES_1D)
    off, cols = synth.toys1d(2000, 1000.0, seed=synth.BASE_SEED + 64)  # 2M events: 16 MB of events alone
    with pytest.raises(gpu_lib.NLLError) as e:
        b.load(off, cols)
    assert e.value.status == gpu_lib.NLL_ERR_OOM
    off, cols = synth.toys1d(20, 1000.0, seed=synth.BASE_SEED + 65)
    b.load(off, cols)
    nll, _, st = b.eval_grad(np.tile(synth.TRUTH_1D, (20, 1)))
    assert np.all(st == 0) and np.all(np.isfinite(nll))
    b.close()
    assert abs(free_device_bytes() - base) < (4 << 20)


def test_server_create_beyond_the_limit_returns_oom_and_submit_allocates_nothing(gpu_lib):
    base = free_device_bytes()
    lo, hi = np.zeros(4), np.zeros(4)
    hi[3] = 1.0
    opts = dict(lo=lo, hi=hi, step=np.array([2.0, 1.0, 2e-4, 0.02]), tol_edm=1e-10, strategy=2, hessian=2)
    with alloc_limit(8 << 20):
        with pytest.raises(gpu_lib.NLLError) as e:
            gpu_lib.Server(gpu_lib.NLL_MODEL_MASS1D, synth.RANGES_1D, 8, 4_000_000, 1024, **opts)
        assert e.value.status == gpu_lib.NLL_ERR_OOM
        s = gpu_lib.Server(gpu_lib.NLL_MODEL_MASS1D, synth.RANGES_1D, 4, 100_000, 1024, **opts)
    # admission uses the pool only: a request larger than the pool is refused, one that does
    # not fit now waits, and neither allocates
    with pytest.raises(gpu_lib.NLLError) as e:
        s.submit(synth.mass1d(150_000, stream=66), synth.TRUTH_1D)
    assert e.value.status == gpu_lib.NLL_ERR_ARG
    r1 = s.submit(synth.mass1d(80_000, stream=67), synth.TRUTH_1D)
    assert r1 is not None and s.submit(synth.mass1d(30_000, stream=68), synth.TRUTH_1D) is None
    s.cancel(r1)
    assert s.status()["free_events"] == 100_000
    r2 = s.submit(synth.mass1d(30_000, stream=68), synth.TRUTH_1D)
    done = []
    for _ in range(2000):
        s.step(2)
        s.sync()
        done += s.poll()
        if done:
            break
    assert [d[0] for d in done] == [r2] and done[0][1]["status"] == 0
    s.close()
    assert abs(free_device_bytes() - base) < (4 << 20)
