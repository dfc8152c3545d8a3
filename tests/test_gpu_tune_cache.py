"""Autotune results kept across processes (GBNLL_TUNE_CACHE): a second model or batch with the
same workload takes the kept result without timing, and a damaged cache line is skipped."""
import numpy as np
import pytest

from paper_2505_12414_gb300 import synth

pytestmark = pytest.mark.gpu


def test_model_autotune_is_kept(gpu_lib, tmp_path, monkeypatch):
    path = tmp_path / "tune.txt"
    monkeypatch.setenv("GBNLL_TUNE_CACHE", str(path))
    cols = synth.mass1d(100_000, stream=31)
    a = gpu_lib.Model(gpu_lib.NLL_MODEL_MASS1D, synth.RANGES_1D).load(cols)
    a.eval_grad(synth.TRUTH_1D)
    gpu_lib.nll_autotune(a.handle)
    lines = path.read_text().splitlines()
    assert len(lines) == 1 and len(lines[0].split()) == 4
    key, bps, thr, var = lines[0].split()
    assert "fused" in key
    launch_a = gpu_lib.nll_get_launch(a.handle)
    assert (launch_a["blocks_per_sm"], launch_a["threads"]) == (int(bps), int(thr))
    a.close()
    # the same workload in a new model: the kept result, nothing appended
    b = gpu_lib.Model(gpu_lib.NLL_MODEL_MASS1D, synth.RANGES_1D).load(cols)
    b.eval_grad(synth.TRUTH_1D)
    gpu_lib.nll_set_launch(b.handle, 1, 64)  # a shape the kept result replaces
    gpu_lib.nll_autotune(b.handle)
    assert path.read_text().splitlines() == lines
    got = gpu_lib.nll_get_launch(b.handle)
    assert got == launch_a
    b.close()
    # a damaged line for the same key is skipped: the last valid line still wins
    path.write_text(lines[0] + "\n" + key + " not numbers\n")
    c = gpu_lib.Model(gpu_lib.NLL_MODEL_MASS1D, synth.RANGES_1D).load(cols)
    c.eval_grad(synth.TRUTH_1D)
    gpu_lib.nll_autotune(c.handle)
    assert gpu_lib.nll_get_launch(c.handle) == launch_a
    c.close()


def test_batch_autotune_is_kept(gpu_lib, tmp_path, monkeypatch):
    path = tmp_path / "tune.txt"
    monkeypatch.setenv("GBNLL_TUNE_CACHE", str(path))
    off, cols = synth.toys1d(200, 1000.0, seed=synth.BASE_SEED + 61)
    a = gpu_lib.Batch(gpu_lib.NLL_MODEL_MASS1D, synth.RANGES_1D).load(off, cols)
    a.autotune()
    sched = a.get_schedule()
    a.close()
    lines = path.read_text().splitlines()
    assert len(lines) == 1 and "batch" in lines[0]
    b = gpu_lib.Batch(gpu_lib.NLL_MODEL_MASS1D, synth.RANGES_1D).load(off, cols)
    b.set_schedule(256, 1)
    b.autotune()
    assert b.get_schedule() == sched
    assert path.read_text().splitlines() == lines
    b.close()
