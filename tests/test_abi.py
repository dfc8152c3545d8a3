"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every declared symbol."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER_DIR = os.path.join(ROOT, "include")


def declared_functions():
    names = []
    for fn in sorted(os.listdir(HEADER_DIR)):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(HEADER_DIR, fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"^\s*(?:const\s+)?(?:int|void|char|double|int64_t)\s*\**\s*(\w+)\s*\(", text, re.M):
            names.append(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2505_12414_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("nll_create_model", "nll_load_events", "nll_eval", "nll_eval_grad", "fit_minimise"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_library_targets_sm_103a():
    from paper_2505_12414_gb300 import build

    assert "arch=compute_103a,code=sm_103a" in build.ARCH


def test_null_and_bad_arguments_are_rejected_without_a_gpu(lib):
    lib.nll_num_params.argtypes = [ctypes.c_void_p]
    assert lib.nll_num_params(None) == -1
    lib.nll_destroy.argtypes = [ctypes.c_void_p]
    lib.nll_destroy(None)  # accepted
    h = ctypes.c_void_p()
    r = (ctypes.c_double * 2)(5170.0, 5970.0)
    lib.nll_create_model.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_size_t,
                                     ctypes.POINTER(ctypes.c_void_p)]
    assert lib.nll_create_model(7, r, 0, 0, ctypes.byref(h)) == 1  # unknown kind -> NLL_ERR_ARG
    bad = (ctypes.c_double * 2)(5970.0, 5170.0)
    assert lib.nll_create_model(1, bad, 0, 0, ctypes.byref(h)) == 1
    assert h.value is None


def test_hessian_slot_counts_without_a_gpu(lib):
    lib.nll_hess_num_slots.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
    assert lib.nll_hess_num_slots(3, 0, 0) == -1
    for kind, npar in ((1, 4), (2, 18)):
        for weighted in (0, 1):
            h = lib.nll_hess_num_slots(kind, weighted, 0)
            hw = lib.nll_hess_num_slots(kind, weighted, 1)
            # at least one slot per Hessian entry; W adds its npar (npar + 1) / 2 products, some
            # of which the unweighted Hessian already holds
            assert npar * (npar + 1) // 2 <= h < hw <= 384
            if weighted:
                assert hw - h == npar * (npar + 1) // 2


def test_fit_result_record_layout_matches_the_header():
    """The binding reads batched fit results as numpy records of the C struct fit_result
    (include/gbnll.h): same size, same field offsets."""
    import numpy as np

    import paper_2505_12414_gb300 as g

    dt = g._FIT_RESULT_DTYPE
    assert dt.itemsize == ctypes.sizeof(g.fit_result)
    for name, _ in g.fit_result._fields_:
        assert dt.fields[name][1] == getattr(g.fit_result, name).offset
    rec = np.zeros(2, dtype=dt)
    rec["theta"][1, :3] = [1.0, 2.0, 3.0]
    rec["cov"][1, :9] = np.arange(9.0)
    rec["status"][1] = 5
    view = (g.fit_result * 2).from_buffer(rec)
    assert view[1].theta[2] == 3.0 and view[1].cov[4] == 4.0 and view[1].status == 5
    out = g._results_of(rec, 3, steps=4)
    assert out["theta"][1].tolist() == [1.0, 2.0, 3.0]
    assert out["cov"][1].tolist() == [[0.0, 1.0, 2.0], [3.0, 4.0, 5.0], [6.0, 7.0, 8.0]]
    assert out["status"].tolist() == [0, 5] and out["steps"] == 4


def test_binding_fails_loudly_without_the_library(tmp_path):
    """No CPU fallback: loading a library path that does not exist raises, in a fresh
    interpreter so the already-loaded library of this process is not reused."""
    import subprocess
    import sys

    code = ("import paper_2505_12414_gb300 as g\n"
            "try:\n"
            "    g.load(%r)\n"
            "except RuntimeError as e:\n"
            "    print('raised', 'not built' in str(e))\n" % str(tmp_path / "libgbnll.so"))
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == "raised True"
