"""The kernels' integer exponential and reciprocal (fexp_scaled, frcp), built for the host from the
same header, against extended-precision references (no GPU).  The exponential is integer
arithmetic throughout, so the host build computes the device's results bit for bit (test_gpu_math
checks that on a GPU); the reciprocal's host build seeds with the rounded single-precision
quotient where the device takes the hardware approximation, and refines the seed the same way."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2505_12414_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2505_12414_gb300", "csrc")
S = 1024.0 / np.log(2.0)  # the kernels pass x * 1024/ln2


def host_math_binary(tmpdir):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    out = os.path.join(str(tmpdir), "math_host")
    subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-I", CSRC,
                           os.path.join(HERE, "host", "math_host.cu"), "-o", out])
    return out


def host_math(binary, fn, xs, tmpdir):
    src, dst = os.path.join(str(tmpdir), "x.bin"), os.path.join(str(tmpdir), "y.bin")
    np.ascontiguousarray(xs, dtype=np.float64).tofile(src)
    subprocess.check_call([binary, fn, src, dst])
    return np.fromfile(dst, dtype=np.float64)


def exp_reference(xs):
    """exp(xs ln2/1024) through the exact split xs = k + f (k = floor xs):
    2^(k >> 10) 2^(((k & 1023) + f)/1024), so that the extended-precision exp2 sees an argument
    in [0, 1) and the reference error stays far below an ulp of the result at any |x| <= 704."""
    k = np.floor(xs)
    f = (xs - k).astype(np.longdouble)  # exact
    ki = k.astype(np.int64)
    return np.ldexp(np.exp2((np.longdouble(1) * (ki & 1023) + f) / np.longdouble(1024)), (ki >> 10).astype(np.int32))


def ulp_error(y, ref):
    return np.abs(y.astype(np.longdouble) - ref) / np.spacing(ref.astype(np.float64)).astype(np.longdouble)


def exp_arguments(seed):
    rs = synth.Stream(seed, 0)
    steps = np.arange(-2048, 2049).astype(np.float64)
    return np.concatenate([
        (2 * rs.uniform(300000) - 1) * 703.0 * S,  # the whole fast range
        (2 * rs.uniform(300000) - 1) * 40.0 * S,   # the range the likelihood uses
        (2 * rs.uniform(50000) - 1) * 2.0,         # a few table steps around zero
        (2 * rs.uniform(50000) - 1) * 1e-3,        # small fractions of both signs
        steps, steps + 0.5, np.nextafter(steps, np.inf), np.nextafter(steps, -np.inf),  # reduction edges
        np.array([0.0, -0.0, 1e-300, -1e-300, 5e-324, -5e-324, 2.0 ** -70, -(2.0 ** -70),
                  703.9 * S, -703.9 * S, 1039871.9, -1039871.9]),
    ])


def test_integer_exponential_accuracy(tmp_path):
    binary = host_math_binary(tmp_path)
    xs = exp_arguments(31)
    y = host_math(binary, "exp", xs, tmp_path)
    err = ulp_error(y, exp_reference(xs))
    assert float(err.max()) < 0.52, float(err.max())  # one rounding from 63 bits, plus < 0.02 ulp
    # exactness where the result is a power of two
    p2 = np.arange(-700, 701) * 1024.0
    np.testing.assert_array_equal(host_math(binary, "exp", p2, tmp_path), np.ldexp(1.0, np.arange(-700, 701)))


def test_integer_exponential_saturation_and_monotonicity(tmp_path):
    binary = host_math_binary(tmp_path)
    big = np.array([-1.04e6, -2e6, -1e300, -np.inf, 1.04e6, 2e6, 1e300, np.inf, np.nan])
    yb = host_math(binary, "exp", big, tmp_path)
    assert np.all(yb[:4] == 0.0) and np.all(np.isinf(yb[4:]))
    # monotone over consecutive doubles across table steps and binades
    x = np.concatenate([v + np.arange(-32, 32) * 2.0 ** -40 for v in (-1024.0, -1.0, 0.0, 1023.0, 5000.0)])
    y = host_math(binary, "exp", np.sort(x), tmp_path)
    assert np.all(np.diff(y) >= 0)


def rcp_arguments(seed):
    rs = synth.Stream(seed, 0)
    m = 1.0 + np.arange(4096) / 4096.0  # every 12-bit mantissa prefix
    return np.concatenate([
        np.exp((2 * rs.uniform(300000) - 1) * 700.0),
        -np.exp((2 * rs.uniform(30000) - 1) * 700.0),
        1.0 + rs.uniform(100000), m, np.nextafter(m, 0.0), np.nextafter(m, 3.0),
        np.array([1.0, 2.0, 3.0, 0.1, 1.0 - 2 ** -52, 1.0 + 2 ** -52, 2.0 - 2 ** -51, 2.0 ** -1022, 2.0 ** 1021,
                  np.finfo(np.float64).max / 4, -1.0, -2.0 ** -1000]),
    ])


def test_integer_reciprocal_accuracy(tmp_path):
    binary = host_math_binary(tmp_path)
    x = rcp_arguments(32)
    y = host_math(binary, "rcp", x, tmp_path)
    ref = np.longdouble(1) / x.astype(np.longdouble)
    err = ulp_error(y, ref)
    assert float(err.max()) < 0.51, float(err.max())
    assert np.all(np.signbit(y) == np.signbit(x))
    # powers of two are exact; out of the normal range: 0 and inf with the sign of x
    p2 = np.ldexp(1.0, np.arange(-1021, 1022))
    np.testing.assert_array_equal(host_math(binary, "rcp", p2, tmp_path), np.ldexp(1.0, -np.arange(-1021, 1022)))
    edge = host_math(binary, "rcp", np.array([2.0 ** 1022, -(2.0 ** 1023), 0.0, -0.0, 1e-310]), tmp_path)
    assert edge[0] == 0.0 and edge[1] == 0.0 and np.signbit(edge[1])
    assert np.isinf(edge[2]) and edge[2] > 0 and np.isinf(edge[3]) and edge[3] < 0 and np.isinf(edge[4])
