"""The kernels' integer exponential, logarithm, reciprocal, square root, sine/cosine and running
product (fexp_scaled, flog, frcp, fsqrt, fsincos_pi, LogProd), built for the host from the same header, against extended-precision references (no GPU).  The exponential, the
logarithm and the sine/cosine are integer arithmetic throughout, so the host build computes the device's results bit
for bit (test_gpu_math checks that on a GPU); the reciprocal's and the square root's host builds seed with rounded
single-precision arithmetic where the device takes the hardware approximations, and refine the
seed the same way."""
import os
import shutil
import subprocess

from decimal import Decimal, getcontext

import numpy as np
import pytest

from paper_2505_12414_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2505_12414_gb300", "csrc")
S = 1024.0 / np.log(2.0)  # the kernels pass x * 1024/ln2


_BINARY = {}


def host_math_binary(tmpdir):
    """The host build of the special functions, compiled once per session (the first caller's
    tmpdir holds it)."""
    if "path" in _BINARY:
        return _BINARY["path"]
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    out = os.path.join(str(tmpdir), "math_host")
    subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-I", CSRC,
                           os.path.join(HERE, "host", "math_host.cu"), "-o", out])
    _BINARY["path"] = out
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


def test_integer_running_product(tmp_path):
    # ln of products of 64 factors spanning many binades, against the sum of extended-precision logs
    binary = host_math_binary(tmp_path)
    rs = synth.Stream(33, 0)
    x = np.exp((2 * rs.uniform(64 * 4000) - 1) * 30.0)
    x[:64] = 1.0                      # the empty product's neutral factors
    x[64:128] = 2.0 ** -1022          # the smallest normal, 64 times
    x[128:192] = 1.0 + 2.0 ** -52     # one ulp above 1, 64 times
    y = host_math(binary, "lprod", x, tmp_path)
    ref = np.log(x.astype(np.longdouble)).reshape(-1, 64).sum(axis=1)
    err = np.abs(y.astype(np.longdouble) - ref)
    # 64 truncated products (< 2^-62 each), the mantissa rounded to 53 bits, log and the e ln2 terms
    bound = 64 * 2.0 ** -62 + 2.0 ** -53 + 4 * np.spacing(np.abs(ref.astype(np.float64))).astype(np.longdouble)
    assert np.all(err <= bound), float((err / bound).max())
    assert y[0] == 0.0


def log_arguments(seed):
    rs = synth.Stream(seed, 0)
    steps = 1.0 + np.arange(257) / 256.0  # table points and the midpoints between them
    return np.concatenate([
        np.exp((2 * rs.uniform(300000) - 1) * 700.0),  # the whole normal range
        rs.uniform(100000) + 1e-300,                    # (0, 1], as in the generator
        1.0 + (2 * rs.uniform(100000) - 1) * 2.0 ** -8,  # around 1, where ln x is small
        1.0 + (2 * rs.uniform(20000) - 1) * 2.0 ** -40,
        steps, np.nextafter(steps, 0.0), np.nextafter(steps, 3.0), steps / 2, np.nextafter(steps / 2, 0.0),
        np.array([1.0, 1.0 + 2.0 ** -52, 1.0 - 2.0 ** -53, 2.0, 0.5, 2.0 ** -1022, np.finfo(np.float64).max,
                  np.e, 10.0, 0.1]),
    ])


def test_integer_logarithm_accuracy(tmp_path):
    binary = host_math_binary(tmp_path)
    x = log_arguments(34)
    y = host_math(binary, "log", x, tmp_path)
    ref = np.log(x.astype(np.longdouble))
    err = ulp_error(y, ref)
    assert float(err.max()) < 0.51, float(err.max())
    assert y[x == 1.0].tolist() == [0.0] * int((x == 1.0).sum())
    np.testing.assert_array_equal(np.sign(y), np.sign(np.log(x)))


def test_logarithm_tables_against_decimal(tmp_path):
    # ln F_j 2^115 and 1/F_j 2^63 (F_j = 1 + j/128) and ln 2 2^115, against 60-digit decimals
    binary = host_math_binary(tmp_path)
    src = tmp_path / "none.bin"
    np.zeros(1).tofile(src)
    out = tmp_path / "tab.bin"
    subprocess.check_call([binary, "logtab", str(src), str(out)])
    w = [int(v) for v in np.fromfile(out, dtype=np.uint64)]
    n = 128
    getcontext().prec = 60
    for j in range(n):
        F = 1 + Decimal(j) / 128
        lnF = (w[j] << 64) | w[n + j]
        exact = F.ln() * (Decimal(2) ** 115)
        assert abs(Decimal(lnF) - exact) <= 1, j
        inv = w[2 * n + j]
        assert abs(Decimal(inv) - (Decimal(2) ** 63) / F) <= Decimal("0.5"), j
    ln2_series = (w[3 * n] << 64) | w[3 * n + 1]
    ln2_const = (w[3 * n + 2] << 64) | w[3 * n + 3]
    assert ln2_series == ln2_const
    assert abs(Decimal(ln2_const) - Decimal(2).ln() * (Decimal(2) ** 115)) <= Decimal("0.5")


def sincos_arguments(seed):
    rs = synth.Stream(seed, 0)
    steps = np.arange(-512, 513) * (np.pi / 512)
    x = np.concatenate([
        (2 * rs.uniform(300000) - 1) * np.pi,
        steps, np.nextafter(steps, 10.0), np.nextafter(steps, -10.0),   # around the table points
        steps + np.pi / 1024, steps - np.pi / 1024,                     # the reduction's edges
        (2 * rs.uniform(20000) - 1) * 1e-3, (2 * rs.uniform(2000) - 1) * 1e-9,
        np.array([0.0, -0.0, 1e-300, -1e-300, 2.0 ** -26, 2.0 ** -27, 1e-8, np.pi, -np.pi, np.pi / 2, -np.pi / 2,
                  np.nextafter(np.pi, 0.0), np.nextafter(np.pi / 2, 0.0), np.nextafter(np.pi / 2, 4.0)]),
    ])
    return x[np.abs(x) <= np.pi]


def sincos_ulp(y, ref):
    out = np.zeros(len(y))
    nz = ref != 0
    out[nz] = np.asarray(ulp_error(y[nz], ref[nz]), dtype=np.float64)
    out[~nz] = np.where(y[~nz] == 0, 0.0, np.inf)
    return out


def test_integer_sincos_accuracy(tmp_path):
    binary = host_math_binary(tmp_path)
    x = sincos_arguments(35)
    y = host_math(binary, "sincos", x, tmp_path).reshape(-1, 2)
    xl = x.astype(np.longdouble)
    es, ec = sincos_ulp(y[:, 0], np.sin(xl)), sincos_ulp(y[:, 1], np.cos(xl))
    assert es.max() < 1.0 and ec.max() < 1.0, (es.max(), ec.max(), x[np.argmax(es)], x[np.argmax(ec)])
    np.testing.assert_array_equal(np.signbit(y[:, 0]), np.signbit(np.sin(x)))
    # exact values: sin 0 = 0 with its sign, cos 0 = 1, |x| < 2^-26 returns (x, 1)
    z = host_math(binary, "sincos", np.array([0.0, -0.0, 1e-10, -1e-10]), tmp_path).reshape(-1, 2)
    assert z[0, 0] == 0.0 and not np.signbit(z[0, 0]) and np.signbit(z[1, 0]) and np.all(z[:, 1] == 1.0)
    assert z[2, 0] == 1e-10 and z[3, 0] == -1e-10


def sqrt_arguments(seed):
    rs = synth.Stream(seed, 0)
    m = 1.0 + np.arange(4096) / 1024.0  # every 12-bit prefix of [1, 5), both exponent parities
    return np.concatenate([
        rs.uniform(200000), rs.uniform(100000) * rs.uniform(100000),  # sin^2 products in [0, 1]
        np.exp((2 * rs.uniform(100000) - 1) * 700.0),
        m, np.nextafter(m, 0.0), np.nextafter(m, 9.0), m * m,
        np.array([1.0, 2.0, 4.0, 0.25, 2.0 - 2.0 ** -52, 4.0 - 2.0 ** -50, 2.0 ** -1022, np.finfo(np.float64).max]),
    ])


def test_integer_sqrt_accuracy(tmp_path):
    binary = host_math_binary(tmp_path)
    x = sqrt_arguments(36)
    y = host_math(binary, "sqrt", x, tmp_path)
    err = ulp_error(y, np.sqrt(x.astype(np.longdouble)))
    assert float(err.max()) < 0.52, (float(err.max()), x[np.argmax(err)])
    sq = np.arange(1, 3000, dtype=np.float64)
    np.testing.assert_array_equal(host_math(binary, "sqrt", sq * sq, tmp_path), sq)  # exact squares
    sp = host_math(binary, "sqrt", np.array([0.0, -0.0, np.inf, -1.0, np.nan, 5e-324]), tmp_path)
    assert sp[0] == 0.0 and not np.signbit(sp[0]) and sp[1] == 0.0 and np.signbit(sp[1])
    assert np.isinf(sp[2]) and np.isnan(sp[3]) and np.isnan(sp[4]) and sp[5] == 0.0
