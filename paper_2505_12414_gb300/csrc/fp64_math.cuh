// fp64_math.cuh -- FP64 building blocks of the fused kernels (device code only).
#pragma once

#include <cuda_runtime.h>

namespace gbnll {

// exp(x) after Tang's table-driven method: x = (256 q + j) ln2/256 + r, |r| <= ln2/512,
// exp(x) = 2^q 2^(j/256) exp(r), exp(r) - 1 = r (1 + r/2 + r^2/6 + r^3/24) (truncation
// below 0.35 ulp).  The reduction constant ln2/256 is split so that k * L_hi is exact.
// |x| >= 707 returns 0 (x < 0) or +inf (x > 0, also NaN); results below 2^-1020 are
// flushed to zero.  9 FP64 instructions on the fast path.
__device__ __forceinline__ double fexp(double x, const double* __restrict__ tab)
{
    const double kInvL = 0x1.71547652b82fep+8;   // 256/ln2
    const double kMagic = 0x1.8p52;              // 1.5 * 2^52: rounds to an integer in the low word
    const double kLhi = 0x1.62e42ff000000p-9;    // ln2/256, 29 significant bits
    const double kLlo = -0x1.718432a1b0e26p-43;  // ln2/256 - kLhi
    double kd = fma(x, kInvL, kMagic);
    int k = __double2loint(kd);
    double kf = kd - kMagic;
    double r = fma(kf, -kLhi, x);
    r = fma(kf, -kLlo, r);
    double t = fma(r, 1.0 / 24.0, 1.0 / 6.0);
    t = fma(t, r, 0.5);
    t = fma(t, r, 1.0);
    double p = t * r;
    double T = tab[k & 255];
    double y = fma(T, p, T);
    int hi = __double2hiint(y) + ((k >> 8) << 20);
    y = __hiloint2double(hi, __double2loint(y));
    int xhi = __double2hiint(x);
    if ((xhi & 0x7fffffff) >= 0x40861800) y = (xhi < 0) ? 0.0 : __longlong_as_double(0x7ff0000000000000ll);
    return y;
}

// 1/x from the hardware approximation plus one cubic correction: with e = 1 - x y0,
// 1/x = y0 / (1 - e) = y0 (1 + e + e^2 + ...).  3 FP64 instructions + 1 MUFU.
__device__ __forceinline__ double frcp(double x)
{
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    double e = fma(-x, y, 1.0);
    double t = fma(e, e, e);
    return fma(y, t, y);
}

// 1 if x is not a positive normal finite double (integer pipe only).
__device__ __forceinline__ int not_positive_normal(double x)
{
    return (unsigned)(__double2hiint(x) - 0x00100000) >= 0x7fe00000u;
}

// Running product with the binary exponent split off: value = m * 2^e, m in [1, 2).
struct LogProd {
    double m;
    int e;
};

__device__ __forceinline__ void logprod_mul(LogProd& lp, double x)
{
    double q = lp.m * x;
    int hi = __double2hiint(q);
    lp.e += (hi >> 20) - 1023;
    lp.m = __hiloint2double((hi & 0x000fffff) | 0x3ff00000, __double2loint(q));
}

__device__ __forceinline__ double logprod_value(const LogProd& lp)
{
    const double kLn2hi = 0x1.62e42ff000000p-1, kLn2lo = -0x1.718432a1b0e26p-35;
    double e = (double)lp.e;
    return fma(e, kLn2hi, fma(e, kLn2lo, log(lp.m)));
}

}  // namespace gbnll
