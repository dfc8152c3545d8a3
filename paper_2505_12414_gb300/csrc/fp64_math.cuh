// fp64_math.cuh -- FP64 building blocks of the fused kernels (device code only).
#pragma once

#include <cuda_runtime.h>
#include <math.h>

namespace gbnll {

// Size of the 2^(j/N) table used by fexp (held in shared memory by every block).
constexpr int kExpTableBits = 10;
constexpr int kExpTable = 1 << kExpTableBits;

// Scale of the exponential's argument: fexp_scaled(x * kExpArgScale) = exp(x).
constexpr double kExpArgScale = 0x1.71547652b82fep+10;  // N/ln2, N = 1024

// log table after the exp table: for F_j = 1 + j/128, j = 0..128, ln F_j split into a head
// (a multiple of 2^-42) and a tail, and 1/F_j; padded to an even count.
constexpr int kLogSteps = 128;
constexpr int kLogTab = 3 * (kLogSteps + 1) + 1;
constexpr int kLogOffset = kExpTable;
// sin/cos table: (cos, sin) of k pi/512 for k = 0..1023 (a full period), after the log table.
constexpr int kTrigSteps = 1024;
constexpr int kTrigOffset = kExpTable + kLogTab;  // even: the (cos, sin) pairs are read as double2
constexpr int kTabDoubles = kTrigOffset + 2 * kTrigSteps;  // one table per translation unit
static_assert(kTrigOffset % 2 == 0, "16-byte aligned (cos, sin) pairs");

// ln 2 split for the logarithm: head with 42 significant bits (e ln2_head is exact for any
// binary exponent e of a double) and the rest.
constexpr double kLn2Head = 0x1.62e42fefa3800p-1;
constexpr double kLn2Tail = 0x1.ef35793c76730p-45;

// Host: the values of the device table, rounded from long double; the exact zeros of sin and
// cos at multiples of pi/2 are set exactly (long double pi is not pi).
inline void fill_device_tables(double* t)
{
    const long double pi = 3.141592653589793238462643383279502884L;
    for (int j = 0; j < kExpTable; ++j) t[j] = (double)exp2l((long double)j / (long double)kExpTable);
    for (int j = 0; j <= kLogSteps; ++j) {
        const long double F = 1.0L + (long double)j / (long double)kLogSteps;
        const long double l = logl(F);
        const double head = (double)(nearbyintl(ldexpl(l, 42)) / 4398046511104.0L);  // multiple of 2^-42
        t[kLogOffset + j] = head;
        t[kLogOffset + (kLogSteps + 1) + j] = (double)(l - (long double)head);
        t[kLogOffset + 2 * (kLogSteps + 1) + j] = (double)(1.0L / F);
    }
    t[kLogOffset + kLogTab - 1] = 0.0;
    for (int k = 0; k < kTrigSteps; ++k) {
        const long double a = pi * (long double)k / 512.0L;
        t[kTrigOffset + 2 * k] = (k % 512 == 256) ? 0.0 : (double)cosl(a);
        t[kTrigOffset + 2 * k + 1] = (k % 512 == 0) ? 0.0 : (double)sinl(a);
    }
}

// exp(xs / S), S = N/ln2, after Tang's table-driven method (P. T. P. Tang, ACM TOMS 15
// (1989) 144), N = 1024.  The argument arrives pre-scaled (the kernels fold S into the
// hoisted constants), so the reduction is exact without a split constant:
//   xs = N q + j + r,  |r| <= 1/2,  exp(xs / S) = 2^q 2^(j/N) exp(r ln2/N).
// exp(r ln2/N) - 1 is a cubic in r obtained by Chebyshev economisation of the degree-4
// Taylor polynomial on [-ln2/2N, ln2/2N] (the r^4 term replaced by its best lower-degree
// approximation), with the powers of ln2/N folded into the coefficients; truncation error
// below 0.62 ulp of 1.  |xs| >= 1.04e6 (|x| >= 704) returns 0 (xs < 0) or +inf (xs > 0,
// and NaN).  7 FP64 instructions on the fast path.
__device__ __forceinline__ double fexp_scaled(double xs, const double* __restrict__ tab)
{
    const double kMagic = 0x1.8p52;  // 1.5 * 2^52: xs + kMagic rounds xs to an integer
    const double C1 = 0x1.62e42fefa39efp-11;  // ln2/N
    const double C2 = 0x1.ebfbe046f706bp-23;  // (1/2 + h^2/24) (ln2/N)^2, h = ln2/2N
    const double C3 = 0x1.c6b08d704a0c0p-35;  // (1/6) (ln2/N)^3
    const double C0 = -0x1.3b2ab6fba4e77p-54;  // -h^4/192
    double kd = xs + kMagic;
    int k = __double2loint(kd);
    double kf = kd - kMagic;
    double r = xs - kf;  // exact
    double T = tab[k & (kExpTable - 1)];
    double p = fma(r, C3, C2);
    p = fma(p, r, C1);
    p = fma(p, r, C0);
    double y = fma(T, p, T);
    int hi = __double2hiint(y) + ((k >> kExpTableBits) << 20);
    y = __hiloint2double(hi, __double2loint(y));
    int xhi = __double2hiint(xs);
    if ((xhi & 0x7fffffff) >= 0x412fbd00) y = (xhi < 0) ? 0.0 : __longlong_as_double(0x7ff0000000000000ll);
    return y;
}

// ln x for a positive normal double x, after Tang's table-driven method (P. T. P. Tang,
// ACM TOMS 16 (1990) 378): x = 2^e m, m in [1, 2), F = 1 + j/128 the table point nearest m
// (j from the top mantissa bits with integer instructions), f = m - F (exact, |f| <= 1/256),
// u = f / F = f (1/F) with |u| <= 2^-8, and
//   ln x = (e ln2_head + ln F_head) + (e ln2_tail + ln F_tail + ln(1 + u)),
// the first sum exact (both heads are multiples of 2^-42), ln(1 + u) from its Taylor series
// through u^7 (the next term is below 2e-18 relative).  14 FP64 instructions.  The caller
// guarantees x positive and normal (the kernels check that before taking the logarithm).
__device__ __forceinline__ double flog(double x, const double* __restrict__ tab)
{
    const int hi = __double2hiint(x);
    const int mh = hi & 0x000fffff;
    const int j = (mh + (1 << 12)) >> 13;                      // nearest of 128 steps (0..128)
    const double m = __hiloint2double(mh | 0x3ff00000, __double2loint(x));
    const double F = __hiloint2double(0x3ff00000 + (j << 13), 0);
    const double ed = (double)((hi >> 20) - 1023);
    const double* lt = tab + kLogOffset;
    const double u = (m - F) * lt[2 * (kLogSteps + 1) + j];
    const double q = u * u;
    double t = fma(u, 1.0 / 7.0, -1.0 / 6.0);
    t = fma(u, t, 1.0 / 5.0);
    t = fma(u, t, -1.0 / 4.0);
    t = fma(u, t, 1.0 / 3.0);
    t = fma(u, t, -1.0 / 2.0);
    const double p = fma(q, t, u);
    const double head = fma(ed, kLn2Head, lt[j]);
    const double tail = fma(ed, kLn2Tail, lt[(kLogSteps + 1) + j]);
    return head + (tail + p);
}

// sin x and cos x for |x| <= pi (any x is safe; accuracy degrades slowly beyond), from the
// classical table method with Cody-Waite reduction (W. J. Cody and W. Waite, Software Manual
// for the Elementary Functions, 1980): x = k pi/512 + r with k = rint(512 x/pi) and
// |r| <= pi/1024, the reduction x - k (P1 + P2) done with two FMAs (P1 + P2 = pi/512 to ~106
// bits, so r carries at most one rounding); sin r and cos r - 1 from their Taylor series
// through r^5 and r^4 (the next terms are below 2e-19 and 2e-18 relative at |r| = pi/1024);
// then
//   sin x = S + (S (cos r - 1) + C sin r),  cos x = C + (C (cos r - 1) - S sin r)
// with (C, S) = (cos, sin)(k pi/512) from the table.  15 FP64 instructions, no branch.
__device__ __forceinline__ void fsincos_pi(double x, const double* __restrict__ trig, double& s, double& c)
{
    const double kMagic = 0x1.8p52;
    const double kScale = 0x1.45f306dc9c883p+7;  // 512/pi
    const double P1 = 0x1.921fb54442d18p-8;      // pi/512, leading 53 bits
    const double P2 = 0x1.1a62633145c07p-62;     // pi/512 - P1
    double kd = fma(x, kScale, kMagic);
    int k = __double2loint(kd);
    double kf = kd - kMagic;
    double r = fma(-kf, P1, x);
    r = fma(-kf, P2, r);
    double r2 = r * r;
    double sr = fma(r * r2, fma(r2, 1.0 / 120.0, -1.0 / 6.0), r);
    double cm = r2 * fma(r2, 1.0 / 24.0, -0.5);  // cos r - 1
    const double2 cs = reinterpret_cast<const double2*>(trig)[k & (kTrigSteps - 1)];
    s = fma(cs.y, cm, fma(cs.x, sr, cs.y));
    c = fma(cs.x, cm, fma(-cs.y, sr, cs.x));
}

// The hardware reciprocal approximation alone (diagnostics: its accuracy decides how many
// correction terms the kernels need).
__device__ __forceinline__ double frcp_approx(double x)
{
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    return y;
}

// 1/x from the hardware approximation plus one cubic correction: with e = 1 - x y0,
// 1/x = y0 / (1 - e) = y0 (1 + e + e^2 + ...).  3 FP64 instructions + 1 MUFU.
__device__ __forceinline__ double frcp(double x)
{
    const double y = frcp_approx(x);
    double e = fma(-x, y, 1.0);
    double t = fma(e, e, e);
    return fma(y, t, y);
}

// 1/x from the hardware approximation plus one Newton step y0 (1 + e): relative error e^2.
// 2 FP64 instructions + 1 MUFU.
__device__ __forceinline__ double frcp_newton(double x)
{
    const double y = frcp_approx(x);
    const double e = fma(-x, y, 1.0);
    return fma(y, e, y);
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

// Product of two running products (exact exponent bookkeeping, one rounding).
__device__ __forceinline__ LogProd logprod_combine(const LogProd& a, const LogProd& b)
{
    LogProd r{a.m, a.e + b.e};
    logprod_mul(r, b.m);
    return r;
}

// Product over the warp (butterfly, every lane ends with the same value).
__device__ __forceinline__ LogProd logprod_warp(LogProd lp)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        LogProd other{__shfl_xor_sync(0xffffffffu, lp.m, o), __shfl_xor_sync(0xffffffffu, lp.e, o)};
        lp = logprod_combine(lp, other);
    }
    return lp;
}

__device__ __forceinline__ double logprod_value(const LogProd& lp)
{
    const double kLn2hi = 0x1.62e42ff000000p-1, kLn2lo = -0x1.718432a1b0e26p-35;
    double e = (double)lp.e;
    return fma(e, kLn2hi, fma(e, kLn2lo, log(lp.m)));
}

}  // namespace gbnll
