// fp64_math.cuh -- FP64 building blocks of the fused kernels (device code; the integer
// exponential and its helpers also compile for the host).
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

namespace gbnll {

// Size of the 2^(j/N) table used by fexp_scaled (held in shared memory by every block).
constexpr int kExpTableBits = 10;
constexpr int kExpTable = 1 << kExpTableBits;

// Scale of the exponential's argument: fexp_scaled(x * kExpArgScale) = exp(x).
constexpr double kExpArgScale = 0x1.71547652b82fep+10;  // N/ln2, N = 1024

// log table after the exp table, for F_j = 1 + j/128, j = 0..127, as integers in the slots'
// bits: ln F_j 2^115 as two 64-bit words (high words, then low words), then 1/F_j 2^63;
// padded to an even count.
constexpr int kLogSteps = 128;
constexpr int kLogTab = 3 * kLogSteps;
constexpr int kLogOffset = kExpTable;
// sin/cos table: |cos| and |sin| of k pi/512 for k = 0..1023 (a full period) as integers
// 2^63 in the slots' bits (pairs), after the log table; the signs follow from k.
constexpr int kTrigSteps = 1024;
constexpr int kTrigOffset = kExpTable + kLogTab;  // even: the (cos, sin) pairs are read as double2
constexpr int kTabDoubles = kTrigOffset + 2 * kTrigSteps;  // one table per translation unit
static_assert(kTrigOffset % 2 == 0, "16-byte aligned (cos, sin) pairs");

// ln 2 2^115 (two 64-bit words), for the logarithm's fixed-point sum; equals
// ln_ratio_q115(2, 1) (checked by the tests).
constexpr uint64_t kLn2Q115Hi = 0x58b90bfbe8e7bull;
constexpr uint64_t kLn2Q115Lo = 0xcd5e4f1d9cc01f98ull;

// Host: ln(a/b) 2^115 for integers 0 < b <= a < 3b, from ln(a/b) = 2 atanh(z), z = (a-b)/(a+b),
// summed as 2 sum z^(2k+1)/(2k+1) in 0.126-bit fixed point (|z| <= 1/2: 64 terms leave less than
// 2^-126; each term is truncated, so the sum is at most 2^-119 low), rounded to 2^-115.  Integer
// arithmetic only, so the tables come out the same on every host.
inline unsigned __int128 ln_ratio_q115(uint64_t a, uint64_t b)
{
    const uint64_t num = a - b, den = a + b;  // z = num/den
    const unsigned __int128 one = (unsigned __int128)1 << 126;
    unsigned __int128 pw = one / den * num + (one % den) * num / den;  // z 2^126
    unsigned __int128 sum = 0;
    for (int k = 0; k < 64 && pw != 0; ++k) {
        sum += pw / (unsigned __int128)(2 * k + 1);
        pw = pw / den * num;  // times z^2 in two steps, each truncated
        pw = pw / den * num;
    }
    return (2 * sum + ((unsigned __int128)1 << 10)) >> 11;  // 2 sum, 2^126 -> 2^115
}

// Host: the values of the device table, all in integer fixed point; the exact zeros and ones
// of sin and cos at multiples of pi/2 are set exactly (long double pi is not pi).
inline void fill_device_tables(double* t)
{
    const long double pi = 3.141592653589793238462643383279502884L;
    for (int j = 0; j < kExpTable; ++j) {  // 2^(j/N) 2^62 as an integer in the slot's bits
        const uint64_t v = (uint64_t)llroundl(ldexpl(exp2l((long double)j / (long double)kExpTable), 62));
        memcpy(t + j, &v, sizeof v);
    }
    for (int j = 0; j < kLogSteps; ++j) {
        const unsigned __int128 l = ln_ratio_q115(kLogSteps + j, kLogSteps);
        const uint64_t words[3] = {(uint64_t)(l >> 64), (uint64_t)l,
                                   (uint64_t)((((unsigned __int128)1 << 70) + (kLogSteps + j) / 2) / (unsigned)(kLogSteps + j))};
        for (int w = 0; w < 3; ++w) memcpy(t + kLogOffset + w * kLogSteps + j, &words[w], sizeof(uint64_t));
    }
    for (int k = 0; k < kTrigSteps; ++k) {
        const long double a = pi * (long double)k / 512.0L;
        uint64_t cs[2];
        cs[0] = (k % 512 == 256) ? 0ull : (k % 512 == 0) ? (1ull << 63) : (uint64_t)llroundl(ldexpl(fabsl(cosl(a)), 63));
        cs[1] = (k % 512 == 0) ? 0ull : (k % 512 == 256) ? (1ull << 63) : (uint64_t)llroundl(ldexpl(fabsl(sinl(a)), 63));
        memcpy(t + kTrigOffset + 2 * k, cs, sizeof cs);
    }
}

// Bit patterns and integer products that compile the same on the host and the device (the
// host build of the exponential below serves its accuracy tests).
__host__ __device__ __forceinline__ uint64_t bits_of(double x)
{
#ifdef __CUDA_ARCH__
    return (uint64_t)__double_as_longlong(x);
#else
    uint64_t b;
    memcpy(&b, &x, sizeof b);
    return b;
#endif
}

__host__ __device__ __forceinline__ double double_of(uint64_t b)
{
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)b);
#else
    double x;
    memcpy(&x, &b, sizeof x);
    return x;
#endif
}

__host__ __device__ __forceinline__ uint32_t umulhi32(uint32_t a, uint32_t b)
{
#ifdef __CUDA_ARCH__
    return __umulhi(a, b);
#else
    return (uint32_t)(((uint64_t)a * b) >> 32);
#endif
}

// floor(a b / 2^64) - d, 0 <= d <= 2: the three upper 32-bit partial products; the lowest one
// and the carries out of the middle column are dropped (3 integer multiplies).
__host__ __device__ __forceinline__ uint64_t umulhi64_trunc(uint64_t a, uint64_t b)
{
    const uint32_t a0 = (uint32_t)a, a1 = (uint32_t)(a >> 32), b0 = (uint32_t)b, b1 = (uint32_t)(b >> 32);
    return (uint64_t)a1 * b1 + ((uint64_t)umulhi32(a1, b0) + umulhi32(a0, b1));
}

// ln 2 in 0.64 fixed point, rounded.
constexpr uint64_t kLn2Q64 = 0xb17217f7d1cf79acull;

// exp(xs / S), S = N/ln2, N = 1024, with Tang's table reduction (P. T. P. Tang, ACM TOMS 15
// (1989) 144) carried out in fixed-point integer arithmetic, so that the exponential costs no
// FP64 instruction (on GB300 an FP64 warp instruction holds its SM sub-partition's FP64 pipe
// for 64 cycles; an integer one a few).  The argument arrives pre-scaled (the kernels fold S
// into the hoisted constants):
//   xs = k + f, k = floor(xs), 0 <= f < 1 (read off the bits of xs exactly),
//   exp(xs / S) = 2^(k >> 10) 2^((k & 1023)/N) exp(x), x = f ln2/N in [0, 6.77e-4),
// exp(x) - 1 = x (1 + x (1/2 + x (1/6 + x/24))) in fixed point, each factor to the precision
// its term needs (the omitted x^5/120 is below 1.2e-18), the table holding 2^(j/N) 2^62 as
// integers.  The result is rounded once from 63 bits: error below 0.52 ulp.  |xs| >= 1.04e6
// (|x| >= 704) returns 0 (xs < 0) or +inf (xs > 0, and NaN).
__host__ __device__ __forceinline__ double fexp_scaled(double xs, const double* __restrict__ tab)
{
    const uint64_t b = bits_of(xs);
    const uint32_t hi = (uint32_t)(b >> 32);
    int sh = 1075 - (int)((hi >> 20) & 0x7ff);  // |xs| = M 2^-sh
    sh = sh > 33 ? sh : 33;                      // reached only by the saturated range
    const uint64_t M = (b & 0x000fffffffffffffull) | (1ull << 52);
    const uint32_t ip = (uint32_t)(M >> 32) >> (sh - 32 < 31 ? sh - 32 : 31);      // floor |xs|
    uint64_t F = sh <= 64 ? M << (64 - sh) : (sh < 128 ? M >> (sh - 64) : 0ull);  // frac |xs|, 2^64
    int k = (int)ip;
    if (hi >> 31) {  // xs = -(ip + frac) = -(ip + 1) + (1 - frac)
        k = -k - (F != 0ull ? 1 : 0);
        F = 0ull - F;
    }
    const uint64_t X = umulhi64_trunc(F, kLn2Q64);                          // x 2^74
    const uint32_t Xh = (uint32_t)(X >> 32);                                // x 2^42
    const uint32_t Q3 = 2863311531u + umulhi32(Xh, 699051u);                // (1/6 + x/24) 2^34
    const uint64_t Q2 = (1ull << 62) + ((uint64_t)umulhi32(Xh, Q3) << 19);  // (1/2 + x q3) 2^63
    const uint64_t Q1 = (1ull << 63) + (umulhi64_trunc(X, Q2) >> 10);       // (1 + x q2) 2^63
    const uint64_t P = umulhi64_trunc(X, Q1);                               // (exp(x) - 1) 2^73
    const uint64_t T = bits_of(tab[k & (kExpTable - 1)]);                   // 2^(j/N) 2^62
    const uint64_t Y = T + (umulhi64_trunc(T, P) >> 9);                     // 2^(j/N) exp(x) 2^62
    const int s = (int)(Y >> 63);                                           // Y < 2^63 but for rounding
    const uint64_t m = (Y + (512ull << s)) >> (10 + s);                     // 53 bits; may carry to 2^53
    double y = double_of(((uint64_t)((k >> kExpTableBits) + 1023 + s) << 52) + (m - (1ull << 52)));
    if ((hi & 0x7fffffff) >= 0x412fbd00u) y = (hi >> 31) ? 0.0 : double_of(0x7ff0000000000000ull);
    return y;
}

// Leading zeros of a 64-bit word (64 for 0).
__host__ __device__ __forceinline__ int clz64(uint64_t v)
{
#ifdef __CUDA_ARCH__
    return __clzll((long long)v);
#else
    return v ? __builtin_clzll(v) : 64;
#endif
}

// a + s t for s = -1 (neg false) or +1 (neg true), in 2^64 arithmetic.
__host__ __device__ __forceinline__ uint64_t add_signed(uint64_t a, uint64_t t, bool neg)
{
    return neg ? a + t : a - t;
}

__host__ __device__ __forceinline__ uint32_t add_signed32(uint32_t a, uint32_t t, bool neg)
{
    return neg ? a + t : a - t;
}

// ln x for a positive normal double x, after Tang's table-driven method (P. T. P. Tang,
// ACM TOMS 16 (1990) 378) carried out in fixed-point integer arithmetic, so that it costs no
// FP64 instruction: x = 2^E m with F = 1 + j/128 (j = 0..127) the table point nearest m (m near
// 2 counts as 2 (m/2) with F = 1), f = m - F exact, u = f/F = f (1/F) with |u| <= 2^-8, and
//   ln x = E ln2 + ln F + u g(u),  g(u) = ln(1 + u)/u = 1 - u/2 + u^2/3 - ... - u^7/8
// (the next term is below 2^-67), summed in a signed 128-bit accumulator at scale 2^115 (ln 2
// and ln F to 2^-115 from the table; u to 2^-70, exact for F = 1, so results near x = 1 keep
// their relative accuracy), then normalised and rounded once: error below 0.51 ulp.  The
// caller guarantees x positive and normal (the kernels check that before taking the log).
__host__ __device__ __forceinline__ double flog(double x, const double* __restrict__ tab)
{
    const uint64_t b = bits_of(x);
    int E = (int)((b >> 52) & 0x7ff) - 1023;
    const uint64_t M = (b & 0x000fffffffffffffull) | (1ull << 52);  // m 2^52
    int j = (int)(((b >> 32) & 0xfffffu) + (1u << 12)) >> 13;       // nearest of 128 steps (0..128)
    int64_t f;                                                       // (m - F) 2^53, |f| <= 2^45
    if (j == kLogSteps) {  // m/2 in [1 - 2^-9, 1): F = 1 at the next exponent
        E += 1;
        j = 0;
        f = (int64_t)M - (1ll << 53);
    } else {
        f = (int64_t)(M << 1) - ((1ll << 53) + ((int64_t)j << 46));
    }
    const bool neg = f < 0;
    const double* lt = tab + kLogOffset;
    // |u| 2^70 (|f| 2^18 (1/F) 2^63 / 2^64); exact for F = 1
    const uint64_t ua = umulhi64_trunc((uint64_t)(neg ? -f : f) << 18, bits_of(lt[2 * kLogSteps + j]));
    // g(u) by Horner from the inside, c_k - u (c_(k+1) - u (...)) with c_k = 1/(k+1); the level
    // of c_k enters g times u^k, so it needs 2^-63 / 2^-8k: 32 bits for c_4..c_6, 64 below
    const uint32_t uh = (uint32_t)(ua >> 31);                                       // |u| 2^39
    uint32_t h = add_signed32(0x24924925u, umulhi32(uh, 0x20000000u) >> 7, neg);    // 1/7 - u/8, 2^32
    h = add_signed32(0x2aaaaaabu, umulhi32(uh, h) >> 7, neg);                        // 1/6 - u (..)
    h = add_signed32(0x33333333u, umulhi32(uh, h) >> 7, neg);                        // 1/5 - u (..)
    uint64_t H = add_signed(0x4000000000000000ull, umulhi64_trunc(ua, (uint64_t)h << 32) >> 6, neg);  // 1/4, 2^64
    H = add_signed(0x5555555555555555ull, umulhi64_trunc(ua, H) >> 6, neg);         // 1/3 - u (..)
    H = add_signed(0x8000000000000000ull, umulhi64_trunc(ua, H) >> 6, neg);         // 1/2 - u (..)
    const uint64_t g = add_signed(1ull << 63, umulhi64_trunc(ua, H) >> 7, neg);     // g(u) 2^63
    // u g(u) 2^115 and the sum
    const unsigned __int128 ug = ((unsigned __int128)ua * g) >> 18;
    const __int128 ln2 = (__int128)(((unsigned __int128)kLn2Q115Hi << 64) | kLn2Q115Lo);
    const __int128 lnF = (__int128)(((unsigned __int128)bits_of(lt[j]) << 64) | bits_of(lt[kLogSteps + j]));
    __int128 acc = (__int128)E * ln2 + lnF;
    acc = neg ? acc - (__int128)ug : acc + (__int128)ug;
    // round to double
    const bool rneg = acc < 0;
    unsigned __int128 a = rneg ? (unsigned __int128)(-acc) : (unsigned __int128)acc;
    const uint64_t ahi = (uint64_t)(a >> 64);
    const int lz = ahi ? clz64(ahi) : 64 + clz64((uint64_t)a);
    if (lz >= 128) return 0.0;  // x = 1
    a <<= lz;
    const uint64_t m = (uint64_t)(((a >> 74) + 1) >> 1);  // 53 bits, rounded; may carry to 2^53
    const uint64_t r = ((uint64_t)(1035 - lz) << 52) + (m - (1ull << 52));
    return double_of(r | (rneg ? 0x8000000000000000ull : 0ull));
}

// sqrt x for x >= 0 in integer arithmetic, so that it costs no FP64 instruction: x = m 2^E with
// E even and m in [1, 4) (in 2.62 fixed point), a single-precision seed y0 ~ 1/sqrt(m) (hardware
// reciprocal square root; on the host the rounded single-precision quotient), the residual
// e = 1 - m y0^2 (|e| < 2^-20), and 1/sqrt(m) = y0 (1 + e/2 + 3e^2/8) + O(e^3), then sqrt(m) =
// m (1/sqrt(m)) and one rounding: error below 0.52 ulp.  +0 and -0 return themselves, +inf
// itself; subnormal x returns 0 and negative x or NaN return NaN.
__host__ __device__ __forceinline__ double fsqrt(double x)
{
    const uint64_t b = bits_of(x);
    const int be = (int)((b >> 52) & 0x7ff);
    const double nan = double_of(0x7ff8000000000000ull);
    if (b >> 63) return (b << 1) == 0 ? x : nan;         // -0 itself; negative x and NaN
    if (be == 0x7ff) return (b << 12) == 0 ? x : nan;    // +inf itself; NaN
    if (be == 0) return double_of(b & 0x8000000000000000ull);  // 0, and subnormals flushed
    const int E = be - 1023;
    const int odd = E & 1;
    const uint64_t MM = ((b & 0x000fffffffffffffull) | (1ull << 52)) << (10 + odd);  // m 2^62, m in [1, 4)
    const uint32_t mf_bits = (uint32_t)(MM >> (39 + odd)) + ((uint32_t)(126 + odd) << 23);  // m to 24 bits as a float
    uint32_t yb;
#ifdef __CUDA_ARCH__
    float y0;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y0) : "f"(__uint_as_float(mf_bits)));
    yb = __float_as_uint(y0);
#else
    float mf;
    memcpy(&mf, &mf_bits, sizeof mf);
    const float y0 = 1.0f / sqrtf(mf);
    memcpy(&yb, &y0, sizeof yb);
#endif
    const int ye = (int)(yb >> 23) - 120;                                        // y0 in (0.49, 1]
    const uint64_t Y0 = (uint64_t)(((yb & 0x7fffffu) | 0x800000u) << (ye > 0 ? ye : 0));  // y0 2^30, exact
    const int64_t e = (int64_t)(1ull << 60) - (int64_t)umulhi64_trunc(MM, (Y0 * Y0) << 2);  // (1 - m y0^2) 2^60
    const int64_t eh = e >> 20;                                                  // e 2^40
    const int64_t t = (e >> 1) + ((3 * (eh * eh)) >> 23);                        // (e/2 + 3e^2/8) 2^60
    const uint64_t Y = (Y0 << 32) + (uint64_t)(int64_t)(((__int128)t * (int64_t)Y0) >> 28);  // 1/sqrt(m) 2^62
    const uint64_t S = (uint64_t)(((unsigned __int128)MM * Y) >> 62);           // sqrt(m) 2^62, in [2^62, 2^63)
    const uint64_t m53 = ((S >> 9) + 1) >> 1;                                    // 53 bits; may carry to 2^53
    return double_of(((uint64_t)((E - odd) / 2 + 1023) << 52) + (m53 - (1ull << 52)));
}

// pi/512 2^116 (two 64-bit words) and 512/pi 2^55, for the sine and cosine's reduction.
constexpr uint64_t kPi512Q116Hi = 0x1921fb54442dull;
constexpr uint64_t kPi512Q116Lo = 0x18469898cc51701cull;
constexpr uint64_t k512PiQ55 = 0x517cc1b727220a95ull;

// v 2^e2 as a double, rounded from v's leading 64 bits (v > 0, result in the normal range).
__host__ __device__ __forceinline__ double u64_scaled_to_double(uint64_t v, int e2)
{
    const int lz = clz64(v);
    const uint64_t m = (((v << lz) >> 10) + 1) >> 1;  // 53 bits, rounded; may carry to 2^53
    return double_of(((uint64_t)(63 - lz + e2 + 1023) << 52) + (m - (1ull << 52)));
}

// A signed 128-bit fixed-point value a 2^-126 as a double (|a| <= 2^127 - 1).
__host__ __device__ __forceinline__ double q126_to_double(__int128 a)
{
    if (a == 0) return 0.0;
    const bool neg = a < 0;
    const unsigned __int128 u = neg ? (unsigned __int128)(-a) : (unsigned __int128)a;
    const uint64_t hi = (uint64_t)(u >> 64);
    const int lz = hi ? clz64(hi) : 64 + clz64((uint64_t)u);
    const double r = u64_scaled_to_double((uint64_t)((u << lz) >> 64), -62 - lz);  // the leading 64 bits
    return neg ? -r : r;
}

// sin x and cos x for |x| < 1024 (NaN beyond), from the classical table method (Cody-Waite
// style reduction to x = k pi/512 + r, W. J. Cody and W. Waite, Software Manual for the
// Elementary Functions, 1980) carried out in fixed-point integer arithmetic, so that it costs
// no FP64 instruction: |x| 2^116 read off the bits exactly, k = round(512 |x|/pi), r = |x| -
// k pi/512 in a signed 128-bit word (pi/512 to 2^-116), |r| <= pi/1024;
//   sin r = r (1 - r^2/6 + r^4/120 - r^6/5040),  1 - cos r = (r^2/2)(1 - r^2/12 + r^4/360)
// (the next terms are below 2^-62 relative); then
//   sin |x| = S (1 - (1 - cos r)) + C sin r,  cos |x| = C (1 - (1 - cos r)) - S sin r
// summed exactly in 128-bit words at 2^-126 from the table's |cos|, |sin| of k pi/512 (2^-63)
// and rounded once.  Where the table's S (or C) is exactly 0 the result is +-sin r itself,
// which keeps its relative accuracy (sin x near 0 and +-pi, cos x near +-pi/2).  |x| < 2^-26
// returns sin x = x, cos x = 1 (correctly rounded there).  Error below 1 ulp.
__host__ __device__ __forceinline__ void fsincos_pi(double x, const double* __restrict__ trig, double& s, double& c)
{
    const uint64_t b = bits_of(x);
    const int be = (int)((b >> 52) & 0x7ff);
    if (be < 1023 - 26) {
        s = x;
        c = 1.0;
        return;
    }
    if (be >= 1023 + 10) {
        s = c = double_of(0x7ff8000000000000ull);
        return;
    }
    const uint64_t M = (b & 0x000fffffffffffffull) | (1ull << 52);
    const unsigned __int128 XF = (unsigned __int128)M << (be - 1023 + 64);                  // |x| 2^116
    const int k = (int)((umulhi64_trunc((uint64_t)(XF >> 64), k512PiQ55) + (1ull << 42)) >> 43);  // round(512|x|/pi)
    const unsigned __int128 P = ((unsigned __int128)kPi512Q116Hi << 64) | kPi512Q116Lo;
    const __int128 R = (__int128)(XF - (unsigned __int128)k * P);                          // r 2^116
    const bool rneg = R < 0;
    const unsigned __int128 Ra = rneg ? (unsigned __int128)(-R) : (unsigned __int128)R;
    const uint64_t Rh = (uint64_t)(Ra >> 52);                                                // |r| 2^64
    const uint64_t r2 = umulhi64_trunc(Rh, Rh);                                              // r^2 2^64
    uint64_t h = 0x0222222222222222ull - umulhi64_trunc(r2, 0x000d00d00d00d00dull);          // 1/120 - r^2/5040
    h = 0x2aaaaaaaaaaaaaabull - umulhi64_trunc(r2, h);                                       // 1/6 - r^2 (..)
    const uint64_t gs = (1ull << 63) - (umulhi64_trunc(r2, h) >> 1);                         // sin r / r, 2^63
    const uint64_t hc = 0x1555555555555555ull - umulhi64_trunc(r2, 0x00b60b60b60b60b6ull);   // 1/12 - r^2/360
    const uint64_t gc = (1ull << 63) - (umulhi64_trunc(r2, hc) >> 1);                        // 2(1 - cos r)/r^2, 2^63
    const uint64_t cm = umulhi64_trunc(r2, gc) >> 1;                                         // 1 - cos r, 2^63
    // |sin r| = sr 2^(-51 - lz): |r| normalised (relative accuracy), times sin r / r
    const uint64_t rhi = (uint64_t)(Ra >> 64);
    const int lz = rhi ? clz64(rhi) : 64 + clz64((uint64_t)Ra);
    const uint64_t sr = lz < 128 ? umulhi64_trunc((uint64_t)((Ra << (lz & 127)) >> 64), gs) : 0ull;
    const uint64_t sr63 = lz < 76 ? sr >> (lz - 12) : 0ull;  // |sin r| 2^63 (lz >= 20; below 2^-63 it is 0)
    // table: |cos|, |sin| of j pi/512 with their signs from j
    const int j = k & (kTrigSteps - 1);
    const uint64_t Cm = bits_of(trig[2 * j]), Sm = bits_of(trig[2 * j + 1]);
    const bool cneg = j > 256 && j < 768, sneg = j > 512;
    const unsigned __int128 pc = (unsigned __int128)Cm * ((1ull << 63) - cm), ps = (unsigned __int128)Sm * ((1ull << 63) - cm);
    const unsigned __int128 qc = (unsigned __int128)Cm * sr63, qs = (unsigned __int128)Sm * sr63;
    // sin |x| = S(1 - cm) + C sin r, cos |x| = C(1 - cm) - S sin r, at 2^-126
    const __int128 as = (sneg ? -(__int128)ps : (__int128)ps) + ((cneg != rneg) ? -(__int128)qc : (__int128)qc);
    const __int128 ac = (cneg ? -(__int128)pc : (__int128)pc) - ((sneg != rneg) ? -(__int128)qs : (__int128)qs);
    double sv = q126_to_double(as), cv = q126_to_double(ac);
    if (lz < 128) {  // a zero table entry: the result is +-sin r, to its relative accuracy
        const double sin_r = u64_scaled_to_double(sr, -51 - lz);
        if (Sm == 0) sv = (cneg != rneg) ? -sin_r : sin_r;
        if (Cm == 0) cv = (sneg != rneg) ? sin_r : -sin_r;
    } else {
        if (Sm == 0) sv = 0.0;
        if (Cm == 0) cv = 0.0;
    }
    s = (b >> 63) ? -sv : sv;
    c = cv;
}

// The hardware reciprocal approximation alone (diagnostics: its accuracy decides how many
// correction terms the kernels need).
__device__ __forceinline__ double frcp_approx(double x)
{
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    return y;
}

// 1/x for a finite normal double x (either sign) in integer arithmetic, so that it costs no FP64
// instruction: x = +-m 2^E, m in [1, 2); a single-precision seed y0 ~ 1/m (hardware reciprocal
// of m's leading 24 bits; on the host, the rounded single-precision quotient), the residual
// e = 1 - m y0 exactly (|e| < 2^-21: the 53 x 31-bit product taken modulo 2^64), and
//   1/m = y0 / (1 - e) = y0 (1 + e + e^2) + y0 e^3 / (1 - e),
// the last term below 2^-62 of the result.  One rounding from 62 bits: error below 0.51 ulp.
// |x| >= 2^1022 returns +-0 (the result would be subnormal), subnormal x and 0 return +-inf.
__host__ __device__ __forceinline__ double frcp(double x)
{
    const uint64_t b = bits_of(x);
    const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
    const int be = (int)((hi >> 20) & 0x7ff);
    const uint64_t M = (b & 0x000fffffffffffffull) | (1ull << 52);  // m 2^52
    const uint32_t mf_bits = 0x3f800000u | ((hi & 0xfffffu) << 3) | (lo >> 29);  // m to 24 bits
    uint32_t yb;
#ifdef __CUDA_ARCH__
    float y0;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y0) : "f"(__uint_as_float(mf_bits)));
    yb = __float_as_uint(y0);
#else
    float mf;
    memcpy(&mf, &mf_bits, sizeof mf);
    const float y0 = 1.0f / mf;
    memcpy(&yb, &y0, sizeof yb);
#endif
    const int ye = (int)(yb >> 23) - 120;                                  // y0 in (0.49, 1]
    const uint32_t Y0 = ((yb & 0x7fffffu) | 0x800000u) << (ye > 0 ? ye : 0);  // y0 2^30, exact
    const int64_t E = (int64_t)(0ull - M * (uint64_t)Y0);                  // e 2^82 (2^82 = 0 mod 2^64)
    const int32_t Eh = (int32_t)(E >> 32);                                 // e 2^50
    const int64_t t = E + (((int64_t)Eh * Eh) >> 18);                      // (e + e^2) 2^82
    const int64_t u = (int64_t)(int32_t)(t >> 32) * (int64_t)Y0 + umulhi32((uint32_t)t, Y0);  // y0 (e + e^2) 2^80
    const uint64_t Y = ((uint64_t)Y0 << 32) + (uint64_t)(u >> 18);         // 1/m 2^62, in (2^61, 2^62]
    const int s = (int)((Y >> 62) & 1);
    const uint64_t m53 = (Y + (256ull << s)) >> (9 + s);                   // 53 bits; may carry to 2^53
    const uint64_t sign = b & 0x8000000000000000ull;
    uint64_t r = sign | ((((uint64_t)(2045 - be + s)) << 52) + (m53 - (1ull << 52)));
    if (be >= 2045) r = sign;                                              // |1/x| below the normal range
    if (be == 0) r = sign | 0x7ff0000000000000ull;
    return double_of(r);
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

// Running product with the binary exponent split off, in integer arithmetic (no FP64
// instruction): value = m 2^(e - 63), m in [2^63, 2^64) (a 64-bit mantissa).  Each factor's
// mantissa multiplies in with the three upper partial products (umulhi64_trunc: at most
// 2^-62 below the exact product, far below a double rounding), its exponent adds to e.
struct LogProd {
    uint64_t m;
    int e;
};

__host__ __device__ __forceinline__ LogProd logprod_one() { return LogProd{1ull << 63, 0}; }

// Multiply by 2^ex q/2^63 for a mantissa q in [2^63, 2^64).
__host__ __device__ __forceinline__ void logprod_mul_mant(LogProd& lp, uint64_t q, int ex)
{
    const uint64_t p = umulhi64_trunc(lp.m, q);  // (m/2^63)(q/2^63) 2^62, in [2^62, 2^64)
    const int top = (int)(p >> 63);
    lp.m = top ? p : p << 1;
    lp.e += ex + top;
}

// Multiply by a positive normal double x (integer pipe only).
__host__ __device__ __forceinline__ void logprod_mul(LogProd& lp, double x)
{
    const uint64_t b = bits_of(x);
    logprod_mul_mant(lp, ((b & 0x000fffffffffffffull) | (1ull << 52)) << 11, (int)((b >> 52) & 0x7ff) - 1023);
}

// Product of two running products.
__host__ __device__ __forceinline__ LogProd logprod_combine(const LogProd& a, const LogProd& b)
{
    LogProd r{a.m, a.e};
    logprod_mul_mant(r, b.m, b.e);
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

// ln of the product: ln(m 2^-63) + e ln2, the mantissa rounded to a double in [1, 2].
__host__ __device__ __forceinline__ double logprod_value(const LogProd& lp)
{
    const double kLn2hi = 0x1.62e42ff000000p-1, kLn2lo = -0x1.718432a1b0e26p-35;
    const double md = double_of((1023ull << 52) + (((lp.m >> 10) + 1) >> 1) - (1ull << 52));
    double e = (double)lp.e;
    return fma(e, kLn2hi, fma(e, kLn2lo, log(md)));
}

}  // namespace gbnll
