// hess_device.cuh -- the Hessian pass shared by the single-sample kernel (hess.cu) and the
// batched one (batch.cu): column layout of the staged event tile, per-event staging, slot
// sums over a tile, and the assembly of NLL, gradient, H and W from the slot sums (host and
// device).  The mathematics is described at the top of hess.cu.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "fp64_math.cuh"
#include "gbnll_internal.h"
#include "nll_device.cuh"

namespace gbnll {

// Parameter-only terms the assembly needs beyond the slot sums.
struct HessTerms {
    double alpha, f, sigma, b0;
    double d2lnN1[3];     // d^2 ln N1 / (dmu dmu, dmu dsigma, dsigma dsigma)
    double d2lnN2t_dal2;  // d^2 ln Ntilde2 / dalpha^2
    double dlnNc_dc2[3];  // d ln Nc_j / dc2_j
};

// Column layout of the staged tile.  Without weights the weighted scores are the scores.
template <int KIND, bool W>
struct HCols {
    static constexpr int NP = KIND == kMass1D ? 4 : 18;
    static constexpr int S = 0;             // scores s_a
    static constexpr int WS = W ? NP : 0;   // w s_a
    static constexpr int X = W ? 2 * NP : NP;
    static constexpr int WPBPHI_MU = X;     // w pb phi_mu
    static constexpr int WPBPHI_SIG = X + 1;
    static constexpr int WPSPHI_AL = X + 2; // w ps phi_alpha
    static constexpr int WPS = X + 3;
    static constexpr int WPB = X + 4;
    static constexpr int D = X + 5;         // m - mu
    static constexpr int WPSD = X + 6;      // w ps d
    static constexpr int WLNP = X + 7;      // w ln Ptilde
    static constexpr int BAD = X + 8;       // 1 for an event with a non-positive density
    static constexpr int ONE = X + 9;
    static constexpr int CROSS = X + 10;    // 4D: pb phi_(j,p) phi_(k,q), j < k (12)
    static constexpr int NC = CROSS + (KIND == kMass1D ? 0 : 12);
};

// ------------------------------------------------------------------------------------
// Device: staging of one event
// ------------------------------------------------------------------------------------
template <int KIND, int VAR, bool W>
__device__ __forceinline__ void stage_event(const HEv& a, const HConst& c, int64_t e, double* z, int t,
                                            const double* tab, LogProd& lp)
{
    using L = HCols<KIND, W>;
    const bool in = e < a.n;
    const int64_t ei = in ? e : 0;
    auto put = [&](int k, double v) { z[k * kHessThreads + t] = v; };
    const double m = in ? __ldg(a.col[kColM] + ei) : c.mu;
    const double w = W ? (in ? __ldg(a.w + ei) : 0.0) : 1.0;
    const double d = m - c.mu;
    // f G e^{-alpha (m - ma)}; the constants carry the exponential's argument scale
    const double E = fexp_scaled(fma(d, fma(c.neg_b0s, d, c.neg_als), c.k0s), tab);
    const double phmu = fma(2.0 * c.b0, d, -c.dlnN1_dmu);
    const double phsig = fma(fma(2.0 * c.b0 * d, d, -1.0), c.inv_sigma, -c.dlnN1_dsig);
    const double phal = d + c.mu_ma - c.dlnN2t_dal;
    double P, ps, pb, r;
    if (KIND == kMass1D) {
        P = E + c.b2;
        r = frcp(P);
        ps = E * r;
        pb = c.b2 * r;
        put(L::S + 0, ps * phmu);
        put(L::S + 1, ps * phsig);
        put(L::S + 2, pb * phal);
        put(L::S + 3, ps * c.inv_f - pb * c.inv_1mf);
    } else {
        double h[9], t2l, t2k, xp, t2p, xl, xk;
        if (VAR == kVarPrecompute) {
#pragma unroll
            for (int j = 0; j < 9; ++j) h[j] = __ldg(a.col[kColH0 + j] + ei);
            xl = __ldg(a.col[kColCtl] + ei);
            xk = __ldg(a.col[kColCtk] + ei);
            t2l = __ldg(a.col[kColT2l] + ei);
            t2k = __ldg(a.col[kColT2k] + ei);
            xp = __ldg(a.col[kColXp] + ei);
            t2p = __ldg(a.col[kColT2p] + ei);
        } else {
            xl = __ldg(a.col[kColCtl] + ei);
            xk = __ldg(a.col[kColCtk] + ei);
            angular_basis(xl, xk, __ldg(a.col[kColPhi] + ei), h, t2l, t2k, xp, t2p, tab + kTrigOffset);
        }
        double A = fma(c.ang[0], h[1], h[0]);
#pragma unroll
        for (int k = 1; k < 8; ++k) A = fma(c.ang[k], h[k + 1], A);
        const double x[3] = {xl, xk, xp}, T2[3] = {t2l, t2k, t2p};
        double Cb[3], nu2[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            Cb[j] = fma(c.c1[j], x[j], fma(c.c2[j], T2[j], 1.0));
            nu2[j] = fma(-c.dl[j], Cb[j], T2[j]);  // numerator of phi_(j,c2): T2 - dl Cbar
        }
        const double O[3] = {Cb[1] * Cb[2], Cb[0] * Cb[2], Cb[0] * Cb[1]};  // the other two factors
        const double sig = A * E, bg = c.b2 * (O[2] * Cb[2]);
        P = sig + bg;
        r = frcp(P);
        ps = sig * r;
        pb = bg * r;
        const double rE = r * E, Q = r * c.b2;
        put(L::S + 0, ps * phmu);
        put(L::S + 1, ps * phsig);
#pragma unroll
        for (int k = 0; k < 8; ++k) put(L::S + 2 + k, rE * h[k + 1]);
        put(L::S + 10, pb * phal);
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const double QO = Q * O[j];
            put(L::S + 11 + 2 * j, QO * x[j]);
            put(L::S + 12 + 2 * j, QO * nu2[j]);
        }
        put(L::S + 17, ps * c.inv_f - pb * c.inv_1mf);
        // pb phi_(j,p) phi_(k,q) = Q nu_(j,p) nu_(k,q) Cbar_l (l the third observable)
        const int jj[3] = {0, 0, 1}, kk[3] = {1, 2, 2}, ll[3] = {2, 1, 0};
#pragma unroll
        for (int q3 = 0; q3 < 3; ++q3) {
            const int j = jj[q3], k = kk[q3];
            const double QC = Q * Cb[ll[q3]];
            const double qn[2] = {QC * x[j], QC * nu2[j]}, nk[2] = {x[k], nu2[k]};
#pragma unroll
            for (int p = 0; p < 2; ++p)
#pragma unroll
                for (int q = 0; q < 2; ++q) put(L::CROSS + 4 * q3 + 2 * p + q, qn[p] * nk[q]);
        }
    }
    if (W) {
#pragma unroll
        for (int k = 0; k < L::NP; ++k) put(L::WS + k, w * z[(L::S + k) * kHessThreads + t]);
    }
    const double wps = w * ps, wpb = w * pb;
    put(L::WPBPHI_MU, wpb * phmu);
    put(L::WPBPHI_SIG, wpb * phsig);
    put(L::WPSPHI_AL, wps * phal);
    put(L::WPS, wps);
    put(L::WPB, wpb);
    put(L::D, d);
    put(L::WPSD, wps * d);
    put(L::ONE, 1.0);
    const bool ok = in && !not_positive_normal(P);
    if (W)
        put(L::WLNP, ok ? w * flog(P, tab) : 0.0);
    else  // one logarithm per thread at the end (running product, exponent split off)
        logprod_mul(lp, ok ? P : 1.0);
    if (ok) {
        if (!W) put(L::WLNP, 0.0);
        put(L::BAD, 0.0);
    } else {  // no contribution; count it if it is a real event
#pragma unroll 1
        for (int k = 0; k < L::NC; ++k) put(k, 0.0);
        put(L::ONE, 1.0);
        put(L::BAD, in ? 1.0 : 0.0);
    }
}

// Slot sums of one tile: thread t owns slots t, t + 128, t + 256 (NPS of them).
template <int NPS>
__device__ __forceinline__ void tile_slots(const double* z, const int (&ci)[3], const int (&cj)[3], double (&acc)[3],
                                           int lane)
{
    const double* zi[NPS];
    const double* zj[NPS];
#pragma unroll
    for (int k = 0; k < NPS; ++k) {
        zi[k] = z + ci[k] * kHessThreads;
        zj[k] = z + cj[k] * kHessThreads;
    }
#pragma unroll 4
    for (int e = 0; e < kHessThreads; ++e) {
        const int i = (e + lane) & (kHessThreads - 1);
#pragma unroll
        for (int k = 0; k < NPS; ++k) acc[k] = fma(zi[k][i], zj[k][i], acc[k]);
    }
}

// ------------------------------------------------------------------------------------
// Device: single-precision staging, for start matrices only (a quasi-Newton start matrix is a
// preconditioner, so its precision does not reach the fitted minimum; FP32 runs at many times
// the FP64 rate).  Same columns as stage_event; the column of ln P is left 0 (a start matrix
// needs H and the gradient, not the NLL).
// ------------------------------------------------------------------------------------
struct HConst32 {
    double mu_d;  // m - mu is formed in double precision (one FP64 add per event), then rounded
    float mu, b0, neg_b0s, neg_als, k0s, b2, inv_sigma;
    float dlnN1_dmu, dlnN1_dsig, mu_ma, dlnN2t_dal, inv_f, inv_1mf;
    float ang[8];
    float c1[3], c2[3], dl[3];
};

__device__ __forceinline__ HConst32 to_single(const HConst& c)
{
    HConst32 r;
    r.mu_d = c.mu;
    r.mu = (float)c.mu;
    r.b0 = (float)c.b0;
    r.neg_b0s = (float)c.neg_b0s;
    r.neg_als = (float)c.neg_als;
    r.k0s = (float)c.k0s;
    r.b2 = (float)c.b2;
    r.inv_sigma = (float)c.inv_sigma;
    r.dlnN1_dmu = (float)c.dlnN1_dmu;
    r.dlnN1_dsig = (float)c.dlnN1_dsig;
    r.mu_ma = (float)c.mu_ma;
    r.dlnN2t_dal = (float)c.dlnN2t_dal;
    r.inv_f = (float)c.inv_f;
    r.inv_1mf = (float)c.inv_1mf;
    for (int k = 0; k < 8; ++k) r.ang[k] = (float)c.ang[k];
    for (int j = 0; j < 3; ++j) {
        r.c1[j] = (float)c.c1[j];
        r.c2[j] = (float)c.c2[j];
        r.dl[j] = (float)c.dl[j];
    }
    return r;
}

// A double in single precision by integer instructions (mantissa truncated; magnitudes below
// the smallest normal float become a signed zero, which covers the exact zeros of the basis
// columns; beyond the float range an infinity, which the assembly then rejects).  Keeps the conversions of every
// event's 16 columns off the FP64 pipe.
__device__ __forceinline__ float d2f_trunc(double x)
{
    const int hi = __double2hiint(x);
    const unsigned lo = (unsigned)__double2loint(x);
    const int e = (hi >> 20) & 0x7ff;
    const unsigned sign = (unsigned)hi & 0x80000000u;
    unsigned bits = sign | ((unsigned)(e - 896) << 23) | (((unsigned)hi & 0xfffffu) << 3) | (lo >> 29);
    if (e <= 896) bits = sign;
    if (e >= 1151) bits = sign | 0x7f800000u;  // beyond the float range (and inf, NaN): infinity
    return __uint_as_float(bits);
}

template <int KIND, int VAR, bool W>
__device__ __forceinline__ void stage_event32(const HEv& a, const HConst32& c, int64_t e, float* z, int t)
{
    using L = HCols<KIND, W>;
    const bool in = e < a.n;
    const int64_t ei = in ? e : 0;
    auto put = [&](int k, float v) { z[k * kHessThreads + t] = v; };
    const float w = W ? (in ? d2f_trunc(__ldg(a.w + ei)) : 0.0f) : 1.0f;
    const float d = in ? d2f_trunc(__ldg(a.col[kColM] + ei) - c.mu_d) : 0.0f;
    // f G e^{-alpha (m - ma)} = 2^(xs / 1024), xs the argument in the exponential's scale
    const float E = exp2f(fmaf(d, fmaf(c.neg_b0s, d, c.neg_als), c.k0s) * 0x1p-10f);
    const float phmu = fmaf(2.0f * c.b0, d, -c.dlnN1_dmu);
    const float phsig = fmaf(fmaf(2.0f * c.b0 * d, d, -1.0f), c.inv_sigma, -c.dlnN1_dsig);
    const float phal = d + c.mu_ma - c.dlnN2t_dal;
    float P, ps, pb;
    if (KIND == kMass1D) {
        P = E + c.b2;
        const float r = 1.0f / P;
        ps = E * r;
        pb = c.b2 * r;
        put(L::S + 0, ps * phmu);
        put(L::S + 1, ps * phsig);
        put(L::S + 2, pb * phal);
        put(L::S + 3, ps * c.inv_f - pb * c.inv_1mf);
    } else {
        float h[9], t2l, t2k, xp, t2p, xl, xk;
        xl = d2f_trunc(__ldg(a.col[kColCtl] + ei));
        xk = d2f_trunc(__ldg(a.col[kColCtk] + ei));
        if (VAR == kVarPrecompute) {
#pragma unroll
            for (int j = 0; j < 9; ++j) h[j] = d2f_trunc(__ldg(a.col[kColH0 + j] + ei));
            t2l = d2f_trunc(__ldg(a.col[kColT2l] + ei));
            t2k = d2f_trunc(__ldg(a.col[kColT2k] + ei));
            xp = d2f_trunc(__ldg(a.col[kColXp] + ei));
            t2p = d2f_trunc(__ldg(a.col[kColT2p] + ei));
        } else {  // the basis of Eq. 3 from the angles (as angular_basis, in single precision)
            const float phi = d2f_trunc(__ldg(a.col[kColPhi] + ei));
            const float cc = 0.08952465548919477f, cc2 = 2.0f * cc;  // 9/(32 pi)
            const float sl2 = fmaf(-xl, xl, 1.0f), sk2 = fmaf(-xk, xk, 1.0f);
            const float sksl = sqrtf(fmaxf(sk2 * sl2, 0.0f));
            float sp, cp;
            sincosf(phi, &sp, &cp);
            t2l = fmaf(-2.0f, sl2, 1.0f);
            t2k = fmaf(-2.0f, sk2, 1.0f);
            const float csk2 = cc * sk2, h0 = csk2 * fmaf(0.25f, t2l, 0.75f);
            const float aa = csk2 * sl2, bb = cc2 * xk * sksl, bc = bb * cp, bs = bb * sp, ctl2 = xl + xl;
            h[0] = h0;
            h[1] = fmaf(fmaf(-2.0f, csk2, cc2), sl2, -h0);
            h[2] = aa * fmaf(cp + cp, cp, -1.0f);
            h[3] = ctl2 * bc;
            h[4] = bc;
            h[5] = csk2 * (4.0f / 3.0f) * xl;
            h[6] = bs;
            h[7] = ctl2 * bs;
            h[8] = aa * ((sp + sp) * cp);
            xp = phi * 0.3183098861837907f;
            t2p = fmaf(xp + xp, xp, -1.0f);
        }
        float A = fmaf(c.ang[0], h[1], h[0]);
#pragma unroll
        for (int k = 1; k < 8; ++k) A = fmaf(c.ang[k], h[k + 1], A);
        const float x[3] = {xl, xk, xp}, T2[3] = {t2l, t2k, t2p};
        float Cb[3], nu2[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            Cb[j] = fmaf(c.c1[j], x[j], fmaf(c.c2[j], T2[j], 1.0f));
            nu2[j] = fmaf(-c.dl[j], Cb[j], T2[j]);
        }
        const float O[3] = {Cb[1] * Cb[2], Cb[0] * Cb[2], Cb[0] * Cb[1]};
        const float sig = A * E, bg = c.b2 * (O[2] * Cb[2]);
        P = sig + bg;
        const float r = 1.0f / P;
        ps = sig * r;
        pb = bg * r;
        const float rE = r * E, Q = r * c.b2;
        put(L::S + 0, ps * phmu);
        put(L::S + 1, ps * phsig);
#pragma unroll
        for (int k = 0; k < 8; ++k) put(L::S + 2 + k, rE * h[k + 1]);
        put(L::S + 10, pb * phal);
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const float QO = Q * O[j];
            put(L::S + 11 + 2 * j, QO * x[j]);
            put(L::S + 12 + 2 * j, QO * nu2[j]);
        }
        put(L::S + 17, ps * c.inv_f - pb * c.inv_1mf);
        const int jj[3] = {0, 0, 1}, kk[3] = {1, 2, 2}, ll[3] = {2, 1, 0};
#pragma unroll
        for (int q3 = 0; q3 < 3; ++q3) {
            const int j = jj[q3], k = kk[q3];
            const float QC = Q * Cb[ll[q3]];
            const float qn[2] = {QC * x[j], QC * nu2[j]}, nk[2] = {x[k], nu2[k]};
#pragma unroll
            for (int p = 0; p < 2; ++p)
#pragma unroll
                for (int q = 0; q < 2; ++q) put(L::CROSS + 4 * q3 + 2 * p + q, qn[p] * nk[q]);
        }
    }
    if (W) {
#pragma unroll
        for (int k = 0; k < L::NP; ++k) put(L::WS + k, w * z[(L::S + k) * kHessThreads + t]);
    }
    const float wps = w * ps, wpb = w * pb;
    put(L::WPBPHI_MU, wpb * phmu);
    put(L::WPBPHI_SIG, wpb * phsig);
    put(L::WPSPHI_AL, wps * phal);
    put(L::WPS, wps);
    put(L::WPB, wpb);
    put(L::D, d);
    put(L::WPSD, wps * d);
    put(L::WLNP, 0.0f);
    put(L::ONE, 1.0f);
    const bool ok = in && P > 0.0f && P < INFINITY;
    if (ok) {
        put(L::BAD, 0.0f);
    } else {  // no contribution; count it if it is a real event
#pragma unroll 1
        for (int k = 0; k < L::NC; ++k) put(k, 0.0f);
        put(L::ONE, 1.0f);
        put(L::BAD, in ? 1.0f : 0.0f);
    }
}

// Slot sums of one single-precision tile (as tile_slots).
template <int NPS>
__device__ __forceinline__ void tile_slots32(const float* z, const int (&ci)[3], const int (&cj)[3], float (&acc)[3],
                                             int lane)
{
    const float* zi[NPS];
    const float* zj[NPS];
#pragma unroll
    for (int k = 0; k < NPS; ++k) {
        zi[k] = z + ci[k] * kHessThreads;
        zj[k] = z + cj[k] * kHessThreads;
    }
#pragma unroll 8
    for (int e = 0; e < kHessThreads; ++e) {
        const int i = (e + lane) & (kHessThreads - 1);
#pragma unroll
        for (int k = 0; k < NPS; ++k) acc[k] = fmaf(zi[k][i], zj[k][i], acc[k]);
    }
}

// Parameter classes: 0 mass shape (mu, sigma), 1 angular coefficient, 2 exponential slope,
// 3 Chebyshev coefficient, 4 signal fraction.
template <int KIND>
__host__ __device__ inline int pclass(int a)
{
    if (KIND == kMass1D) return a < 2 ? 0 : (a == 2 ? 2 : 4);
    if (a < 2) return 0;
    if (a < 10) return 1;
    if (a == 10) return 2;
    if (a < 17) return 3;
    return 4;
}

// Out: double* or any type whose operator[] gives a double& (the batched passes store their
// toys entry-major).  Rows a0, a0 + astep, ... of H (and W) are assembled, and the NLL and
// gradient with a0 == 0 (the batched passes split the rows over warps); the default is all.
template <int KIND, bool W, class Get, class Out>
__host__ __device__ double assemble_t(const HessTerms& Hh, double sum_wdm, bool want_w2, Get& S, Out nll, Out grad,
                                      Out Hm, Out Wm, int a0 = 0, int astep = 1)
{
    using L = HCols<KIND, W>;
    constexpr int NP = L::NP;
    const int F = NP - 1, AL = KIND == kMass1D ? 2 : 10;
    const double bad = S(L::BAD, L::ONE);
    if (a0 == 0) {
        nll[0] = -(Hh.alpha * sum_wdm + S(L::WLNP, L::ONE));
        for (int a = 0; a < NP; ++a) grad[a] = -S(L::WS + a, L::ONE);
    }
    const double f = Hh.f, g = 1.0 / (f * (1.0 - f));
    const double sg = Hh.sigma, b0 = Hh.b0;
    auto sig = [](int c) { return c == 0 || c == 1; };
    for (int a = a0; a < NP; a += astep) {
        for (int b = a; b < NP; ++b) {
            const int ca = pclass<KIND>(a), cb = pclass<KIND>(b);
            double h;
            if (cb == 4) {  // b == f (last), a <= b
                if (a == F)
                    h = S(L::WS + F, L::S + F);
                else if (sig(ca))
                    h = -g * S(L::WPB, L::S + a);
                else
                    h = g * S(L::WPS, L::S + a);
            } else if (ca == 0 && cb == 0) {  // mass shape block, plus the Gaussian curvature
                h = -S(L::WPBPHI_MU + a, L::S + b);
                const double wps = S(L::WPS, L::ONE);
                if (a == 0 && b == 0)
                    h += (2.0 * b0 + Hh.d2lnN1[0]) * wps;
                else if (a == 0)
                    h += 2.0 / (sg * sg * sg) * S(L::WPSD, L::ONE) + Hh.d2lnN1[1] * wps;
                else
                    h += 3.0 / (sg * sg * sg * sg) * S(L::WPSD, L::D) - (1.0 / (sg * sg) - Hh.d2lnN1[2]) * wps;
            } else if (ca == 0 && cb == 1) {
                h = -S(L::WPBPHI_MU + a, L::S + b);
            } else if (ca == 1 && cb == 1) {
                h = S(L::WS + a, L::S + b);
            } else if (sig(ca) != sig(cb)) {  // signal x background
                h = S(L::WS + a, L::S + b);
            } else if (ca == 2 && cb == 2) {
                h = -S(L::WPSPHI_AL, L::S + AL) + Hh.d2lnN2t_dal2 * S(L::WPB, L::ONE);
            } else if (ca == 2) {  // slope x Chebyshev
                h = -S(L::WPSPHI_AL, L::S + b);
            } else {  // Chebyshev x Chebyshev
                const int ja = (a - 11) / 2, pa = (a - 11) % 2, jb = (b - 11) / 2, pb = (b - 11) % 2;
                if (ja == jb) {
                    h = S(L::WS + a, L::S + b);
                    if (pb == 1) h += (pa == 0 ? 1.0 : 2.0) * Hh.dlnNc_dc2[ja] * S(L::WS + a, L::ONE);
                } else {
                    const int q3 = ja == 0 ? (jb == 1 ? 0 : 1) : 2;
                    h = -S(L::WPS, L::CROSS + 4 * q3 + 2 * pa + pb);
                }
            }
            Hm[a * NP + b] = Hm[b * NP + a] = h;
        }
    }
    // W's slots come after all of H's, so H's slots (and their summation order) do not
    // depend on whether W is requested
    if (want_w2)
        for (int a = a0; a < NP; a += astep)
            for (int b = a; b < NP; ++b) Wm[a * NP + b] = Wm[b * NP + a] = S(L::WS + a, L::WS + b);
    return bad;
}


}  // namespace gbnll
