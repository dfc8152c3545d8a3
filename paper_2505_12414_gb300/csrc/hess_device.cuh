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

template <int KIND, bool W, class Get>
__host__ __device__ double assemble_t(const HessTerms& Hh, double sum_wdm, bool want_w2, Get& S, double* nll,
                                      double* grad, double* Hm, double* Wm)
{
    using L = HCols<KIND, W>;
    constexpr int NP = L::NP;
    const int F = NP - 1, AL = KIND == kMass1D ? 2 : 10;
    const double bad = S(L::BAD, L::ONE);
    *nll = -(Hh.alpha * sum_wdm + S(L::WLNP, L::ONE));
    for (int a = 0; a < NP; ++a) grad[a] = -S(L::WS + a, L::ONE);
    const double f = Hh.f, g = 1.0 / (f * (1.0 - f));
    const double sg = Hh.sigma, b0 = Hh.b0;
    auto sig = [](int c) { return c == 0 || c == 1; };
    for (int a = 0; a < NP; ++a) {
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
        for (int a = 0; a < NP; ++a)
            for (int b = a; b < NP; ++b) Wm[a * NP + b] = Wm[b * NP + a] = S(L::WS + a, L::WS + b);
    return bad;
}


}  // namespace gbnll
