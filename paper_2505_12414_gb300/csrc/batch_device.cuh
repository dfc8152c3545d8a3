// batch_device.cuh -- device code shared by the batched fit loop (batch.cu) and the batched
// Hessian passes (batch_hess.cu): the device table, the parameter-only terms of a toy's point
// (Sec. 2.4.1 hoisting, as the host's), the NLL and gradient from a step's sums, the sine
// transform of bounded parameters, and the warp-level helpers of the minimiser (sums, the
// symmetric inverse, the first quasi-Newton step).
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include "../../include/gbnll.h"
#include "batch_internal.h"
#include "fp64_math.cuh"
#include "gbnll_internal.h"
#include "nll_device.cuh"

namespace gbnll {
namespace {

const double kPiH = 3.14159265358979323846;

// the exponential's table (and the logarithm's and sin/cos tables after it): one copy per
// translation unit, uploaded by that unit's own set-up (ensure_btab in batch.cu, the Hessian
// work arrays' set-up in batch_hess.cu)
__device__ double g_btab[kTabDoubles];


// ---------------------------------------------------------------------------------
// device-side parameter-only terms and gradient assembly (same formulas as runtime.cu)
// ---------------------------------------------------------------------------------
__device__ inline double dev_gauss_norm(double za, double zb)
{
    if (zb > 0.0) return 0.5 * (erfc(zb) - erfc(za));
    if (za < 0.0) return 0.5 * (erfc(-za) - erfc(-zb));
    return 0.5 * (erf(za) - erf(zb));
}

// second: also the second derivatives of the normalisations (the Hessian passes need them,
// the steps of the fit loop do not)
__device__ inline bool dev_hoist(int kind, const double* ranges, const double* th, KConst& k, DConst& H, bool second)
{
    const int npar = kind == kMass1D ? 4 : 18;
    for (int i = 0; i < npar; ++i)
        if (!isfinite(th[i])) return false;
    const double ma = ranges[0], mb = ranges[1], D = mb - ma;
    double mu = th[0], sigma = th[1];
    double alpha = kind == kMass1D ? th[2] : th[10];
    double f = kind == kMass1D ? th[3] : th[17];
    if (!(sigma > 0.0) || !(f > 0.0 && f < 1.0)) return false;
    // the formulas of the host hoisting, with the divisions by the same quantity taken as one
    // reciprocal each (this chain runs once per toy and step, and FP64 is scarce)
    const double kInvSqrt2 = 0.70710678118654752440, kInvSqrtPi = 0.56418958354775628695;
    const double kInvSqrt2Pi = 0.39894228040143267794, kHalfLn2Pi = 0.91893853320467274178;
    const double inv_s = 1.0 / sigma, r2s = kInvSqrt2 * inv_s;
    double za = (mu - ma) * r2s, zb = (mu - mb) * r2s;
    double N1 = dev_gauss_norm(za, zb);
    if (!(N1 > 1e-300)) return false;
    double ea = exp(-za * za), eb = exp(-zb * zb);
    const double q = inv_s / N1;  // 1 / (sigma N1)
    H.dlnN1_dmu = (ea - eb) * (kInvSqrt2Pi * q);
    H.dlnN1_dsig = -(za * ea - zb * eb) * (kInvSqrtPi * q);
    if (second) {  // second derivatives of ln N1 (as the host hoisting)
        const double q2 = q * inv_s;  // 1 / (sigma^2 N1)
        H.d2lnN1[0] = -(za * ea - zb * eb) * (kInvSqrtPi * q2) - H.dlnN1_dmu * H.dlnN1_dmu;
        H.d2lnN1[1] = (ea * (2.0 * za * za - 1.0) - eb * (2.0 * zb * zb - 1.0)) * (kInvSqrt2Pi * q2) -
                      H.dlnN1_dmu * H.dlnN1_dsig;
        H.d2lnN1[2] = 2.0 * (za * ea * (1.0 - za * za) - zb * eb * (1.0 - zb * zb)) * (kInvSqrtPi * q2) -
                      H.dlnN1_dsig * H.dlnN1_dsig;
    }
    double t = alpha * D, Nt2;
    if (second) {  // d^2 ln Ntilde2 / dalpha^2 = D^2 v(|t|), v(a) = 1/a^2 - e^-a/(1 - e^-a)^2, series below 1/2
        const double a = fabs(t);
        double v;
        if (a < 0.5) {
            const double c[9] = {1.0 / 12.0,
                                 -1.0 / 240.0,
                                 1.0 / 6048.0,
                                 -1.0 / 172800.0,
                                 9.0 * (5.0 / 66.0) / 3628800.0,
                                 11.0 * (-691.0 / 2730.0) / 479001600.0,
                                 13.0 * (7.0 / 6.0) / 87178291200.0,
                                 15.0 * (-3617.0 / 510.0) / 20922789888000.0,
                                 17.0 * (43867.0 / 798.0) / 6402373705728000.0};
            const double a2 = a * a;
            v = c[8];
            for (int q = 7; q >= 0; --q) v = fma(v, a2, c[q]);
        } else {
            const double em = expm1(-a);
            v = 1.0 / (a * a) - exp(-a) / (em * em);
        }
        H.d2lnN2t_dal2 = D * D * v;
    }
    if (alpha == 0.0) {
        Nt2 = D;
        H.dlnN2t_dal = 0.5 * D;
    } else {
        const double em = expm1(t);
        Nt2 = em / alpha;
        if (fabs(t) > 1e-3)  // -1/expm1(-t) = 1 + 1/expm1(t)
            H.dlnN2t_dal = D * ((1.0 + 1.0 / em) - 1.0 / t);
        else
            H.dlnN2t_dal = D * (0.5 + t / 12.0 - t * t * t / 720.0 + t * t * t * t * t / 30240.0);
    }
    double b0 = 0.5 * inv_s * inv_s;
    double lnb1 = log(f * q) - kHalfLn2Pi;  // ln(f / (sqrt(2 pi) sigma N1))
    double b2 = (1.0 - f) / Nt2;
    if (kind == kKstar4D) {
        double rprod = 1.0 / kPiH;  // 1 / (pi Nc_0 Nc_1 Nc_2)
        for (int j = 0; j < 3; ++j) {
            double nc = 2.0 - (2.0 / 3.0) * th[12 + 2 * j];
            if (!(nc > 0.0)) return false;
            const double rnc = 1.0 / nc;
            H.dlnNc[j] = (-2.0 / 3.0) * rnc;
            rprod *= rnc;
        }
        b2 *= rprod;
    }
    if (fabs(alpha) * D + fmax(lnb1, 0.0) > 700.0) return false;
    H.mu = mu;
    H.sigma = sigma;
    H.alpha = alpha;
    H.f = f;
    H.ma = ma;
    H.b0 = b0;
    H.b2 = b2;
    H.lnb1 = lnb1;
    const double S = kExpArgScale;
    k.mu = mu;
    k.neg_b0 = -b0 * S;
    k.neg_alpha = -alpha * S;
    k.k0 = (lnb1 - alpha * (mu - ma)) * S;
    k.b2 = b2;
    if (kind == kKstar4D) {
        for (int j = 0; j < 8; ++j) k.ang[j] = th[2 + j];
        k.k0d = (lnb1 + kLnBasisC - alpha * (mu - ma)) * S;
        for (int j = 0; j < 8; ++j) k.angd[j] = th[2 + j] * direct_factor(j + 1);
        k.cq[0] = b2;
        k.cq[1] = b2 * th[11];
        k.cq[2] = b2 * th[12];
        k.cq[3] = 1.0;
        k.cq[4] = th[13];
        k.cq[5] = th[14];
        k.cq[6] = 1.0;
        k.cq[7] = th[15];
        k.cq[8] = th[16];
    }
    H.ok = 1;
    return true;
}

// NLL and full external gradient from the sums S; false if the density was not positive.
__device__ inline bool dev_assemble(int kind, const DConst& H, double sum_wdm, const double* S, double& nll, double* g)
{
    const int K = kind == kMass1D ? kAcc1D : kAcc4D;
    if (S[K - 1] != 0.0 || !isfinite(S[0])) return false;
    nll = -(H.alpha * sum_wdm + S[0]);
    const double two_b0 = 2.0 * H.b0, dma = H.mu - H.ma;
    double dL[kNP];
    dL[0] = two_b0 * S[2] - H.dlnN1_dmu * S[1];
    dL[1] = two_b0 / H.sigma * S[3] - (1.0 / H.sigma + H.dlnN1_dsig) * S[1];
    int npar;
    if (kind == kMass1D) {
        double sre = H.b2 * S[4], sred = H.b2 * S[5];
        dL[2] = sred + dma * sre - H.dlnN2t_dal * sre;
        dL[3] = S[1] / H.f - sre / (1.0 - H.f);
        npar = 4;
    } else {
        for (int k = 0; k < 8; ++k) dL[2 + k] = S[4 + k];
        double sre = S[12], sred = S[13];
        dL[10] = sred + dma * sre - H.dlnN2t_dal * sre;
        dL[11] = H.b2 * S[14];
        dL[12] = H.b2 * S[15] - H.dlnNc[0] * sre;
        dL[13] = S[16];
        dL[14] = S[17] - H.dlnNc[1] * sre;
        dL[15] = S[18];
        dL[16] = S[19] - H.dlnNc[2] * sre;
        dL[17] = S[1] / H.f - sre / (1.0 - H.f);
        npar = 18;
    }
#pragma unroll
    for (int k = 0; k < kNP; ++k)
        if (k < npar) g[k] = -dL[k];
    return isfinite(nll);
}

// ---------------------------------------------------------------------------------
// sine transform of bounded parameters (Minuit manual)
// ---------------------------------------------------------------------------------
__device__ __forceinline__ double to_ext(const FitConfig& c, int i, double x)
{
    int k = c.idx[i];
    return c.bounded[k] ? c.lo[k] + (c.hi[k] - c.lo[k]) * 0.5 * (sin(x) + 1.0) : x;
}

__device__ __forceinline__ double jac(const FitConfig& c, int i, double x)
{
    int k = c.idx[i];
    return c.bounded[k] ? (c.hi[k] - c.lo[k]) * 0.5 * cos(x) : 1.0;
}

// ---------------------------------------------------------------------------------
// warp helpers of the minimiser (warp per toy)
// ---------------------------------------------------------------------------------
__device__ __forceinline__ double wsum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// inverse of the symmetric positive-definite n x n matrix A (row-major, smem; its upper
// triangle is read and destroyed) into Out by a warp, with the sweep operator (Beaton 1964;
// Goodnight, Am. Stat. 33 (1979) 149): sweeping pivot k replaces
//   A_kk -> -1/A_kk,  A_ik -> A_ik / A_kk (i != k),  A_ij -> A_ij - A_ik A_kj / A_kk (i, j != k),
// which keeps A symmetric, and after every pivot has been swept A holds -A^-1.  Each lane owns
// up to kSweepPerLane entries of the upper triangle, so one pivot costs a reciprocal and two
// FP64 instructions per owned entry (the FP64 pipe is charged per warp instruction, however few
// lanes take part).  The pivots are the diagonal of the successive Schur complements: a pivot
// that is not positive and finite means A is not positive definite, and the call returns false
// (all lanes).
constexpr int kSweepPerLane = (kNP * (kNP + 1) / 2 + 31) / 32;

__device__ inline bool warp_spd_inverse(int n, double* A, double* Out)
{
    const int lane = threadIdx.x & 31;
    const int ne = n * (n + 1) / 2;
    int ei[kSweepPerLane], ej[kSweepPerLane];
#pragma unroll
    for (int q = 0; q < kSweepPerLane; ++q) {
        int idx = lane + 32 * q, i = 0;
        if (idx < ne) {
            while (idx >= n - i) idx -= n - i++;
            ei[q] = i;
            ej[q] = i + idx;
        } else {
            ei[q] = -1;
            ej[q] = -1;
        }
    }
    __syncwarp();
    for (int k = 0; k < n; ++k) {
        const double D = A[k * n + k];
        if (!(D > 0.0) || !isfinite(D)) return false;  // the same value on every lane
        const double r = frcp(D);  // 3 FP64 instructions where a division takes several more
        double nv[kSweepPerLane];
#pragma unroll
        for (int q = 0; q < kSweepPerLane; ++q) {
            const int i = ei[q], j = ej[q];
            nv[q] = 0.0;
            if (i < 0) continue;
            const double aij = A[i * n + j];
            if (i == k && j == k)
                nv[q] = -r;
            else if (i == k || j == k)
                nv[q] = aij * r;
            else {
                const double aik = i < k ? A[i * n + k] : A[k * n + i];
                const double akj = k < j ? A[k * n + j] : A[j * n + k];
                nv[q] = fma(-aik * r, akj, aij);
            }
        }
        __syncwarp();
#pragma unroll
        for (int q = 0; q < kSweepPerLane; ++q)
            if (ei[q] >= 0) A[ei[q] * n + ej[q]] = nv[q];
        __syncwarp();
    }
#pragma unroll
    for (int q = 0; q < kSweepPerLane; ++q)
        if (ei[q] >= 0) Out[ei[q] * n + ej[q]] = Out[ej[q] * n + ei[q]] = -A[ei[q] * n + ej[q]];
    __syncwarp();
    return true;
}

// The minimiser's first step from its start point x = F.xt (warp per toy): f0 and the free
// components of the external gradient there (lane i holds component i of g0), the start
// matrix in F.V when `have` (else diag(step^2) is set).  Records the point, its gradient and
// EDM and proposes the trial point x + p, p = -V g (phase kPhSearch).  Returns true when the
// EDM already meets the tolerance; with `defer` (and `have`) it then changes nothing, leaving
// the start to the fit loop's first step.
__device__ inline bool begin_search(const FitConfig& c, ToyFit& F, double f0, double g0, bool have, bool defer, int lane)
{
    const int nf = c.nf;
    const bool mine = lane < nf;
    const double xi = mine ? F.xt[lane] : 0.0;
    const double gi = mine ? g0 * jac(c, lane, xi) : 0.0;
    if (!have && mine)
        for (int j = 0; j < nf; ++j) F.V[lane * nf + j] = lane == j ? F.sint[lane] * F.sint[lane] : 0.0;
    __syncwarp();
    double vg = 0.0;
    if (mine)
        for (int j = 0; j < nf; ++j) vg += F.V[lane * nf + j] * __shfl_sync(0xffffffffu, gi, j);
    else
        for (int j = 0; j < nf; ++j) (void)__shfl_sync(0xffffffffu, gi, j);
    const double edm = 0.5 * wsum(mine ? gi * vg : 0.0);
    const bool met = edm < c.tol_edm;
    if (defer && met) return true;
    const double pi = -vg;
    const double gp = wsum(mine ? gi * pi : 0.0);
    if (mine) {
        F.x[lane] = xi;
        F.g[lane] = gi;
        F.gext[lane] = g0;
        F.th[c.idx[lane]] = to_ext(c, lane, xi);
        F.p[lane] = pi;
        F.xt[lane] = xi + pi;
    }
    if (lane == 0) {
        F.f = f0;
        F.first = have ? 0 : 1;
        F.edm = edm;
        F.gp = gp;
        F.alpha = 1.0;
        F.iter = 1;
        if (!met) F.phase = kPhSearch;
    }
    __syncwarp();
    return met;
}

}  // namespace
}  // namespace gbnll
