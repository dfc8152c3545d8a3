// batch.cu -- batched pseudo-experiments: many independent fits of one model, each toy
// with its own sample (CSR, uneven sizes), evaluated and minimised on the device.
//
// The paper validates fits with pseudo-experiments and uses them for coverage corrections
// (Sec. 1, Sec. 2.5, Sec. 3.1); its toy study runs generate -> fit -> HESSE one toy at a time
// with the minimiser on the host.  Here one device step advances every active toy:
//   batch_prepare  (thread per toy)  parameter-only terms of each toy's trial point(s)
//                                    (Sec. 2.4.1 hoisting, computed on the device), one work
//                                    item per (toy, point) and one work unit per event tile;
//   batch_eval     (persistent)      blocks pull units from a device counter and run the
//                                    fused per-event NLL+gradient pass of the single-sample
//                                    kernel over the unit's tile, writing the unit's sums;
//   batch_update   (warp per toy)    sums the units of each item in tile order, assembles
//                                    NLL and gradient and advances the toy's minimiser:
//                                    BFGS on sine-transformed bounded parameters with an
//                                    Armijo line search, optionally started from and finished
//                                    with a finite-difference Hessian of the analytic gradient
//                                    (all stencil points of all toys in one step).
// The three launches (plus a counter reset) and a one-thread control kernel are the body of
// a while node of a CUDA graph, so one launch runs the whole fit loop on the device.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/gbnll.h"
#include "fp64_math.cuh"
#include "gbnll_internal.h"
#include "batch_internal.h"
#include "hess_device.cuh"
#include "nll_device.cuh"
#include "trace.h"
#include "tune_cache.h"

namespace gbnll {
namespace {

const double kPiH = 3.14159265358979323846;

__device__ double g_btab[kTabDoubles];


// ---------------------------------------------------------------------------------
// device-side parameter-only terms and gradient assembly (same formulas as runtime.cu)
// ---------------------------------------------------------------------------------
__device__ double dev_gauss_norm(double za, double zb)
{
    if (zb > 0.0) return 0.5 * (erfc(zb) - erfc(za));
    if (za < 0.0) return 0.5 * (erfc(-za) - erfc(-zb));
    return 0.5 * (erf(za) - erf(zb));
}

// second: also the second derivatives of the normalisations (the Hessian passes need them,
// the steps of the fit loop do not)
__device__ bool dev_hoist(int kind, const double* ranges, const double* th, KConst& k, DConst& H, bool second)
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
__device__ bool dev_assemble(int kind, const DConst& H, double sum_wdm, const double* S, double& nll, double* g)
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
// prepare: one thread per toy
// ---------------------------------------------------------------------------------
// event pairs per work unit this step (0: one unit per item)
__device__ __forceinline__ int step_tile(const BatchDev& b) { return (b.tile_pairs && b.step_tp) ? *b.step_tp : b.tile_pairs; }

__device__ void emit_item(const BatchDev& b, int toy, int slot, const double* th, int64_t npairs)
{
    ToyFit& F = b.fits[toy];
    int nt = 0;
    const int tp = step_tile(b);
    if (npairs > 0) nt = tp ? (int)((npairs + tp - 1) / tp) : 1;
    KConst kc;
    DConst dc;
    memset(&kc, 0, sizeof kc);
    memset(&dc, 0, sizeof dc);
    bool ok = dev_hoist(b.cfg.kind, b.cfg.ranges, th, kc, dc, false);
    if (!ok) nt = 0;
    int it = atomicAdd(&b.counters[0], 1);
    if (it >= b.max_items) {  // cannot happen with the host's sizing; keep the toy consistent
        F.item[slot] = -1;
        return;
    }
    int u0 = nt ? atomicAdd(&b.counters[1], nt) : 0;
    if (u0 + nt > b.max_units) {
        nt = 0;
        dc.ok = 0;
    }
    b.item_toy[it] = toy;
    b.item_u0[it] = u0;
    b.item_nt[it] = nt;
    b.item_kc[it] = kc;
    b.item_dc[it] = dc;
    for (int j = 0; j < nt; ++j) {
        b.unit_item[u0 + j] = it;
        b.unit_tile[u0 + j] = j;
    }
    F.item[slot] = it;
}

__global__ void batch_prepare(BatchDev b)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= b.n_toys) return;
    ToyFit& F = b.fits[t];
    if (F.phase == kPhDone) {
        F.nitem = 0;
        return;
    }
    const FitConfig& c = b.cfg;
    const int64_t npairs = (b.ev_end[t] - b.ev_begin[t] + 1) / 2;
    double th[kNP];
    for (int k = 0; k < c.npar; ++k) th[k] = F.th[k];
    int ni = 0;  // item slots written this step
    if (F.phase == kPhInit || F.phase == kPhSearch) {
        for (int i = 0; i < c.nf; ++i) th[c.idx[i]] = to_ext(c, i, F.xt[i]);
        emit_item(b, t, 0, th, npairs);
        ni = 1;
        if (F.phase == kPhInit && c.strategy == 1) {
            ni = 1 + 2 * c.nf;
            // stencil in internal coordinates around the start point
            for (int j = 0; j < c.nf; ++j)
                for (int sgn = 0; sgn < 2; ++sgn) {
                    for (int i = 0; i < c.nf; ++i) th[c.idx[i]] = to_ext(c, i, F.xt[i]);
                    double h = 0.1 * F.sint[j];
                    th[c.idx[j]] = to_ext(c, j, F.xt[j] + (sgn ? -h : h));
                    emit_item(b, t, 1 + 2 * j + sgn, th, npairs);
                }
        }
    } else if (F.phase == kPhHess) {
        // stencil in external coordinates around the minimum (slot 0 unused)
        F.item[0] = -1;
        ni = 1 + 2 * c.nf;
        for (int j = 0; j < c.nf; ++j)
            for (int sgn = 0; sgn < 2; ++sgn) {
                for (int k = 0; k < c.npar; ++k) th[k] = F.th[k];
                th[c.idx[j]] += sgn ? -F.hstep[j] : F.hstep[j];
                emit_item(b, t, 1 + 2 * j + sgn, th, npairs);
            }
    }
    F.nitem = ni;
}

// ---------------------------------------------------------------------------------
// evaluate: persistent blocks over work units
// ---------------------------------------------------------------------------------
template <int KIND, int VAR, bool W>
__global__ void __launch_bounds__(kEvalThreads, 1) batch_eval(BatchDev b)
{
    constexpr int K = KIND == kMass1D ? kAcc1D : kAcc4D;
    __shared__ double s_tab[(KIND == kKstar4D && VAR == kVarDirect) ? kTabDoubles : (W ? kTrigOffset : kExpTable)];
    __shared__ double s_red[(kEvalThreads / 32) * K];
    __shared__ int s_u;
    constexpr int ntab = (KIND == kKstar4D && VAR == kVarDirect) ? kTabDoubles : (W ? kTrigOffset : kExpTable);
    for (int j = threadIdx.x; j < ntab; j += blockDim.x) s_tab[j] = g_btab[j];
    __syncthreads();
    const int nunits = min(b.counters[1], b.max_units);
    const int tp = step_tile(b);
    while (true) {
        if (threadIdx.x == 0) s_u = atomicAdd(&b.counters[2], 1);
        __syncthreads();
        const int u = s_u;
        __syncthreads();
        if (u >= nunits) break;
        const int item = b.unit_item[u], tile = b.unit_tile[u];
        const int toy = b.item_toy[item];
        const KConst c = b.item_kc[item];
        const int64_t ev_end = b.ev_end[toy];
        const int64_t p_first = b.ev_begin[toy] / 2, p_last = (ev_end + 1) / 2;
        int64_t pb = p_first, pe = p_last;
        if (tp) {
            pb = p_first + (int64_t)tile * tp;
            pe = min(pb + (int64_t)tp, p_last);
        }
        double acc[K];
#pragma unroll
        for (int k = 0; k < K; ++k) acc[k] = 0.0;
        LogProd lpx{1.0, 0}, lpy{1.0, 0};
        int bad = 0;
        for (int64_t p = pb + threadIdx.x; p < pe; p += blockDim.x) {
            PairIn in;
            load_pair<KIND, VAR, W>(b.cols, p, in);
            process_pair<KIND, VAR, W, true>(c, in, (2 * p + 1) < ev_end, acc, lpx, lpy, bad, s_tab);
        }
        if (!W) {
            double lw = logprod_value(logprod_warp(logprod_combine(lpx, lpy)));
            acc[0] = (threadIdx.x & 31) == 0 ? lw : 0.0;
        }
        acc[K - 1] = (double)bad;
        if (KIND == kKstar4D && VAR == kVarDirect) direct_unscale<K>(acc);
        double r = block_reduce<K>(acc, s_red);
        if (threadIdx.x < K) b.unit_sums[(size_t)u * kAccMax + threadIdx.x] = r;
    }
}

// ---------------------------------------------------------------------------------
// update: one warp per toy
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

__device__ bool warp_spd_inverse(int n, double* A, double* Out)
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
__device__ bool begin_search(const FitConfig& c, ToyFit& F, double f0, double g0, bool have, bool defer, int lane)
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

template <int KIND>
__global__ void __launch_bounds__(kUpdWarps * 32) batch_update(BatchDev b)
{
    constexpr int K = KIND == kMass1D ? kAcc1D : kAcc4D;
    __shared__ double s_S[kUpdWarps][32];
    __shared__ double s_g[kUpdWarps][kNP];
    __shared__ double s_mat[kUpdWarps][2][kNP * kNP];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int t = blockIdx.x * kUpdWarps + wib;
    if (t >= b.n_toys) return;
    ToyFit& F = b.fits[t];
    if (F.phase == kPhDone) return;
    const FitConfig& c = b.cfg;
    const int nf = c.nf;
    const bool mine = lane < nf;

    // assemble every evaluated slot: f_s and the free components of the external gradient
    double f0 = INFINITY, g0 = 0.0;  // slot 0 (lane-uniform f0; lane i holds component i)
    bool ok0 = false, sten_ok = true;
    int nslots = 0;
    const int ni = F.nitem;
    for (int s = 0; s < ni; ++s) {
        const int it = F.item[s];
        if (it < 0) continue;
        ++nslots;
        const int u0 = b.item_u0[it], nt = b.item_nt[it];
        double v = 0.0;
        if (lane < K)
            for (int j = 0; j < nt; ++j) v += b.unit_sums[(size_t)(u0 + j) * kAccMax + lane];
        s_S[wib][lane] = v;
        __syncwarp();
        double fv = INFINITY;
        int okv = 0;
        if (lane == 0) {  // the full external gradient into shared memory
            const DConst dc = b.item_dc[it];
            if (dc.ok && dev_assemble(c.kind, dc, b.sum_wdm[t], s_S[wib], fv, s_g[wib])) okv = 1;
        }
        __syncwarp();
        fv = __shfl_sync(0xffffffffu, fv, 0);
        okv = __shfl_sync(0xffffffffu, okv, 0);
        double gi = (mine && okv) ? s_g[wib][c.idx[lane]] : 0.0;
        __syncwarp();
        if (s == 0) {
            f0 = fv;
            ok0 = okv;
            g0 = gi;
        } else {
            if (!okv) sten_ok = false;
            if (mine) F.gsten[s - 1][lane] = gi;
        }
    }
    if (lane == 0) F.n_eval += nslots;

    double* A = s_mat[wib][0];
    double* Out = s_mat[wib][1];
    const double c1 = 1e-4;
    bool finish = false;      // reached the convergence test (go to the Hessian or done)
    int done_status = -1;     // >= 0: toy ends with this status

    if (F.phase == kPhInit) {
        if (!ok0) {
            done_status = NLL_ERR_NONPOSITIVE_PDF;
        } else {
            // initial inverse Hessian: from the analytic Hessian pass, the inverse of the
            // stencil Hessian, or diag(step^2)
            bool have = false;
            if (c.strategy == 2) {
                have = F.vset != 0;  // set by the analytic Hessian pass before the first step
            } else if (c.strategy && sten_ok) {
                const double xi = mine ? F.xt[lane] : 0.0;
                const double Ji = mine ? jac(c, lane, xi) : 0.0;
                for (int j = 0; j < nf; ++j) {
                    double h = 0.1 * F.sint[j];
                    if (mine) {
                        // internal gradient at x +- h e_j: the Jacobian changes only in component j
                        double Jp = lane == j ? jac(c, lane, xi + h) : Ji;
                        double Jm = lane == j ? jac(c, lane, xi - h) : Ji;
                        A[lane * nf + j] = (F.gsten[2 * j][lane] * Jp - F.gsten[2 * j + 1][lane] * Jm) / (2.0 * h);
                    }
                }
                __syncwarp();
                if (mine)
                    for (int j = 0; j < lane; ++j) {
                        double sym = 0.5 * (A[lane * nf + j] + A[j * nf + lane]);
                        A[lane * nf + j] = sym;
                    }
                __syncwarp();
                if (mine)
                    for (int j = lane + 1; j < nf; ++j) A[lane * nf + j] = A[j * nf + lane];
                __syncwarp();
                have = warp_spd_inverse(nf, A, Out);
                if (have && mine)
                    for (int j = 0; j < nf; ++j) F.V[lane * nf + j] = Out[lane * nf + j];
                __syncwarp();
            }
            finish = begin_search(c, F, f0, g0, have, false, lane);
        }
    } else if (F.phase == kPhSearch) {
        const double f = F.f, alpha = F.alpha, gp = F.gp;
        const bool accept = ok0 && f0 <= f + c1 * alpha * gp;
        if (accept) {
            const double xt = mine ? F.xt[lane] : 0.0, x = mine ? F.x[lane] : 0.0, gi_old = mine ? F.g[lane] : 0.0;
            const double gt = mine ? g0 * jac(c, lane, xt) : 0.0;
            const double si = xt - x, yi = gt - gi_old;
            const double ys = wsum(yi * si), yy = wsum(yi * yi), ss = wsum(si * si);
            // the lane's row of V in registers: one load and one store per step instead of a
            // global round trip per product (lanes beyond nf and columns beyond nf hold 0)
            double vr[kNP];
#pragma unroll
            for (int j = 0; j < kNP; ++j) vr[j] = (mine && j < nf) ? F.V[lane * nf + j] : 0.0;
            if (ys > 1e-300 && ys > 1e-12 * sqrt(yy * ss)) {
                if (F.first) {
#pragma unroll
                    for (int j = 0; j < kNP; ++j) vr[j] = (mine && lane == j) ? ys / yy : 0.0;
                }
                double vy = 0.0;
#pragma unroll
                for (int j = 0; j < kNP; ++j) vy += vr[j] * __shfl_sync(0xffffffffu, yi, j);
                const double yvy = wsum(mine ? yi * vy : 0.0);
                const double rho = 1.0 / ys;
#pragma unroll
                for (int j = 0; j < kNP; ++j) {
                    const double sj = __shfl_sync(0xffffffffu, si, j), vyj = __shfl_sync(0xffffffffu, vy, j);
                    if (mine && j < nf) vr[j] += rho * ((1.0 + rho * yvy) * si * sj - vy * sj - si * vyj);
                }
                if (lane == 0) F.first = 0;
            }
            if (mine) {
                F.x[lane] = xt;
                F.g[lane] = gt;
                F.gext[lane] = g0;
                F.th[c.idx[lane]] = to_ext(c, lane, xt);
            }
            if (lane == 0) F.f = f0;
            double vg = 0.0;
#pragma unroll
            for (int j = 0; j < kNP; ++j) vg += vr[j] * __shfl_sync(0xffffffffu, gt, j);
            const double edm = 0.5 * wsum(mine ? gt * vg : 0.0);
            if (lane == 0) F.edm = edm;
            // an accepted step that did not lower the NLL (its change is below the rounding of
            // the sum near the minimum): stop, as the host minimiser does
            const bool stalled = !(f0 < f) && F.iter > 2;
            if (edm < c.tol_edm) {
                finish = true;
            } else if (stalled) {
                if (c.hessian) {
                    finish = true;
                } else {
                    done_status = edm < 100.0 * c.tol_edm ? NLL_OK : NLL_ERR_NOT_CONVERGED;
                    finish = done_status == NLL_OK;
                    if (finish) done_status = -1;
                }
            } else if (F.iter >= c.max_iter) {
                done_status = NLL_ERR_NOT_CONVERGED;
            } else {
                double pi = -vg;
                double gpn = wsum(mine ? gt * pi : 0.0);
                if (!(gpn < 0.0)) {  // not a descent direction: restart from the diagonal
                    const double s2 = mine ? F.sint[lane] * F.sint[lane] : 0.0;
#pragma unroll
                    for (int j = 0; j < kNP; ++j) vr[j] = (mine && lane == j) ? s2 : 0.0;
                    pi = -s2 * gt;
                    gpn = wsum(mine ? gt * pi : 0.0);
                }
                if (mine) {
                    F.p[lane] = pi;
                    F.xt[lane] = xt + pi;
                }
                if (lane == 0) {
                    F.gp = gpn;
                    F.alpha = 1.0;
                    F.iter += 1;
                }
            }
            if (mine) {
#pragma unroll
                for (int j = 0; j < kNP; ++j)
                    if (j < nf) F.V[lane * nf + j] = vr[j];
            }
            __syncwarp();
        } else {
            double anew;
            if (ok0 && isfinite(f0)) {
                const double denom = 2.0 * (f0 - f - gp * alpha);
                anew = denom > 0.0 ? -gp * alpha * alpha / denom : 0.5 * alpha;
                anew = fmin(fmax(anew, 0.1 * alpha), 0.5 * alpha);
            } else {
                anew = 0.25 * alpha;
            }
            if (anew < 1e-12) {
                done_status = F.edm < 100.0 * c.tol_edm ? NLL_OK : NLL_ERR_NOT_CONVERGED;
                finish = done_status == NLL_OK;
                if (finish) done_status = -1;
            } else {
                if (mine) F.xt[lane] = F.x[lane] + anew * F.p[lane];
                if (lane == 0) F.alpha = anew;
            }
        }
    } else if (F.phase == kPhHess) {
        bool have = false;
        if (sten_ok) {
            for (int j = 0; j < nf; ++j)
                if (mine) A[lane * nf + j] = (F.gsten[2 * j][lane] - F.gsten[2 * j + 1][lane]) / (2.0 * F.hstep[j]);
            __syncwarp();
            if (mine)
                for (int j = 0; j < lane; ++j) A[lane * nf + j] = 0.5 * (A[lane * nf + j] + A[j * nf + lane]);
            __syncwarp();
            if (mine)
                for (int j = lane + 1; j < nf; ++j) A[lane * nf + j] = A[j * nf + lane];
            __syncwarp();
            have = warp_spd_inverse(nf, A, Out);
        }
        if (have) {
            if (mine)
                for (int j = 0; j < nf; ++j) F.cov[lane * nf + j] = Out[lane * nf + j];
            __syncwarp();
            const double ge = mine ? F.gext[lane] : 0.0;
            double cg = 0.0;
            if (mine)
                for (int j = 0; j < nf; ++j) cg += F.cov[lane * nf + j] * __shfl_sync(0xffffffffu, ge, j);
            else
                for (int j = 0; j < nf; ++j) (void)__shfl_sync(0xffffffffu, ge, j);
            const double edm = 0.5 * wsum(mine ? ge * cg : 0.0);
            if (lane == 0) F.edm = edm;
        }
        // (without a positive-definite Hessian the BFGS covariance set before stays)
        if (mine) F.err[lane] = sqrt(fmax(F.cov[lane * nf + lane], 0.0));
        done_status = NLL_OK;
    }

    if (finish) {
        // covariance from the BFGS matrix in external coordinates, C = J V J
        const double Ji = mine ? jac(c, lane, F.x[lane]) : 0.0;
        for (int j = 0; j < nf; ++j) {
            const double Jj = __shfl_sync(0xffffffffu, Ji, j);
            if (mine) F.cov[lane * nf + j] = Ji * F.V[lane * nf + j] * Jj;
        }
        __syncwarp();
        if (mine) F.err[lane] = sqrt(fmax(F.cov[lane * nf + lane], 0.0));
        if (c.hessian) {
            if (mine) {
                double sd = F.err[lane];
                if (!(sd > 0.0)) sd = F.sint[lane];
                F.hstep[lane] = 1e-3 * sd;
            }
            if (lane == 0) F.phase = kPhHess;
        } else {
            done_status = NLL_OK;
        }
    }
    __syncwarp();  // every lane's writes to F come before the flag below
    if (done_status >= 0 && lane == 0) {
        F.status = done_status;
        F.phase = kPhDone;
        // a host thread that sees the done flag may collect this fit's state from another
        // stream while later steps run: make the state visible first
        __threadfence_system();
        atomicSub(b.n_active, 1);
        if (b.done_flags) b.done_flags[t] = 1;
    }
}

// ---------------------------------------------------------------------------------
// analytic Hessian pass over all toys (paper Sec. 2.1): the start matrix of strategy 2,
// the covariance of hessian 2 / 3, and nll_batch_eval_hess.  The per-event work is the
// single-sample Hessian pass (hess_device.cuh) over (toy, 1024-event) units; a warp per
// toy then sums its units in order, assembles H (and W) and inverts.
// ---------------------------------------------------------------------------------

struct HessDev {
    int n_toys, mode, want_w2, n_units, nslots, lnp_slot, ncols;
    int subsample;              // the units cover part of each toy's events: scale the sums to all of them
    int single;                 // start matrices from the single-precision event pass
    int tail_begin, tail_count;  // slots summed while staging (HessLayout)
    int pass;                   // covariance modes: polish pass (0: the loop's final point)
    int* n_polish;              // covariance modes: toys still polishing after this pass (mapped)
    const int* sel;             // per toy: take part in this pass (NULL: every toy)
    const int64_t* ev_begin;
    const int64_t* ev_end;
    const double* sum_wdm;
    HEv ev;                     // columns and weights; n is set per unit
    ToyFit* fits;
    const double* thetas;       // kHmEval: [n_toys][npar]
    HConst* hc;                 // per toy
    HessTerms* ht;              // per toy
    int* hok;                   // per toy: parameter point valid
    const int* unit_toy;        // per unit
    const int64_t* unit_e0;     // per unit: first event
    const int* toy_u0;          // per toy: first unit
    const int* toy_nu;          // per toy: units
    double* unit_sums;          // [n_units][nslots]
    double* tot;                // per toy slot totals, [nslots][n_toys]
    double* asmb;               // per toy assembly, [kAsmEntries][n_toys]: nll, grad, H, W, bad
    const uint16_t* slot_of;    // [ncols][ncols] -> slot, 0xffff = none
    double* out;                // kHmEval: per toy nll, grad[np], H[np*np], W[np*np]
    int* status;                // kHmEval: per toy
    FitConfig cfg;
    uint8_t si[kHessMaxSlots], sj[kHessMaxSlots];
};

// thread per toy: the toy's parameter point and its parameter-only terms
__global__ void batch_hess_prep(HessDev h)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    // covariance modes: the count of toys that propose another polish step restarts with every
    // pass (the host reads it after the last pass it queued)
    if (t == 0 && (h.mode == kHmCov || h.mode == kHmSandwich)) *h.n_polish = 0;
    if (t >= h.n_toys) return;
    if (h.sel && !h.sel[t]) {
        h.hok[t] = 0;
        return;
    }
    const FitConfig& c = h.cfg;
    const int np = c.npar;
    double th[kNP];
    bool use = true;
    if (h.mode == kHmEval) {
        for (int k = 0; k < np; ++k) th[k] = h.thetas[(size_t)t * np + k];
    } else {
        const ToyFit& F = h.fits[t];
        for (int k = 0; k < np; ++k) th[k] = F.th[k];
        // covariance modes: the toys still polishing (set up by the host before pass 0)
        if (h.mode != kHmStart) use = F.pol > 0;
    }
    KConst kc;
    DConst dc;
    memset(&kc, 0, sizeof kc);
    memset(&dc, 0, sizeof dc);
    const bool ok = use && dev_hoist(c.kind, c.ranges, th, kc, dc, true);
    h.hok[t] = ok ? 1 : 0;
    if (!ok) return;
    HConst hc;
    memset(&hc, 0, sizeof hc);
    hc.mu = dc.mu;
    hc.b0 = dc.b0;
    hc.neg_b0s = kc.neg_b0;
    hc.neg_als = kc.neg_alpha;
    hc.k0s = kc.k0;
    hc.b2 = dc.b2;
    hc.inv_sigma = 1.0 / dc.sigma;
    hc.dlnN1_dmu = dc.dlnN1_dmu;
    hc.dlnN1_dsig = dc.dlnN1_dsig;
    hc.mu_ma = dc.mu - dc.ma;
    hc.dlnN2t_dal = dc.dlnN2t_dal;
    hc.inv_f = 1.0 / dc.f;
    hc.inv_1mf = 1.0 / (1.0 - dc.f);
    if (c.kind == kKstar4D) {
        for (int k = 0; k < 8; ++k) hc.ang[k] = th[2 + k];
        for (int j = 0; j < 3; ++j) {
            hc.c1[j] = th[11 + 2 * j];
            hc.c2[j] = th[12 + 2 * j];
            hc.dl[j] = dc.dlnNc[j];
        }
    }
    h.hc[t] = hc;
    HessTerms T;
    T.alpha = dc.alpha;
    T.f = dc.f;
    T.sigma = dc.sigma;
    T.b0 = dc.b0;
    for (int k = 0; k < 3; ++k) {
        T.d2lnN1[k] = dc.d2lnN1[k];
        T.dlnNc_dc2[k] = dc.dlnNc[k];
    }
    T.d2lnN2t_dal2 = dc.d2lnN2t_dal2;
    h.ht[t] = T;
}

// persistent blocks over units: unit u covers events [e0, min(e0 + kHessUnitEvents, end)) of its toy
template <int KIND, int VAR, bool W>
__global__ void __launch_bounds__(kHessThreads) batch_hess_units(const HessDev h)
{
    extern __shared__ double z[];
    __shared__ double s_tab[(KIND == kKstar4D && VAR == kVarDirect) ? kTabDoubles : (W ? kTrigOffset : kExpTable)];
    constexpr int TM = HessTailMax<KIND>::value;
    __shared__ HConst s_c;
    __shared__ double s_lnp[kHessThreads / 32];
    __shared__ double s_tred[(kHessThreads / 32) * TM];
    __shared__ uint8_t s_ti[TM], s_tj[TM];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    constexpr int ntab = (KIND == kKstar4D && VAR == kVarDirect) ? kTabDoubles : (W ? kTrigOffset : kExpTable);
    for (int j = t; j < ntab; j += kHessThreads) s_tab[j] = g_btab[j];
    const int ns = h.nslots;
    // tail slots [tb, tb + tn): summed by each event's staging thread (as in hess_kernel; the
    // mass model's whole table)
    const int tb = h.tail_begin, tn = h.tail_count;
    if (t < TM) {
        const int sr = t < tn ? tb + t : 0;
        s_ti[t] = h.si[sr];
        s_tj[t] = h.sj[sr];
    }
    const int ns_rows = (tn > 0 && tb + tn == ns) ? tb : ns;
    const int w0 = t & ~31;
    const int nrow = ns_rows > w0 ? min(3, (ns_rows - w0 + kHessThreads - 1) / kHessThreads) : 0;
    const int ls = h.lnp_slot;
    const bool lnp_in_tail = ls >= tb && ls < tb + tn;
    int ci[3], cj[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int sl = t + k * kHessThreads;
        const int sc = sl < ns ? sl : 0;
        ci[k] = h.si[sc];
        cj[k] = h.sj[sc];
    }
    for (int u = blockIdx.x; u < h.n_units; u += gridDim.x) {
        const int toy = h.unit_toy[u];
        const bool ok = h.hok[toy] != 0;  // uniform over the block
        __syncthreads();                  // s_c and z of the previous unit are no longer read
        if (t == 0 && ok) s_c = h.hc[toy];
        HEv ev = h.ev;
        const int64_t e0 = h.unit_e0[u];
        ev.n = min(e0 + (int64_t)kHessUnitEvents, h.ev_end[toy]);
        __syncthreads();
        double acc[3] = {0.0, 0.0, 0.0};
        double tacc[TM];
#pragma unroll
        for (int r = 0; r < TM; ++r) tacc[r] = 0.0;
        LogProd lp{1.0, 0};
        double lnp_tot = 0.0;
        if (ok) {
            for (int64_t e = e0; e < ev.n; e += kHessThreads) {
                stage_event<KIND, VAR, W>(ev, s_c, e + t, z, t, s_tab, lp);
#pragma unroll
                for (int r = 0; r < TM; ++r)  // this thread's own event, just staged
                    if (r < tn) tacc[r] = fma(z[s_ti[r] * kHessThreads + t], z[s_tj[r] * kHessThreads + t], tacc[r]);
                if (ns_rows > 0) {  // the tile's warp rows read every thread's columns
                    __syncthreads();
                    if (nrow == 1)
                        tile_slots<1>(z, ci, cj, acc, lane);
                    else if (nrow == 2)
                        tile_slots<2>(z, ci, cj, acc, lane);
                    else if (nrow == 3)
                        tile_slots<3>(z, ci, cj, acc, lane);
                    __syncthreads();
                }
            }
            if (!W) {  // sum over the block of ln(products) into the ln P slot
                double v = logprod_value(lp);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (lane == 0) s_lnp[warp] = v;
                __syncthreads();
                lnp_tot = (s_lnp[0] + s_lnp[1]) + (s_lnp[2] + s_lnp[3]);
                if (ls >= 0 && !lnp_in_tail && t == (ls & (kHessThreads - 1))) {
                    const double tot = lnp_tot;
                    const int row = ls / kHessThreads;
                    if (row == 0)
                        acc[0] += tot;
                    else if (row == 1)
                        acc[1] += tot;
                    else
                        acc[2] += tot;
                }
            }
        }
        if (tn > 0) {  // tail slots: fixed tree over the block (slot tb + t in thread t)
            double tot = block_reduce<TM>(tacc, s_tred);
            if (t < tn) {
                if (!W && tb + t == ls) tot += lnp_tot;
                h.unit_sums[(size_t)u * ns + tb + t] = tot;
            }
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int sl = t + k * kHessThreads;
            if (sl < ns && !(sl >= tb && sl < tb + tn)) h.unit_sums[(size_t)u * ns + sl] = acc[k];
        }
    }
}

// The same pass in single precision (start matrices only, HessDev::single): staging, slot
// products and the per-unit sums in float, the unit sums stored as doubles for the (double)
// totals and assembly.  The ln P column is zero, so the NLL it gives is not the sample's; the
// start matrix needs H and the gradient only.
template <int KIND, int VAR, bool W>
__global__ void __launch_bounds__(kHessThreads) batch_hess32_units(const HessDev h)
{
    constexpr int TM = HessTailMax<KIND>::value;
    extern __shared__ float z32[];
    __shared__ HConst32 s_c;
    __shared__ double s_tred[(kHessThreads / 32) * TM];
    __shared__ uint8_t s_ti[TM], s_tj[TM];
    const int t = threadIdx.x, lane = t & 31;
    const int ns = h.nslots;
    const int tb = h.tail_begin, tn = h.tail_count;
    if (t < TM) {
        const int sr = t < tn ? tb + t : 0;
        s_ti[t] = h.si[sr];
        s_tj[t] = h.sj[sr];
    }
    const int ns_rows = (tn > 0 && tb + tn == ns) ? tb : ns;
    const int w0 = t & ~31;
    const int nrow = ns_rows > w0 ? min(3, (ns_rows - w0 + kHessThreads - 1) / kHessThreads) : 0;
    int ci[3], cj[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int sl = t + k * kHessThreads;
        const int sc = sl < ns ? sl : 0;
        ci[k] = h.si[sc];
        cj[k] = h.sj[sc];
    }
    for (int u = blockIdx.x; u < h.n_units; u += gridDim.x) {
        const int toy = h.unit_toy[u];
        const bool ok = h.hok[toy] != 0;  // uniform over the block
        __syncthreads();                  // s_c and z32 of the previous unit are no longer read
        if (t == 0 && ok) s_c = to_single(h.hc[toy]);
        HEv ev = h.ev;
        const int64_t e0 = h.unit_e0[u];
        ev.n = min(e0 + (int64_t)kHessUnitEvents, h.ev_end[toy]);
        __syncthreads();
        float acc[3] = {0.0f, 0.0f, 0.0f};
        float tacc[TM];
#pragma unroll
        for (int r = 0; r < TM; ++r) tacc[r] = 0.0f;
        if (ok) {
            for (int64_t e = e0; e < ev.n; e += kHessThreads) {
                stage_event32<KIND, VAR, W>(ev, s_c, e + t, z32, t);
#pragma unroll
                for (int r = 0; r < TM; ++r)
                    if (r < tn) tacc[r] = fmaf(z32[s_ti[r] * kHessThreads + t], z32[s_tj[r] * kHessThreads + t], tacc[r]);
                if (ns_rows > 0) {
                    __syncthreads();
                    if (nrow == 1)
                        tile_slots32<1>(z32, ci, cj, acc, lane);
                    else if (nrow == 2)
                        tile_slots32<2>(z32, ci, cj, acc, lane);
                    else if (nrow == 3)
                        tile_slots32<3>(z32, ci, cj, acc, lane);
                    __syncthreads();
                }
            }
        }
        if (tn > 0) {  // per-thread float sums, then the block tree in double
            double td[TM];
#pragma unroll
            for (int r = 0; r < TM; ++r) td[r] = (double)tacc[r];
            const double tot = block_reduce<TM>(td, s_tred);
            if (t < tn) h.unit_sums[(size_t)u * ns + tb + t] = tot;
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int sl = t + k * kHessThreads;
            if (sl < ns && !(sl >= tb && sl < tb + tn)) h.unit_sums[(size_t)u * ns + sl] = (double)acc[k];
        }
    }
}

// Newton polish helpers (warp per toy).  propose: the point th_acc - lam d, halving lam until
// every bounded parameter stays inside its bounds; reject: halve lam and propose again, or stop
// at the accepted point once the step is negligible.
__device__ void polish_propose(const HessDev& h, ToyFit& F, int lane)
{
    const FitConfig& c = h.cfg;
    const int nf = c.nf;
    double lam = F.lam;
    bool inside = false;
    for (int tries = 0; tries < 40 && !inside; ++tries) {
        int out = 0;
        if (lane < nf) {
            const int k = c.idx[lane];
            const double v = F.th_acc[k] - lam * F.dN[lane];
            out = c.bounded[k] && !(v > c.lo[k] && v < c.hi[k]);
        }
        inside = __all_sync(0xffffffffu, out == 0);
        if (!inside) lam *= 0.5;
    }
    if (!inside || lam < 1e-6) {  // no admissible step: stay at the accepted point
        for (int k = lane; k < c.npar; k += 32) F.th[k] = F.th_acc[k];
        if (lane == 0) F.pol = 0;
        return;
    }
    for (int k = lane; k < c.npar; k += 32) F.th[k] = F.th_acc[k];
    __syncwarp();
    if (lane < nf) F.th[c.idx[lane]] = F.th_acc[c.idx[lane]] - lam * F.dN[lane];
    if (lane == 0) {
        F.lam = lam;
        F.pol = 1;
        atomicAdd(h.n_polish, 1);
    }
}

__device__ void polish_reject(const HessDev& h, ToyFit& F, int lane)
{
    if (h.pass == 0) {  // the loop's own final point failed here: nothing to step from
        if (lane == 0) {
            F.pol = 0;
            F.n_eval += 1;
        }
        return;
    }
    if (lane == 0) {
        F.lam *= 0.5;
        F.n_eval += 1;
    }
    __syncwarp();
    polish_propose(h, F, lane);
}

// thread per toy: toys that finished the loop at a parameter point (converged, or stopped by a
// stalled line search or the iteration limit) are polished; after the last pass a toy still
// polishing returns to its accepted point
// Every toy's fit state set up on the device (block per toy): zeroed, then the start state
// from th0 (one shared point, or n x npar) and the steps (or NULL).
static_assert(sizeof(ToyFit) % 8 == 0, "ToyFit is zeroed as 64-bit words");
// Start state of one toy's fit (F zeroed by the caller): transformed start point and
// internal steps.  Host (served fits) and device (batched fits) share it.
__host__ __device__ void init_fit_fields(ToyFit& F, const FitConfig& c, const double* th0, const double* step)
{
    for (int k = 0; k < c.npar; ++k) F.th[k] = th0[k];
    for (int i = 0; i < c.nf; ++i) {
        const int k = c.idx[i];
        double x = th0[k];
        double J = 1.0;
        if (c.bounded[k]) {
            double u = 2.0 * (x - c.lo[k]) / (c.hi[k] - c.lo[k]) - 1.0;
            u = fmin(fmax(u, -1.0 + 1e-10), 1.0 - 1e-10);
            x = asin(u);
            J = (c.hi[k] - c.lo[k]) * 0.5 * cos(x);
        }
        F.xt[i] = x;
        double s0 = step && step[k] > 0.0 ? step[k] : fmax(1e-3 * fabs(th0[k]), 1e-3);
        double si = s0 / fmax(fabs(J), 1e-8);
        if (c.bounded[k]) si = fmin(si, 0.5);
        F.sint[i] = si;
    }
    F.phase = kPhInit;
    F.status = NLL_ERR_NOT_CONVERGED;
    for (int s = 0; s < kMaxSlots; ++s) F.item[s] = -1;
}

__global__ void __launch_bounds__(128) batch_init_fits(ToyFit* fits, int n, const FitConfig c, const double* th0,
                                                       int shared, const double* step)
{
    const int t = blockIdx.x;
    if (t >= n) return;
    unsigned long long* w = reinterpret_cast<unsigned long long*>(fits + t);
    for (int i = threadIdx.x; i < (int)(sizeof(ToyFit) / 8); i += blockDim.x) w[i] = 0ull;
    __syncthreads();
    if (threadIdx.x == 0) init_fit_fields(fits[t], c, shared ? th0 : th0 + (size_t)t * c.npar, step);
}

// The results of nll_batch_fit_arrays, written by the device straight into the caller's
// arrays (block per toy; each toy's rows are contiguous), laid out as that call documents.
struct ArrayOut {
    double* theta;
    double* err;
    double* cov;
    double* nll;
    double* edm;
    int* n_eval;
    int* n_iter;
    int* status;
};

__global__ void __launch_bounds__(128) batch_write_arrays(const ToyFit* fits, int n, const FitConfig c, ArrayOut o)
{
    __shared__ int s_inv[kNP];  // parameter -> free index, -1 for a fixed one
    const int t = blockIdx.x;
    if (t >= n) return;
    const ToyFit& F = fits[t];
    const int np = c.npar, nf = c.nf;
    for (int k = threadIdx.x; k < np; k += blockDim.x) s_inv[k] = -1;
    __syncthreads();
    for (int i = threadIdx.x; i < nf; i += blockDim.x) s_inv[c.idx[i]] = i;
    __syncthreads();
    for (int k = threadIdx.x; k < np; k += blockDim.x) {
        if (o.theta) o.theta[(size_t)t * np + k] = F.th[k];
        if (o.err) o.err[(size_t)t * np + k] = s_inv[k] >= 0 ? F.err[s_inv[k]] : 0.0;
    }
    if (o.cov)
        for (int q = threadIdx.x; q < np * np; q += blockDim.x) {
            const int ia = s_inv[q / np], ib = s_inv[q % np];
            o.cov[(size_t)t * np * np + q] = (ia >= 0 && ib >= 0) ? F.cov[ia * nf + ib] : 0.0;
        }
    if (threadIdx.x == 0) {
        if (o.nll) o.nll[t] = F.f;
        if (o.edm) o.edm[t] = F.edm;
        if (o.n_eval) o.n_eval[t] = F.n_eval;
        if (o.n_iter) o.n_iter[t] = F.iter;
        if (o.status) o.status[t] = F.phase == kPhDone ? F.status : NLL_ERR_NOT_CONVERGED;
    }
}

// Results of every toy packed for the host (block per toy), kResStride doubles each:
// th[npar] | err[nf] | cov[nf x nf] (free parameters) | nll, edm, n_eval, n_iter, status.
__global__ void __launch_bounds__(128) batch_pack_results(const ToyFit* fits, const int* idx, int n, int np, int nf,
                                                          double* res)
{
    const int t = blockIdx.x;
    if (t >= n) return;
    const ToyFit& F = fits[idx ? idx[t] : t];
    double* r = res + (size_t)t * kResStride;
    for (int i = threadIdx.x; i < np; i += blockDim.x) r[i] = F.th[i];
    for (int i = threadIdx.x; i < nf; i += blockDim.x) r[kNP + i] = F.err[i];
    for (int i = threadIdx.x; i < nf * nf; i += blockDim.x) r[2 * kNP + i] = F.cov[i];
    if (threadIdx.x == 0) {
        double* tail = r + 2 * kNP + kNP * kNP;
        tail[0] = F.f;
        tail[1] = F.edm;
        tail[2] = (double)F.n_eval;
        tail[3] = (double)F.iter;
        tail[4] = (double)(F.phase == kPhDone ? F.status : NLL_ERR_NOT_CONVERGED);
    }
}

__global__ void batch_polish_init(ToyFit* fits, int n, const int* sel)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n || (sel && !sel[t])) return;
    ToyFit& F = fits[t];
    const bool go = F.phase == kPhDone && (F.status == NLL_OK || F.status == NLL_ERR_NOT_CONVERGED);
    F.pol = go ? 1 : 0;
    F.lam = 1.0;
    F.f_acc = F.f;
    for (int k = 0; k < kNP; ++k) F.th_acc[k] = F.th[k];
}

__global__ void batch_polish_close(ToyFit* fits, int n, int npar, const int* sel)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n || (sel && !sel[t])) return;
    ToyFit& F = fits[t];
    if (F.pol > 0) {
        for (int k = 0; k < npar; ++k) F.th[k] = F.th_acc[k];
        F.f = F.f_acc;
        F.pol = 0;
    }
}

// a toy whose sums this pass assembles: selected, still polishing (covariance modes) and at a
// valid parameter point
__device__ __forceinline__ bool hess_toy_assembled(const HessDev& h, int t)
{
    if (h.sel && !h.sel[t]) return false;
    if ((h.mode == kHmCov || h.mode == kHmSandwich) && h.fits[t].pol <= 0) return false;
    return h.hok[t] != 0;
}

// warp per toy: the toy's slot totals, its units added in order (lanes over slots), stored
// slot-major so that the assembly reads them coalesced
__global__ void __launch_bounds__(128) batch_hess_totals(const HessDev h)
{
    const int lane = threadIdx.x & 31;
    const int t = blockIdx.x * 4 + (threadIdx.x >> 5);
    if (t >= h.n_toys || !hess_toy_assembled(h, t)) return;
    const int u0 = h.toy_u0[t], nu = h.toy_nu[t];
    double scale = 1.0;
    if (h.subsample) {  // events of the toy over events in its units (a start matrix only)
        int64_t covered = 0;
        for (int j = 0; j < nu; ++j) covered += min((int64_t)kHessUnitEvents, h.ev_end[t] - h.unit_e0[u0 + j]);
        if (covered > 0) scale = (double)(h.ev_end[t] - h.ev_begin[t]) / (double)covered;
    }
    for (int sl = lane; sl < h.nslots; sl += 32) {
        double v = 0.0;
        for (int j = 0; j < nu; ++j) v += h.unit_sums[(size_t)(u0 + j) * h.nslots + sl];
        h.tot[(size_t)sl * h.n_toys + t] = v * scale;
    }
}

// column of an entry-major per-toy array: element i of toy t at p[i * stride]
struct Strided {
    double* p;
    int stride;
    __device__ double& operator[](int i) const { return p[(size_t)i * stride]; }
};

// slot totals of the block's toys staged in shared memory ([slot][toy]) and the
// (column pair -> slot) table after them
struct StagedSlots {
    const double* tot;  // this toy's first total; slot s at tot[s * stride]
    int stride;
    const uint16_t* slot_of;
    int nc;
    __device__ double operator()(int i, int j) const
    {
        const unsigned s = slot_of[i * nc + j];
        return s == 0xffffu ? NAN : tot[(size_t)s * stride];
    }
};

// Shared memory of batch_hess_assemble stays within the 48 KB every kernel may take without
// opting in: a kernel that needs a larger shared-memory carve-out cannot start on an SM that
// runs blocks of other kernels under a smaller one, so it would wait for idle SMs behind the
// fit loop's (or a server's step) kernels.  The block therefore takes as many toys as the
// table allows: 32 for the 4D table without W (195 slots), fewer with W.
constexpr int kAsmSmemMax = 48 * 1024;
constexpr int kAsmWarps = 4;

size_t asm_smem(int nslots, int ncols, int tpb)
{
    return (((size_t)nslots * tpb * sizeof(double) + 15) / 16) * 16 + ((ncols * ncols * 2 + 15) / 16) * 16;
}

int asm_toys_per_block(int nslots, int ncols)
{
    for (int tpb : {32, 24, 16, 12, 8, 4})
        if (asm_smem(nslots, ncols, tpb) <= (size_t)kAsmSmemMax) return tpb;
    return 2;  // (the largest table, 384 slots of 64 columns, fits 12)
}

// a block per tpb toys, thread per toy (lanes 0 .. tpb-1 of each warp): NLL, gradient, H (and
// W) from the totals, the single-sample assembly.  A thread per toy runs each FP64 instruction
// for up to 32 toys at once, where a lane per toy would occupy the FP64 pipe for a whole warp
// instruction per toy; the totals and the slot table are staged in shared memory first
// (coalesced, independent loads), and the block's kAsmWarps warps take every kAsmWarps-th row
// of H each (the assembly is bound by instruction issue, not by the FP64 pipe).
template <int KIND, bool W>
__global__ void __launch_bounds__(kAsmWarps * 32) batch_hess_assemble(const HessDev h, int tpb)
{
    using L = HCols<KIND, W>;
    constexpr int NP = L::NP;
    extern __shared__ double sm[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, n = h.n_toys, ns = h.nslots, nc = h.ncols;
    const int t = blockIdx.x * tpb + lane;
    const bool use = lane < tpb && t < n && hess_toy_assembled(h, t);
    uint16_t* s_slot = reinterpret_cast<uint16_t*>(sm + (((size_t)ns * tpb + 1) / 2) * 2);
    const int nv = (nc * nc + 7) / 8;  // whole 16-byte vectors of the table (64 x 64 allocated)
    for (int k = threadIdx.x; k < nv; k += kAsmWarps * 32)
        reinterpret_cast<uint4*>(s_slot)[k] = reinterpret_cast<const uint4*>(h.slot_of)[k];
    if (lane < tpb) {
#pragma unroll 4
        for (int sl = warp; sl < ns; sl += kAsmWarps) sm[sl * tpb + lane] = use ? h.tot[(size_t)sl * n + t] : 0.0;
    }
    __syncthreads();
    if (!use) return;
    StagedSlots S{sm + lane, tpb, s_slot, nc};
    double* a = h.asmb + t;
    const double bad = assemble_t<KIND, W>(h.ht[t], h.sum_wdm[t], h.want_w2 != 0, S, Strided{a, n},
                                           Strided{a + (size_t)n, n}, Strided{a + (size_t)(1 + NP) * n, n},
                                           Strided{a + (size_t)(1 + NP + NP * NP) * n, n}, warp, kAsmWarps);
    if (warp == 0) a[(size_t)(1 + NP + 2 * NP * NP) * n] = (bad != 0.0 || !isfinite(a[0])) ? 1.0 : 0.0;
}

// warp per toy: the mode's matrix work on the assembled pass
// (two warps per block: 31 KB of static shared memory for the 18-parameter model)
constexpr int kFinWarps = 2;

// slot totals of one toy in shared memory, found through the (column pair -> slot) table
struct SumSlots {
    const double* sums;
    const uint16_t* slot_of;
    int nc;
    __device__ double operator()(int i, int j) const
    {
        const unsigned s = slot_of[i * nc + j];
        return s == 0xffffu ? NAN : sums[s];
    }
};

// SMALL (passes over at most kFinSmallToys toys, such as a server's collections): the toy's
// slot totals and its assembly are done here, by the toy's warp (totals) and lane 0 (assembly),
// instead of by batch_hess_totals and batch_hess_assemble: two launches fewer per pass, and for
// a few toys a lane's FP64 instructions cost little.  Both paths add the same unit sums in the
// same order and assemble with the same code.
constexpr int kFinSmallToys = 64;

template <int KIND, bool W, bool SMALL>
__global__ void __launch_bounds__(kFinWarps * 32) batch_hess_finish(const HessDev h)
{
    constexpr int NPK = KIND == kMass1D ? 4 : 18;
    __shared__ double s_sum[SMALL ? kFinWarps : 1][SMALL ? kHessMaxSlots : 1];
    __shared__ double s_H[kFinWarps][NPK * NPK];
    __shared__ double s_W[kFinWarps][NPK * NPK];
    __shared__ double s_mat[kFinWarps][4][NPK * NPK];
    __shared__ double s_g[kFinWarps][NPK];
    __shared__ double s_nll[kFinWarps];
    __shared__ int s_bad[kFinWarps];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int t = blockIdx.x * kFinWarps + wib;
    if (t >= h.n_toys) return;
    const FitConfig& c = h.cfg;
    const int np = c.npar, nf = c.nf;
    const bool mine = lane < nf;
    if (h.sel && !h.sel[t]) return;
    const bool polish = h.mode == kHmCov || h.mode == kHmSandwich;
    if (polish && h.fits[t].pol <= 0) return;
    if (!h.hok[t] && polish) {  // the proposed point is not a valid parameter point: shorter step
        polish_reject(h, h.fits[t], lane);
        return;
    }
    if (!h.hok[t]) {
        if (h.mode == kHmEval) {
            if (lane == 0) h.status[t] = NLL_ERR_ARG;
            double* o = h.out + (size_t)t * (1 + np + 2 * np * np);
            for (int k = lane; k < 1 + np + 2 * np * np; k += 32) o[k] = k == 0 ? INFINITY : NAN;
        }
        return;
    }
    if (SMALL) {
        const int u0 = h.toy_u0[t], nu = h.toy_nu[t];
        double scale = 1.0;
        if (h.subsample) {  // events of the toy over events in its units (a start matrix only)
            int64_t covered = 0;
            for (int j = 0; j < nu; ++j) covered += min((int64_t)kHessUnitEvents, h.ev_end[t] - h.unit_e0[u0 + j]);
            if (covered > 0) scale = (double)(h.ev_end[t] - h.ev_begin[t]) / (double)covered;
        }
        for (int sl = lane; sl < h.nslots; sl += 32) {
            double v = 0.0;
            for (int j = 0; j < nu; ++j) v += h.unit_sums[(size_t)(u0 + j) * h.nslots + sl];
            s_sum[wib][sl] = v * scale;
        }
        __syncwarp();
        if (lane == 0) {
            SumSlots S{s_sum[wib], h.slot_of, h.ncols};
            const double bad = assemble_t<KIND, W>(h.ht[t], h.sum_wdm[t], h.want_w2 != 0, S, &s_nll[wib], s_g[wib],
                                                   s_H[wib], s_W[wib]);
            s_bad[wib] = (bad != 0.0 || !isfinite(s_nll[wib])) ? 1 : 0;
        }
    } else {
        const int n = h.n_toys;
        const double* a = h.asmb + t;
        for (int k = lane; k < NPK; k += 32) s_g[wib][k] = a[(size_t)(1 + k) * n];
#pragma unroll 4
        for (int k = lane; k < NPK * NPK; k += 32) {
            s_H[wib][k] = a[(size_t)(1 + NPK + k) * n];
            if (h.want_w2) s_W[wib][k] = a[(size_t)(1 + NPK + NPK * NPK + k) * n];
        }
        if (lane == 0) {
            s_nll[wib] = a[0];
            s_bad[wib] = a[(size_t)(1 + NPK + 2 * NPK * NPK) * n] != 0.0;
        }
    }
    __syncwarp();
    const bool bad = s_bad[wib] != 0;
    if (h.mode == kHmEval) {
        double* o = h.out + (size_t)t * (1 + np + 2 * np * np);
        if (lane == 0) {
            h.status[t] = bad ? NLL_ERR_NONPOSITIVE_PDF : NLL_OK;
            o[0] = bad ? INFINITY : s_nll[wib];
        }
        for (int k = lane; k < np; k += 32) o[1 + k] = bad ? NAN : s_g[wib][k];
        for (int k = lane; k < np * np; k += 32) {
            o[1 + np + k] = bad ? NAN : s_H[wib][k];
            o[1 + np + np * np + k] = (bad || !h.want_w2) ? NAN : s_W[wib][k];
        }
        return;
    }
    ToyFit& F = h.fits[t];
    if (bad) {  // start: keep the diagonal start matrix; polish: a shorter step
        if (polish) polish_reject(h, F, lane);
        return;
    }
    double* A = s_mat[wib][0];
    double* Lm = s_mat[wib][1];
    double* Mm = s_mat[wib][2];
    double* Out = s_mat[wib][3];
    if (mine)
        for (int j = 0; j < nf; ++j) A[lane * nf + j] = s_H[wib][c.idx[lane] * np + c.idx[j]];
    __syncwarp();
    if (h.mode == kHmStart) {
        // internal coordinates: J H J + diag(dNLL/dext d2ext/dx2) (sine transform)
        const double xi = mine ? F.xt[lane] : 0.0;
        const double Ji = mine ? jac(c, lane, xi) : 0.0;
        for (int j = 0; j < nf; ++j) {
            const double Jj = __shfl_sync(0xffffffffu, Ji, j);
            if (mine) A[lane * nf + j] *= Ji * Jj;
        }
        if (mine && c.bounded[c.idx[lane]]) {
            const int k = c.idx[lane];
            A[lane * nf + lane] += s_g[wib][k] * (-(c.hi[k] - c.lo[k]) * 0.5 * sin(xi));
        }
        __syncwarp();
        if (warp_spd_inverse(nf, A, Out)) {
            if (mine)
                for (int j = 0; j < nf; ++j) F.V[lane * nf + j] = Out[lane * nf + j];
            if (lane == 0) F.vset = 1;
            __syncwarp();
            // the pass gave the NLL and gradient at the start point as well: the first step is
            // taken from them here, so that the fit loop starts with the first trial point (a
            // subsampled or single-precision pass gives estimates only)
            if (!h.subsample && !h.single)
                begin_search(c, F, s_nll[wib], mine ? s_g[wib][c.idx[lane]] : 0.0, true, true, lane);
        }
        if (lane == 0) F.n_eval += 1;
        return;
    }
    // Newton polish step (as the single-sample minimiser): accept the point if the NLL did not
    // rise, take H^-1 (or H^-1 W H^-1) there as the covariance, stop when the EDM with H is
    // below the tolerance, else propose the Newton step from the accepted point
    const double fnew = s_nll[wib];
    const bool accept = h.pass == 0 || fnew <= F.f_acc + 1e-15 * fabs(F.f_acc);
    if (!accept) {
        polish_reject(h, F, lane);
        return;
    }
    const bool inv = warp_spd_inverse(nf, A, Out);
    if (lane == 0) F.n_eval += 1;
    if (!inv) {  // no positive-definite Hessian here: the last covariance stays, stop
        if (lane == 0) F.pol = 0;
        return;
    }
    if (h.mode == kHmSandwich) {
        double* Wf = Lm;  // reuse: W (free block), then T = Hi W
        if (mine)
            for (int j = 0; j < nf; ++j) Wf[lane * nf + j] = s_W[wib][c.idx[lane] * np + c.idx[j]];
        __syncwarp();
        if (mine)
            for (int j = 0; j < nf; ++j) {
                double acc = 0.0;
                for (int k = 0; k < nf; ++k) acc += Out[lane * nf + k] * Wf[k * nf + j];
                Mm[lane * nf + j] = acc;
            }
        __syncwarp();
        if (mine)
            for (int j = 0; j < nf; ++j) {
                double acc = 0.0;
                for (int k = 0; k < nf; ++k) acc += Mm[lane * nf + k] * Out[k * nf + j];
                F.cov[lane * nf + j] = acc;
            }
    } else if (mine) {
        for (int j = 0; j < nf; ++j) F.cov[lane * nf + j] = Out[lane * nf + j];
    }
    // accepted point: gradient, EDM with H, Newton direction d = H^-1 g
    const double ge = mine ? s_g[wib][c.idx[lane]] : 0.0;
    double hg = 0.0;
    if (mine)
        for (int j = 0; j < nf; ++j) hg += Out[lane * nf + j] * __shfl_sync(0xffffffffu, ge, j);
    else
        for (int j = 0; j < nf; ++j) (void)__shfl_sync(0xffffffffu, ge, j);
    const double edm = 0.5 * wsum(mine ? ge * hg : 0.0);
    if (mine) {
        F.err[lane] = sqrt(fmax(F.cov[lane * nf + lane], 0.0));
        F.gext[lane] = ge;
        F.dN[lane] = hg;
    }
    for (int k = lane; k < np; k += 32) F.th_acc[k] = F.th[k];
    if (lane == 0) {
        F.edm = edm;
        F.f = fnew;
        F.f_acc = fnew;
        F.lam = 1.0;
    }
    __syncwarp();
    if (edm < c.tol_edm) {
        if (lane == 0) {
            F.status = NLL_OK;
            F.pol = 0;
        }
        return;
    }
    polish_propose(h, F, lane);
}

template <int KIND, int VAR, bool W>
size_t hess_units_smem()
{
    return (size_t)HCols<KIND, W>::NC * kHessThreads * sizeof(double);
}

template <int KIND, int VAR, bool W>
cudaError_t launch_hess_units_t(int blocks, cudaStream_t s, const HessDev& h)
{
    const size_t smem = hess_units_smem<KIND, VAR, W>();
    cudaError_t e =
        cudaFuncSetAttribute(batch_hess_units<KIND, VAR, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    batch_hess_units<KIND, VAR, W><<<blocks, kHessThreads, smem, s>>>(h);
    return cudaGetLastError();
}

template <int KIND, int VAR, bool W>
cudaError_t launch_hess32_units_t(int blocks, cudaStream_t s, const HessDev& h)
{
    const size_t smem = (size_t)HCols<KIND, W>::NC * kHessThreads * sizeof(float);  // below 48 KB
    batch_hess32_units<KIND, VAR, W><<<blocks, kHessThreads, smem, s>>>(h);
    return cudaGetLastError();
}

cudaError_t launch_hess_pass(int kind, int var, bool w, int unit_blocks, cudaStream_t s, const HessDev& h)
{
    batch_hess_prep<<<(h.n_toys + 31) / 32, 32, 0, s>>>(h);  // a warp per block: see launch_step
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (h.n_units > 0 && h.single) {
        if (kind == kMass1D)
            e = w ? launch_hess32_units_t<kMass1D, kVarPrecompute, true>(unit_blocks, s, h)
                  : launch_hess32_units_t<kMass1D, kVarPrecompute, false>(unit_blocks, s, h);
        else if (var == kVarDirect)
            e = w ? launch_hess32_units_t<kKstar4D, kVarDirect, true>(unit_blocks, s, h)
                  : launch_hess32_units_t<kKstar4D, kVarDirect, false>(unit_blocks, s, h);
        else
            e = w ? launch_hess32_units_t<kKstar4D, kVarPrecompute, true>(unit_blocks, s, h)
                  : launch_hess32_units_t<kKstar4D, kVarPrecompute, false>(unit_blocks, s, h);
        if (e != cudaSuccess) return e;
    } else if (h.n_units > 0) {
        if (kind == kMass1D)
            e = w ? launch_hess_units_t<kMass1D, kVarPrecompute, true>(unit_blocks, s, h)
                  : launch_hess_units_t<kMass1D, kVarPrecompute, false>(unit_blocks, s, h);
        else if (var == kVarDirect)
            e = w ? launch_hess_units_t<kKstar4D, kVarDirect, true>(unit_blocks, s, h)
                  : launch_hess_units_t<kKstar4D, kVarDirect, false>(unit_blocks, s, h);
        else
            e = w ? launch_hess_units_t<kKstar4D, kVarPrecompute, true>(unit_blocks, s, h)
                  : launch_hess_units_t<kKstar4D, kVarPrecompute, false>(unit_blocks, s, h);
        if (e != cudaSuccess) return e;
    }
    const int fb = (h.n_toys + kFinWarps - 1) / kFinWarps;
    if (h.n_toys <= kFinSmallToys) {  // totals and assembly inside the finish
        if (kind == kMass1D)
            w ? batch_hess_finish<kMass1D, true, true><<<fb, kFinWarps * 32, 0, s>>>(h)
              : batch_hess_finish<kMass1D, false, true><<<fb, kFinWarps * 32, 0, s>>>(h);
        else
            w ? batch_hess_finish<kKstar4D, true, true><<<fb, kFinWarps * 32, 0, s>>>(h)
              : batch_hess_finish<kKstar4D, false, true><<<fb, kFinWarps * 32, 0, s>>>(h);
        return cudaGetLastError();
    }
    batch_hess_totals<<<(h.n_toys + 3) / 4, 128, 0, s>>>(h);
    const int tpb = asm_toys_per_block(h.nslots, h.ncols);
    const int ab = (h.n_toys + tpb - 1) / tpb, at = kAsmWarps * 32;
    const size_t asmem = asm_smem(h.nslots, h.ncols, tpb);
    if (kind == kMass1D)
        w ? batch_hess_assemble<kMass1D, true><<<ab, at, asmem, s>>>(h, tpb)
          : batch_hess_assemble<kMass1D, false><<<ab, at, asmem, s>>>(h, tpb);
    else
        w ? batch_hess_assemble<kKstar4D, true><<<ab, at, asmem, s>>>(h, tpb)
          : batch_hess_assemble<kKstar4D, false><<<ab, at, asmem, s>>>(h, tpb);
    if (kind == kMass1D) {
        if (w)
            batch_hess_finish<kMass1D, true, false><<<fb, kFinWarps * 32, 0, s>>>(h);
        else
            batch_hess_finish<kMass1D, false, false><<<fb, kFinWarps * 32, 0, s>>>(h);
    } else {
        if (w)
            batch_hess_finish<kKstar4D, true, false><<<fb, kFinWarps * 32, 0, s>>>(h);
        else
            batch_hess_finish<kKstar4D, false, false><<<fb, kFinWarps * 32, 0, s>>>(h);
    }
    return cudaGetLastError();
}

}  // namespace

template <int KIND, int VAR, bool W>
cudaError_t launch_eval_t(int blocks, cudaStream_t s, const BatchDev& b)
{
    batch_eval<KIND, VAR, W><<<blocks, kEvalThreads, 0, s>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_eval(int kind, int var, bool w, int blocks, cudaStream_t s, const BatchDev& b)
{
    if (kind == kMass1D) return w ? launch_eval_t<kMass1D, kVarPrecompute, true>(blocks, s, b)
                                  : launch_eval_t<kMass1D, kVarPrecompute, false>(blocks, s, b);
    if (var == kVarDirect) return w ? launch_eval_t<kKstar4D, kVarDirect, true>(blocks, s, b)
                                    : launch_eval_t<kKstar4D, kVarDirect, false>(blocks, s, b);
    return w ? launch_eval_t<kKstar4D, kVarPrecompute, true>(blocks, s, b)
             : launch_eval_t<kKstar4D, kVarPrecompute, false>(blocks, s, b);
}

namespace {
std::mutex g_btab_mutex;
bool g_btab_ready[64];
}  // namespace

cudaError_t ensure_btab(int device)
{
    std::lock_guard<std::mutex> lock(g_btab_mutex);
    if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
    if (g_btab_ready[device]) return cudaSuccess;
    std::vector<double> tab(kTabDoubles);
    fill_device_tables(tab.data());
    cudaError_t e = cudaMemcpyToSymbol(g_btab, tab.data(), sizeof(double) * kTabDoubles);
    if (e == cudaSuccess) g_btab_ready[device] = true;
    return e;
}

// End of one iteration of the device-resident fit loop (a while node of the fit graph): count
// the step and continue while some toy is still fitting and the step limit is not reached.
// One thread: the condition is set once per iteration.
// The tile of the next step: the schedule's, or a quarter of it once at most a quarter of the
// toys are still fitting (a unit of the schedule's tile keeps one SM busy for ~15 us of FP64
// work, so a few toys' units would leave most SMs idle).
__global__ void batch_loop_control(cudaGraphConditionalHandle handle, const int* n_active, int* steps, int max_steps,
                                   int* step_tp, int n_toys, int base_tp)
{
    const int s = *steps + 1;
    *steps = s;
    const int active = *(volatile const int*)n_active;
    *step_tp = (4 * active <= n_toys) ? max(base_tp / 4, 64) : base_tp;  // 64: the smallest tile the work arrays are sized for
    cudaGraphSetConditional(handle, (active > 0 && s < max_steps) ? 1u : 0u);
}

__global__ void batch_loop_init(int* steps, int* step_tp, int base_tp)
{
    *steps = 0;
    *step_tp = base_tp;
}

// One device step of the batched fit loop on stream s (for graph capture): reset the work
// counters, prepare (hoisting of every active toy's points), evaluate, update.
cudaError_t launch_step(const BatchDev& d, int var, bool weighted, int eval_blocks, cudaStream_t s)
{
    cudaError_t e = launch_step_eval(d, var, weighted, eval_blocks, s);
    return e == cudaSuccess ? launch_step_update(d, s) : e;
}

// The first part of a step: counters reset, prepare, evaluate.
cudaError_t launch_step_eval(const BatchDev& d, int var, bool weighted, int eval_blocks, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(d.counters, 0, sizeof(int) * 3, s);
    if (e != cudaSuccess) return e;
    // one warp per block: each toy's hoisting is a long dependent FP64 chain, so the warps go
    // to different SMs instead of sharing one SM's FP64 pipe
    batch_prepare<<<(d.n_toys + 31) / 32, 32, 0, s>>>(d);
    return launch_eval(d.cfg.kind, var, weighted, eval_blocks, s, d);
}

// The second part: every toy's minimiser advances.
cudaError_t launch_step_update(const BatchDev& d, cudaStream_t s)
{
    const int ub = (d.n_toys + kUpdWarps - 1) / kUpdWarps;
    if (d.cfg.kind == kMass1D)
        batch_update<kMass1D><<<ub, kUpdWarps * 32, 0, s>>>(d);
    else
        batch_update<kKstar4D><<<ub, kUpdWarps * 32, 0, s>>>(d);
    return cudaGetLastError();
}

// Results of n toys packed for the host, kResStride doubles each (batch_pack_results): toys
// idx[0..n) (device array), or 0 .. n-1 when idx is NULL.
cudaError_t launch_pack_results(const ToyFit* fits, const int* idx, int n, int np, int nf, double* res,
                                cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    batch_pack_results<<<n, 128, 0, s>>>(fits, idx, n, np, nf, res);
    return cudaGetLastError();
}

}  // namespace gbnll

using namespace gbnll;

// ------------------------------------------------------------------------------------
// host runtime
// ------------------------------------------------------------------------------------
namespace gbnll {


void hw_free(HessWork& w)
{
    if (w.staged_pending) cudaEventSynchronize(w.staged_ev);
    void* ptrs[] = {w.d_unit_toy, w.d_unit_e0, w.d_toy_u0, w.d_toy_nu, w.d_hc,    w.d_ht,     w.d_hok, w.d_unit_sums,
                    w.d_tot,      w.d_asm,    w.d_slot_of, w.d_thetas, w.d_out, w.d_status,  w.d_sel};
    for (void* p : ptrs)
        if (p) gb_free(p);
    void* hptrs[] = {w.h_npol, w.h_unit_toy, w.h_unit_e0, w.h_toy_u0, w.h_toy_nu, w.h_sel};
    for (void* p : hptrs)
        if (p) cudaFreeHost(p);
    if (w.staged_ev) cudaEventDestroy(w.staged_ev);
    DevBudget* budget = w.budget;
    w = HessWork();
    w.budget = budget;
}

cudaError_t hw_alloc(HessWork& w, int cap_toys, int cap_units, int np)
{
    hw_free(w);
    const size_t nt = std::max(cap_toys, 1), nu = std::max(cap_units, 1);
    cudaError_t e = gb_malloc(w.budget, &w.d_unit_toy, sizeof(int) * nu);
    if (e == cudaSuccess) e = gb_malloc(w.budget, &w.d_unit_e0, sizeof(int64_t) * nu);
    if (e == cudaSuccess) e = gb_malloc(w.budget, &w.d_toy_u0, sizeof(int) * nt);
    if (e == cudaSuccess) e = gb_malloc(w.budget, &w.d_toy_nu, sizeof(int) * nt);
    if (e == cudaSuccess) e = gb_malloc(w.budget, &w.d_hc, sizeof(HConst) * nt);
    if (e == cudaSuccess) e = gb_malloc(w.budget, &w.d_ht, sizeof(HessTerms) * nt);
    if (e == cudaSuccess) e = gb_malloc(w.budget, &w.d_hok, sizeof(int) * nt);
    if (e == cudaSuccess) e = gb_malloc(w.budget, &w.d_unit_sums, sizeof(double) * kHessMaxSlots * nu);
    if (e == cudaSuccess) e = gb_malloc(w.budget, &w.d_tot, sizeof(double) * kHessMaxSlots * nt);
    if (e == cudaSuccess) e = gb_malloc(w.budget, &w.d_asm, sizeof(double) * kAsmEntries * nt);
    if (e == cudaSuccess) e = gb_malloc(w.budget, &w.d_slot_of, sizeof(uint16_t) * 64 * 64);
    if (e == cudaSuccess) e = gb_malloc(w.budget, &w.d_thetas, sizeof(double) * np * nt);
    if (e == cudaSuccess) e = gb_malloc(w.budget, &w.d_out, sizeof(double) * (1 + np + 2 * np * np) * nt);
    if (e == cudaSuccess) e = gb_malloc(w.budget, &w.d_status, sizeof(int) * nt);
    if (e == cudaSuccess) e = gb_malloc(w.budget, &w.d_sel, sizeof(int) * nt);
    if (e == cudaSuccess) e = cudaHostAlloc(&w.h_npol, sizeof(int), cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer(&w.d_npol, w.h_npol, 0);
    // pinned staging of the unit lists, so that they can be copied without the host waiting
    if (e == cudaSuccess) e = cudaHostAlloc(&w.h_unit_toy, sizeof(int) * nu, cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaHostAlloc(&w.h_unit_e0, sizeof(int64_t) * nu, cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaHostAlloc(&w.h_toy_u0, sizeof(int) * nt, cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaHostAlloc(&w.h_toy_nu, sizeof(int) * nt, cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaHostAlloc(&w.h_sel, sizeof(int) * nt, cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&w.staged_ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        hw_free(w);
        return e;
    }
    w.cap_toys = (int)nt;
    w.cap_units = (int)nu;
    w.np = np;
    w.ready = true;
    return cudaSuccess;
}

// Unit lists for toys t with events [begin[t], end[t]) (host positions); toys with sel[t] == 0
// get no units (sel empty: every toy).  Fails if the units exceed the capacity.  The lists go
// through pinned staging; with wait the call returns once they are on the device, without it
// as soon as the copies are queued (the staging is reused only after they have completed).
// units of a toy with `total` units that a subsampled pass takes: the first 1024 events of a
// sample of up to 8192, else four 1024-event blocks spread evenly over the sample (so that a
// sample stored in some order still contributes from its whole range); at most kSubsampleMax
constexpr int kSubsampleBlock = 1024 / kHessUnitEvents;  // units per 1024-event block
constexpr int kSubsampleMax = 4 * kSubsampleBlock;
static_assert(1024 % kHessUnitEvents == 0, "1024-event blocks of whole units");
static int subsample_units(int64_t total, int64_t* pick)
{
    if (total <= 0) return 0;
    int k = 0;
    if (total <= 8 * kSubsampleBlock) {
        for (int j = 0; j < kSubsampleBlock && j < total; ++j) pick[k++] = j;
        return k;
    }
    for (int q = 0; q < 4; ++q) {
        const int64_t start = q * (total / 4);
        for (int j = 0; j < kSubsampleBlock && start + j < total; ++j) pick[k++] = start + j;
    }
    return k;
}

cudaError_t hw_set_units(HessWork& w, const std::vector<int64_t>& begin, const std::vector<int64_t>& end,
                         const std::vector<int>& sel, cudaStream_t stream, bool wait, bool subsample)
{
    const int n = (int)begin.size();
    if (n > w.cap_toys) return cudaErrorInvalidValue;
    int64_t nu = 0;
    for (int t = 0; t < n; ++t)
        if (sel.empty() || sel[t]) {
            const int64_t total = (std::max<int64_t>(end[t] - begin[t], 0) + kHessUnitEvents - 1) / kHessUnitEvents;
            int64_t pick[kSubsampleMax];
            nu += subsample ? subsample_units(total, pick) : total;
        }
    if (nu > w.cap_units) return cudaErrorInvalidValue;
    cudaError_t e = cudaSuccess;
    if (w.staged_pending) {  // the previous lists may still be in flight from the staging
        e = cudaEventSynchronize(w.staged_ev);
        if (e != cudaSuccess) return e;
        w.staged_pending = false;
    }
    int u = 0;
    for (int t = 0; t < n; ++t) {
        w.h_toy_u0[t] = u;
        w.h_toy_nu[t] = 0;
        if (!sel.empty() && !sel[t]) continue;
        if (subsample) {
            const int64_t total = (std::max<int64_t>(end[t] - begin[t], 0) + kHessUnitEvents - 1) / kHessUnitEvents;
            int64_t pick[kSubsampleMax];
            const int k = subsample_units(total, pick);
            for (int j = 0; j < k; ++j) {
                w.h_unit_toy[u] = t;
                w.h_unit_e0[u] = begin[t] + pick[j] * kHessUnitEvents;
                ++u;
            }
        } else {
            for (int64_t ev = begin[t]; ev < end[t]; ev += kHessUnitEvents) {
                w.h_unit_toy[u] = t;
                w.h_unit_e0[u] = ev;
                ++u;
            }
        }
        w.h_toy_nu[t] = u - w.h_toy_u0[t];
    }
    if (!sel.empty())
        for (int t = 0; t < n; ++t) w.h_sel[t] = sel[t];
    if (u > 0) e = cudaMemcpyAsync(w.d_unit_toy, w.h_unit_toy, sizeof(int) * u, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess && u > 0)
        e = cudaMemcpyAsync(w.d_unit_e0, w.h_unit_e0, sizeof(int64_t) * u, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess && n)
        e = cudaMemcpyAsync(w.d_toy_u0, w.h_toy_u0, sizeof(int) * n, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess && n)
        e = cudaMemcpyAsync(w.d_toy_nu, w.h_toy_nu, sizeof(int) * n, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess && !sel.empty())
        e = cudaMemcpyAsync(w.d_sel, w.h_sel, sizeof(int) * n, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaEventRecord(w.staged_ev, stream);
    if (e == cudaSuccess) w.staged_pending = true;
    if (e == cudaSuccess && wait) e = cudaStreamSynchronize(stream);
    if (e == cudaSuccess) w.n_units = u;
    return e;
}

// One Hessian pass (see HessDev); use_sel restricts it to the toys hw_set_units selected.
cudaError_t run_hess_core(const HessTarget& T, HessWork& w, const FitConfig& cfg, int mode, bool want_w2,
                          const double* thetas, int pass, bool use_sel, bool wait, bool subsample, bool single)
{
    HessLayout L;
    if (!hess_layout(T.kind, T.weighted, want_w2, &L)) return cudaErrorInvalidValue;
    const int n = T.n_toys, np = cfg.npar;
    cudaError_t e = cudaSuccess;
    const int key = T.kind * 4 + (T.weighted ? 2 : 0) + (want_w2 ? 1 : 0);
    if (key != w.layout_key) {  // (slot -> column pair) inverse table, uploaded when it changes
        std::vector<uint16_t> slot_of(64 * 64, 0xffff);
        for (int k = 0; k < L.nslots; ++k) slot_of[L.si[k] * L.ncols + L.sj[k]] = (uint16_t)k;
        e = cudaMemcpy(w.d_slot_of, slot_of.data(), sizeof(uint16_t) * slot_of.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) w.layout_key = key;
    }
    if (e == cudaSuccess && mode == kHmEval)
        e = cudaMemcpyAsync(w.d_thetas, thetas, sizeof(double) * np * n, cudaMemcpyHostToDevice, T.stream);
    if (e != cudaSuccess) return e;
    HessDev h;
    memset(&h, 0, sizeof h);
    h.n_toys = n;
    h.mode = mode;
    h.want_w2 = want_w2 ? 1 : 0;
    h.pass = pass;
    h.n_polish = w.d_npol;
    h.sel = use_sel ? w.d_sel : nullptr;
    h.n_units = w.n_units;
    h.subsample = subsample ? 1 : 0;
    h.single = single && mode == kHmStart ? 1 : 0;
    h.nslots = L.nslots;
    h.lnp_slot = L.lnp_slot;
    h.tail_begin = L.tail_begin;
    h.tail_count = L.tail_count;
    h.ncols = L.ncols;
    h.ev_begin = T.d_begin;
    h.ev_end = T.d_end;
    h.sum_wdm = T.d_sum_wdm;
    h.ev = T.ev;
    h.fits = T.d_fits;
    h.thetas = w.d_thetas;
    h.hc = w.d_hc;
    h.ht = w.d_ht;
    h.hok = w.d_hok;
    h.unit_toy = w.d_unit_toy;
    h.unit_e0 = w.d_unit_e0;
    h.toy_u0 = w.d_toy_u0;
    h.toy_nu = w.d_toy_nu;
    h.unit_sums = w.d_unit_sums;
    h.tot = w.d_tot;
    h.asmb = w.d_asm;
    h.slot_of = w.d_slot_of;
    h.out = w.d_out;
    h.status = w.d_status;
    h.cfg = cfg;
    memcpy(h.si, L.si, sizeof h.si);
    memcpy(h.sj, L.sj, sizeof h.sj);
    static_assert(sizeof(HessDev) <= 4096, "kernel parameters");
    const int occ = hess_occupancy(T.kind, T.variant, T.weighted);
    const int bps = std::max(1, std::min(occ, T.max_bps > 0 ? T.max_bps : 4));
    const int unit_blocks = std::max(1, std::min(w.n_units, T.sm_count * bps));
    e = launch_hess_pass(T.kind, T.variant, T.weighted, unit_blocks, T.stream, h);
    if (e == cudaSuccess && wait) e = cudaStreamSynchronize(T.stream);
    return e;
}

// Newton polish passes with the analytic Hessian at the final points of the finished toys
// (all toys, or those hw_set_units selected), then the accepted points stay.
cudaError_t polish_core(const HessTarget& T, HessWork& w, const FitConfig& cfg, int hessian, bool use_sel,
                        bool speculate)
{
    const int tb = (T.n_toys + 127) / 128;
    const int* sel = use_sel ? w.d_sel : nullptr;
    batch_polish_init<<<tb, 128, 0, T.stream>>>(T.d_fits, T.n_toys, sel);
    cudaError_t e = cudaGetLastError();
    // with `speculate`, passes 0 and 1 are queued back to back (nearly every large batch has
    // some toy that takes a Newton step after pass 0, and a pass over no polishing toy costs
    // little); otherwise, and from then on, the host looks at the count after each pass
    for (int pass = 0; pass < 6 && e == cudaSuccess; ++pass) {
        const bool wait = pass >= 1 || !speculate;
        e = run_hess_core(T, w, cfg, hessian == 3 ? kHmSandwich : kHmCov, hessian == 3, nullptr, pass, use_sel, wait);
        if (e == cudaSuccess && wait && __atomic_load_n(w.h_npol, __ATOMIC_ACQUIRE) == 0) break;
    }
    if (e == cudaSuccess) {
        batch_polish_close<<<tb, 128, 0, T.stream>>>(T.d_fits, T.n_toys, cfg.npar, sel);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(T.stream);
    return e;
}

}  // namespace gbnll

struct nll_batch {
    int kind = 0, ndim = 0, npar = 0, device = 0, sm_count = 0;
    DevBudget budget;  // device memory of this batch (limit from GBNLL_DEVICE_ALLOC_LIMIT)
    cudaStream_t user_stream = nullptr;  // caller's stream (0 = default)
    cudaStream_t stream = nullptr;       // the batch's own stream (graph capture needs one)
    double ranges[8] = {0};
    int n_toys = 0;
    int64_t n_pad = 0;                   // padded events per column
    int ncols = 0;
    bool weighted = false, has_basis = false, loaded = false;
    double* d_ev = nullptr;
    double* d_w = nullptr;
    std::vector<int64_t> begin, end;     // padded positions per toy
    std::vector<double> sum_wdm;
    int64_t* d_begin = nullptr;
    int64_t* d_end = nullptr;
    double* d_sum_wdm = nullptr;
    // work arrays
    int max_items = 0, max_units = 0;
    int* d_counters = nullptr;
    int* h_active = nullptr;  // mapped
    int* d_active = nullptr;
    int* d_item_toy = nullptr;
    int* d_item_u0 = nullptr;
    int* d_item_nt = nullptr;
    KConst* d_item_kc = nullptr;
    DConst* d_item_dc = nullptr;
    int* d_unit_item = nullptr;
    int* d_unit_tile = nullptr;
    double* d_unit_sums = nullptr;
    ToyFit* d_fits = nullptr;
    // fit set-up and results (allocated at the first nll_batch_fit for the loaded toys)
    double* d_init = nullptr;  // start points [n_toys x npar] then steps [npar]
    double* h_res = nullptr;   // mapped pinned, kResStride doubles per toy (batch_pack_results)
    double* d_res = nullptr;
    cudaStream_t aux_stream = nullptr;  // start-matrix passes that run beside the loop's first step
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // the instantiated device step of nll_batch_fit and the parameters it was captured with
    cudaGraph_t fit_graph = nullptr;
    cudaGraphExec_t fit_exec = nullptr;
    BatchDev fit_dev;
    int fit_shape[4] = {0, 0, 0, 0};
    // analytic Hessian pass (allocated at its first use for the loaded toys)
    HessWork hw;
    // schedule
    int tile_events = 0, bps = 2;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    std::string err;
};

namespace {

int bfail(nll_batch* b, int status, const char* fmt, ...)
{
    if (b) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        b->err = buf;
    }
    return status;
}

int bcuda(nll_batch* b, cudaError_t e, const char* what)
{
    return bfail(b, e == cudaErrorMemoryAllocation ? NLL_ERR_OOM : NLL_ERR_CUDA, "%s: %s", what,
                 cudaGetErrorString(e));
}

void free_work(nll_batch* b)
{
    hw_free(b->hw);
    if (b->fit_exec) cudaGraphExecDestroy(b->fit_exec);
    if (b->fit_graph) cudaGraphDestroy(b->fit_graph);
    b->fit_exec = nullptr;
    b->fit_graph = nullptr;
    if (b->d_init) gb_free(b->d_init);
    if (b->h_res) cudaFreeHost(b->h_res);
    b->d_init = b->h_res = b->d_res = nullptr;
    void* ptrs[] = {b->d_ev, b->d_begin, b->d_end, b->d_sum_wdm, b->d_item_toy, b->d_item_u0, b->d_item_nt,
                    b->d_item_kc, b->d_item_dc, b->d_unit_item, b->d_unit_tile, b->d_unit_sums, b->d_fits};
    for (void* p : ptrs)
        if (p) gb_free(p);
    b->d_ev = nullptr;
    b->d_w = nullptr;
    b->d_begin = b->d_end = nullptr;
    b->d_sum_wdm = nullptr;
    b->d_item_toy = b->d_item_u0 = b->d_item_nt = nullptr;
    b->d_item_kc = nullptr;
    b->d_item_dc = nullptr;
    b->d_unit_item = b->d_unit_tile = nullptr;
    b->d_unit_sums = nullptr;
    b->d_fits = nullptr;
    b->loaded = false;
}

int tile_pairs_of(const nll_batch* b) { return b->tile_events > 0 ? b->tile_events / 2 : 0; }

// work already queued on the caller's stream completes before the batch's own stream runs
cudaError_t follow_user_stream(nll_batch* b)
{
    cudaError_t e = cudaEventRecord(b->ev0, b->user_stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->ev0, 0);
    return e;
}

BatchDev make_dev(nll_batch* b)
{
    BatchDev d;
    memset(&d, 0, sizeof d);
    d.n_toys = b->n_toys;
    d.tile_pairs = tile_pairs_of(b);
    d.ev_begin = b->d_begin;
    d.ev_end = b->d_end;
    d.sum_wdm = b->d_sum_wdm;
    for (int c = 0; c < kNumCols; ++c) d.cols.col[c] = c < b->ncols ? b->d_ev + (size_t)c * b->n_pad : nullptr;
    d.cols.w = b->weighted ? b->d_w : nullptr;
    d.fits = b->d_fits;
    d.counters = b->d_counters;
    d.n_active = b->d_active;
    d.item_toy = b->d_item_toy;
    d.item_u0 = b->d_item_u0;
    d.item_nt = b->d_item_nt;
    d.item_kc = b->d_item_kc;
    d.item_dc = b->d_item_dc;
    d.unit_item = b->d_unit_item;
    d.unit_tile = b->d_unit_tile;
    d.unit_sums = b->d_unit_sums;
    d.max_items = b->max_items;
    d.max_units = b->max_units;
    d.cfg.kind = b->kind;
    d.cfg.npar = b->npar;
    for (int i = 0; i < 8; ++i) d.cfg.ranges[i] = b->ranges[i];
    return d;
}

int variant_of(const nll_batch* b) { return (b->kind == kKstar4D && !b->has_basis) ? kVarDirect : kVarPrecompute; }

// host-hoisted evaluation of every toy at thetas (one item per toy); fills nll, grad, status
int eval_all(nll_batch* b, const double* thetas, double* nll_out, double* grad_out, int* status_out, float* ms)
{
    const int n = b->n_toys, np = b->npar;
    const int tp = tile_pairs_of(b);
    std::vector<KConst> kc(n);
    std::vector<Hoist> hs(n);
    std::vector<int> item_toy(n), item_u0(n), item_nt(n), unit_item, unit_tile;
    std::vector<int> st(n, NLL_OK);
    int nunits = 0;
    for (int t = 0; t < n; ++t) {
        std::string e;
        memset(&kc[t], 0, sizeof(KConst));
        int s = hoist_core(b->kind, b->ranges, thetas + (size_t)t * np, true, hs[t], &e);
        int64_t npairs = (b->end[t] - b->begin[t] + 1) / 2;
        int nt = npairs > 0 ? (tp ? (int)((npairs + tp - 1) / tp) : 1) : 0;
        if (s != NLL_OK) {
            st[t] = s;
            nt = 0;
        } else {
            kc[t] = hs[t].k;
        }
        item_toy[t] = t;
        item_u0[t] = nunits;
        item_nt[t] = nt;
        for (int j = 0; j < nt; ++j) {
            unit_item.push_back(t);
            unit_tile.push_back(j);
        }
        nunits += nt;
    }
    if (nunits > b->max_units || n > b->max_items) return bfail(b, NLL_ERR_ARG, "work arrays too small");
    int counters[3] = {n, nunits, 0};
    cudaError_t e = cudaMemcpyAsync(b->d_item_kc, kc.data(), sizeof(KConst) * n, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_item_toy, item_toy.data(), sizeof(int) * n, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_item_u0, item_u0.data(), sizeof(int) * n, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_item_nt, item_nt.data(), sizeof(int) * n, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess && nunits)
        e = cudaMemcpyAsync(b->d_unit_item, unit_item.data(), sizeof(int) * nunits, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess && nunits)
        e = cudaMemcpyAsync(b->d_unit_tile, unit_tile.data(), sizeof(int) * nunits, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_counters, counters, sizeof counters, cudaMemcpyHostToDevice, b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "batch upload");
    BatchDev d = make_dev(b);
    int blocks = std::max(1, std::min(b->sm_count * b->bps, nunits));
    if (ms) cudaEventRecord(b->ev0, b->stream);
    if (nunits) e = launch_eval(b->kind, variant_of(b), b->weighted, blocks, b->stream, d);
    if (ms) cudaEventRecord(b->ev1, b->stream);
    std::vector<double> sums((size_t)std::max(nunits, 1) * kAccMax);
    if (e == cudaSuccess && nunits)
        e = cudaMemcpyAsync(sums.data(), b->d_unit_sums, sizeof(double) * kAccMax * nunits, cudaMemcpyDeviceToHost,
                            b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "batch evaluation");
    if (ms) cudaEventElapsedTime(ms, b->ev0, b->ev1);
    const int K = num_acc(b->kind, true);
    int first_bad = NLL_OK;
    for (int t = 0; t < n; ++t) {
        double* g = grad_out ? grad_out + (size_t)t * np : nullptr;
        if (st[t] == NLL_OK) {
            double S[kAccMax] = {0};
            for (int j = 0; j < item_nt[t]; ++j)
                for (int k = 0; k < K; ++k) S[k] += sums[(size_t)(item_u0[t] + j) * kAccMax + k];
            if (S[K - 1] != 0.0 || !isfinite(S[0])) {
                st[t] = NLL_ERR_NONPOSITIVE_PDF;
            } else {
                double gg[18];
                assemble_core(b->kind, hs[t], b->sum_wdm[t], S, &nll_out[t], gg);
                if (g)
                    for (int k = 0; k < np; ++k) g[k] = gg[k];
            }
        }
        if (st[t] != NLL_OK) {
            nll_out[t] = INFINITY;
            if (g)
                for (int k = 0; k < np; ++k) g[k] = NAN;
            if (first_bad == NLL_OK) first_bad = st[t];
        }
        if (status_out) status_out[t] = st[t];
    }
    return first_bad;
}



HessTarget target_of(nll_batch* b)
{
    HessTarget T;
    memset(&T, 0, sizeof T);
    T.kind = b->kind;
    T.variant = variant_of(b);
    T.sm_count = b->sm_count;
    T.n_toys = b->n_toys;
    T.weighted = b->weighted;
    for (int c = 0; c < kNumCols; ++c) T.ev.col[c] = c < b->ncols ? b->d_ev + (size_t)c * b->n_pad : nullptr;
    T.ev.w = b->weighted ? b->d_w : nullptr;
    T.d_begin = b->d_begin;
    T.d_end = b->d_end;
    T.d_sum_wdm = b->d_sum_wdm;
    T.d_fits = b->d_fits;
    T.stream = b->stream;
    return T;
}

// work arrays of the Hessian pass for the loaded toys (every toy, units of kHessUnitEvents)
int ensure_hess_work(nll_batch* b)
{
    if (b->hw.ready) return NLL_OK;
    int64_t units = 0;
    for (int t = 0; t < b->n_toys; ++t) units += (b->end[t] - b->begin[t] + kHessUnitEvents - 1) / kHessUnitEvents;
    if (units > (1 << 28)) return bfail(b, NLL_ERR_ARG, "too many Hessian units");
    cudaError_t e = hw_alloc(b->hw, b->n_toys, (int)units, b->npar);
    if (e == cudaSuccess) e = hw_set_units(b->hw, b->begin, b->end, std::vector<int>(), b->stream);
    if (e != cudaSuccess) {
        hw_free(b->hw);
        return bcuda(b, e, "Hessian work arrays");
    }
    return NLL_OK;
}

// One Hessian pass over all toys on the batch's stream.  kHmEval takes the host thetas
// ([n_toys][npar]) and leaves per-toy results in hw.d_out / hw.d_status; the other modes read
// and write the toys' fit states (the fits must be on the device).
int run_hess_pass(nll_batch* b, const FitConfig& cfg, int mode, bool want_w2, const double* thetas)
{
    int st = ensure_hess_work(b);
    if (st != NLL_OK) return st;
    cudaError_t e = run_hess_core(target_of(b), b->hw, cfg, mode, want_w2, thetas, 0, false);
    if (e != cudaSuccess) return bcuda(b, e, "Hessian pass");
    return NLL_OK;
}

// after the events are in d_ev: angular basis, per-toy arrays and work arrays sized for the
// largest step (every toy with a full stencil); device_sums computes sum (m - ma) per toy
// on the device instead of uploading b->sum_wdm
cudaError_t finish_store(nll_batch* b, bool basis, int64_t pos, bool device_sums)
{
    const int n_toys = b->n_toys;
    const int64_t n_pad = b->n_pad;
    const int64_t total = pos;
    cudaError_t e = cudaSuccess;
    if (basis && total > 0) {
        BArgs ba;
        ba.ctl = b->d_ev + (size_t)kColCtl * n_pad;
        ba.ctk = b->d_ev + (size_t)kColCtk * n_pad;
        ba.phi = b->d_ev + (size_t)kColPhi * n_pad;
        for (int j = 0; j < 13; ++j) ba.out[j] = b->d_ev + (size_t)(kColH0 + j) * n_pad;
        ba.n = pos;
        int blocks = (int)std::min<int64_t>((pos + 255) / 256, (int64_t)b->sm_count * 8);
        e = launch_basis(std::max(blocks, 1), 256, b->stream, ba);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
        if (e != cudaSuccess) {
            free_work(b);
            return e;
        }
    }
    b->has_basis = basis;
    // per-toy arrays and work arrays sized for the largest step (every toy with a full stencil)
    int64_t tiles_max = 0;
    const int64_t min_tile_pairs = 64;  // smallest split-toy tile the schedule accepts
    for (int t = 0; t < n_toys; ++t) {
        int64_t np = (b->end[t] - b->begin[t] + 1) / 2;
        tiles_max += np ? (np + min_tile_pairs - 1) / min_tile_pairs : 0;
    }
    int64_t max_items = (int64_t)std::max(n_toys, 1) * (2 * b->npar + 1);
    int64_t max_units = std::max<int64_t>(tiles_max, 1) * (2 * b->npar + 1);
    if (max_units > (1ll << 30)) {
        free_work(b);
        return cudaErrorInvalidValue;
    }
    b->max_items = (int)max_items;
    b->max_units = (int)max_units;
    e = gb_malloc(&b->budget, &b->d_begin, sizeof(int64_t) * std::max(n_toys, 1));
    if (e == cudaSuccess) e = gb_malloc(&b->budget, &b->d_end, sizeof(int64_t) * std::max(n_toys, 1));
    if (e == cudaSuccess) e = gb_malloc(&b->budget, &b->d_sum_wdm, sizeof(double) * std::max(n_toys, 1));
    if (e == cudaSuccess) e = gb_malloc(&b->budget, &b->d_item_toy, sizeof(int) * max_items);
    if (e == cudaSuccess) e = gb_malloc(&b->budget, &b->d_item_u0, sizeof(int) * max_items);
    if (e == cudaSuccess) e = gb_malloc(&b->budget, &b->d_item_nt, sizeof(int) * max_items);
    if (e == cudaSuccess) e = gb_malloc(&b->budget, &b->d_item_kc, sizeof(KConst) * max_items);
    if (e == cudaSuccess) e = gb_malloc(&b->budget, &b->d_item_dc, sizeof(DConst) * max_items);
    if (e == cudaSuccess) e = gb_malloc(&b->budget, &b->d_unit_item, sizeof(int) * max_units);
    if (e == cudaSuccess) e = gb_malloc(&b->budget, &b->d_unit_tile, sizeof(int) * max_units);
    if (e == cudaSuccess) e = gb_malloc(&b->budget, &b->d_unit_sums, sizeof(double) * kAccMax * max_units);
    if (e == cudaSuccess) e = gb_malloc(&b->budget, &b->d_fits, sizeof(ToyFit) * std::max(n_toys, 1));
    // every index the kernels can read is valid from the start
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_item_toy, 0, sizeof(int) * max_items, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_item_u0, 0, sizeof(int) * max_items, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_item_nt, 0, sizeof(int) * max_items, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_unit_item, 0, sizeof(int) * max_units, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_unit_tile, 0, sizeof(int) * max_units, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_counters, 0, sizeof(int) * 4, b->stream);
    if (e == cudaSuccess && n_toys) {
        e = cudaMemcpyAsync(b->d_begin, b->begin.data(), sizeof(int64_t) * n_toys, cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(b->d_end, b->end.data(), sizeof(int64_t) * n_toys, cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess && !device_sums)
            e = cudaMemcpyAsync(b->d_sum_wdm, b->sum_wdm.data(), sizeof(double) * n_toys, cudaMemcpyHostToDevice,
                                b->stream);
        if (e == cudaSuccess && device_sums) {
            e = toy_sums(b->d_ev, b->d_begin, b->d_end, b->ranges[0], n_toys, b->d_sum_wdm, b->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(b->sum_wdm.data(), b->d_sum_wdm, sizeof(double) * n_toys, cudaMemcpyDeviceToHost,
                                    b->stream);
        }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) free_work(b);
    return e;
}

}  // namespace

namespace gbnll {

// minimiser settings shared by all toys
void setup_config(FitConfig& c, int np, const double* lo, const double* hi, const double* step, const int* fixed,
                  const fit_options& opt)
{
    c.strategy = (opt.strategy == 3 || opt.strategy == 5) ? 2 : opt.strategy;  // 2, 3, 5: start matrix from a Hessian pass
    c.hessian = opt.hessian == 1;       // in-loop finite-difference Hessian; 2/3 run after the loop
    c.max_iter = opt.max_iter;
    c.tol_edm = opt.tol_edm;
    int nf = 0;
    for (int k = 0; k < np; ++k) {
        c.bounded[k] = 0;
        c.lo[k] = c.hi[k] = 0.0;
        if (lo && hi && lo[k] < hi[k] && isfinite(lo[k]) && isfinite(hi[k])) {
            c.bounded[k] = 1;
            c.lo[k] = lo[k];
            c.hi[k] = hi[k];
        }
        if (fixed && fixed[k]) continue;
        c.idx[nf++] = k;
    }
    c.nf = nf;
}

// initial minimiser state of one toy at th0 (internal coordinates and steps)
void init_fit(ToyFit& F, const FitConfig& c, const double* th0, const double* step)
{
    memset(&F, 0, sizeof F);
    init_fit_fields(F, c, th0, step);
}

// fit_result of one finished toy
void fill_result(const ToyFit& F, const FitConfig& c, fit_result& r)
{
    const int np = c.npar, nf = c.nf;
    memset(&r, 0, sizeof r);
    for (int k = 0; k < np; ++k) r.theta[k] = F.th[k];
    for (int i = 0; i < nf; ++i) {
        r.err[c.idx[i]] = F.err[i];
        for (int j = 0; j < nf; ++j) r.cov[c.idx[i] * np + c.idx[j]] = F.cov[i * nf + j];
    }
    r.nll = F.f;
    r.edm = F.edm;
    r.n_eval = F.n_eval;
    r.n_iter = F.iter;
    r.status = F.phase == kPhDone ? F.status : NLL_ERR_NOT_CONVERGED;
}

// fit_result of one toy from its batch_pack_results record
void fill_result_packed(const double* p, const FitConfig& c, fit_result& r)
{
    const int np = c.npar, nf = c.nf;
    memset(&r, 0, sizeof r);
    for (int k = 0; k < np; ++k) r.theta[k] = p[k];
    for (int i = 0; i < nf; ++i) {
        r.err[c.idx[i]] = p[kNP + i];
        for (int j = 0; j < nf; ++j) r.cov[c.idx[i] * np + c.idx[j]] = p[2 * kNP + i * nf + j];
    }
    const double* tail = p + 2 * kNP + kNP * kNP;
    r.nll = tail[0];
    r.edm = tail[1];
    r.n_eval = (int)tail[2];
    r.n_iter = (int)tail[3];
    r.status = (int)tail[4];
}

}  // namespace gbnll

extern "C" {

int nll_batch_create(int kind, const double* obs_ranges, int device, uintptr_t cuda_stream, nll_batch** out)
{
    if (!out) return NLL_ERR_ARG;
    *out = nullptr;
    if ((kind != NLL_MODEL_MASS1D && kind != NLL_MODEL_KSTARMUMU4D) || !obs_ranges) return NLL_ERR_ARG;
    if (!(isfinite(obs_ranges[0]) && isfinite(obs_ranges[1]) && obs_ranges[0] < obs_ranges[1])) return NLL_ERR_ARG;
    if (kind == NLL_MODEL_KSTARMUMU4D) {
        const double want[6] = {-1.0, 1.0, -1.0, 1.0, -kPiH, kPiH};
        for (int i = 0; i < 6; ++i)
            if (fabs(obs_ranges[2 + i] - want[i]) > 1e-12) return NLL_ERR_ARG;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return NLL_ERR_CUDA;
    if (cudaSetDevice(device) != cudaSuccess) return NLL_ERR_CUDA;
    nll_batch* b = new nll_batch();
    b->budget.limit = dev_budget_limit_from_env();
    b->hw.budget = &b->budget;
    b->kind = kind;
    b->ndim = kind == NLL_MODEL_MASS1D ? 1 : 4;
    b->npar = kind == NLL_MODEL_MASS1D ? 4 : 18;
    b->device = device;
    b->user_stream = (cudaStream_t)cuda_stream;
    memcpy(b->ranges, obs_ranges, sizeof(double) * 2 * b->ndim);
    if (kind == NLL_MODEL_KSTARMUMU4D) {
        b->ranges[6] = -kPiH;
        b->ranges[7] = kPiH;
    }
    cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, device);
    cudaError_t e = ensure_btab(device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->aux_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming);
    if (e == cudaSuccess) e = gb_malloc(&b->budget, &b->d_counters, sizeof(int) * 8);  // items, units, next, steps, tile
    if (e == cudaSuccess) e = cudaHostAlloc(&b->h_active, sizeof(int), cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer(&b->d_active, b->h_active, 0);
    if (e == cudaSuccess) e = cudaEventCreate(&b->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&b->ev1);
    if (e != cudaSuccess) {
        nll_batch_destroy(b);
        return e == cudaErrorMemoryAllocation ? NLL_ERR_OOM : NLL_ERR_CUDA;
    }
    *out = b;
    return NLL_OK;
}

void nll_batch_destroy(nll_batch* b)
{
    if (!b) return;
    cudaSetDevice(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    free_work(b);
    if (b->d_counters) gb_free(b->d_counters);
    if (b->h_active) cudaFreeHost(b->h_active);
    if (b->ev0) cudaEventDestroy(b->ev0);
    if (b->ev1) cudaEventDestroy(b->ev1);
    if (b->stream) cudaStreamDestroy(b->stream);
    if (b->aux_stream) cudaStreamDestroy(b->aux_stream);
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    if (b->ev_join) cudaEventDestroy(b->ev_join);
    delete b;
}

int nll_batch_load(nll_batch* b, const int64_t* offsets, int n_toys, const double* const* columns,
                   const double* weights, int precompute)
{
    if (!b) return NLL_ERR_ARG;
    if (n_toys < 0 || !offsets || offsets[0] != 0) return bfail(b, NLL_ERR_ARG, "bad offsets");
    for (int t = 0; t < n_toys; ++t)
        if (offsets[t + 1] < offsets[t]) return bfail(b, NLL_ERR_ARG, "offsets must not decrease");
    const int64_t total = offsets[n_toys];
    if (total > 0 && !columns) return bfail(b, NLL_ERR_ARG, "null columns");
    for (int d = 0; d < b->ndim && total > 0; ++d)
        if (!columns[d]) return bfail(b, NLL_ERR_ARG, "column %d is NULL", d);
    if (cudaSetDevice(b->device) != cudaSuccess) return bfail(b, NLL_ERR_CUDA, "cudaSetDevice failed");
    if (follow_user_stream(b) != cudaSuccess) return bfail(b, NLL_ERR_CUDA, "stream ordering failed");
    cudaStreamSynchronize(b->stream);
    free_work(b);
    // padded positions: every toy starts on an even event index (pairs of events per load)
    b->n_toys = n_toys;
    b->begin.assign(n_toys, 0);
    b->end.assign(n_toys, 0);
    b->sum_wdm.assign(n_toys, 0.0);
    int64_t pos = 0;
    for (int t = 0; t < n_toys; ++t) {
        pos = (pos + 1) & ~int64_t(1);
        b->begin[t] = pos;
        pos += offsets[t + 1] - offsets[t];
        b->end[t] = pos;
    }
    const int64_t n_pad = std::max<int64_t>((pos + 63) / 64 * 64, 64);
    // validate on the host, and sum w (m - ma) per toy (fixed order)
    for (int t = 0; t < n_toys; ++t) {
        double s = 0.0;
        for (int64_t i = offsets[t]; i < offsets[t + 1]; ++i) {
            double w = weights ? weights[i] : 1.0;
            if (!(w >= 0.0 && w <= 1e300)) return bfail(b, NLL_ERR_ARG, "invalid weight at event %lld", (long long)i);
            for (int d = 0; d < b->ndim; ++d) {
                double x = columns[d][i];
                if (!(x >= b->ranges[2 * d] && x <= b->ranges[2 * d + 1]))
                    return bfail(b, NLL_ERR_ARG, "event %lld outside the observable ranges", (long long)i);
            }
            s += w * (columns[0][i] - b->ranges[0]);
        }
        b->sum_wdm[t] = s;
    }
    const bool basis = b->kind == kKstar4D && precompute;
    b->ncols = b->kind == kMass1D ? 1 : (basis ? kNumCols : 4);
    const int nalloc = b->ncols + (weights ? 1 : 0);
    b->n_pad = n_pad;
    cudaError_t e = gb_malloc(&b->budget, &b->d_ev, sizeof(double) * n_pad * nalloc);
    if (e != cudaSuccess) {
        b->d_ev = nullptr;
        return bcuda(b, e, "batch event store");
    }
    e = cudaMemsetAsync(b->d_ev, 0, sizeof(double) * n_pad * nalloc, b->stream);
    // host staging in the padded layout, one copy per column
    std::vector<double> stage(n_pad);
    auto put = [&](const double* src, double* dst) {
        std::fill(stage.begin(), stage.end(), 0.0);
        for (int t = 0; t < n_toys; ++t)
            memcpy(stage.data() + b->begin[t], src + offsets[t], sizeof(double) * (offsets[t + 1] - offsets[t]));
        cudaError_t e2 = cudaMemcpyAsync(dst, stage.data(), sizeof(double) * n_pad, cudaMemcpyHostToDevice, b->stream);
        if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(b->stream);
        return e2;
    };
    for (int d = 0; d < b->ndim && e == cudaSuccess && total > 0; ++d) e = put(columns[d], b->d_ev + (size_t)d * n_pad);
    b->weighted = weights != nullptr;
    if (weights) {
        b->d_w = b->d_ev + (size_t)b->ncols * n_pad;
        if (e == cudaSuccess && total > 0) e = put(weights, b->d_w);
    }
    if (e != cudaSuccess) {
        free_work(b);
        return bcuda(b, e, "batch copy");
    }
    e = finish_store(b, basis, pos, false);
    if (e != cudaSuccess) return bcuda(b, e, "batch work arrays");
    b->loaded = true;
    b->err.clear();
    return NLL_OK;
}

int nll_batch_generate(nll_batch* b, const double* theta, const int64_t* counts, int n_toys, uint64_t seed,
                       int precompute)
{
    if (!b) return NLL_ERR_ARG;
    if (n_toys < 0 || (n_toys > 0 && (!counts || !theta))) return bfail(b, NLL_ERR_ARG, "bad arguments");
    for (int t = 0; t < n_toys; ++t)
        if (counts[t] < 0) return bfail(b, NLL_ERR_ARG, "negative event count");
    if (cudaSetDevice(b->device) != cudaSuccess) return bfail(b, NLL_ERR_CUDA, "cudaSetDevice failed");
    if (follow_user_stream(b) != cudaSuccess) return bfail(b, NLL_ERR_CUDA, "stream ordering failed");
    cudaStreamSynchronize(b->stream);
    free_work(b);
    b->n_toys = n_toys;
    b->begin.assign(n_toys, 0);
    b->end.assign(n_toys, 0);
    b->sum_wdm.assign(n_toys, 0.0);
    int64_t pos = 0;
    for (int t = 0; t < n_toys; ++t) {
        pos = (pos + 1) & ~int64_t(1);
        b->begin[t] = pos;
        pos += counts[t];
        b->end[t] = pos;
    }
    const int64_t n_pad = std::max<int64_t>((pos + 63) / 64 * 64, 64);
    const bool basis = b->kind == kKstar4D && precompute;
    b->ncols = b->kind == kMass1D ? 1 : (basis ? kNumCols : 4);
    b->n_pad = n_pad;
    b->weighted = false;
    cudaError_t e = gb_malloc(&b->budget, &b->d_ev, sizeof(double) * n_pad * b->ncols);
    if (e != cudaSuccess) {
        b->d_ev = nullptr;
        return bcuda(b, e, "batch event store");
    }
    e = cudaMemsetAsync(b->d_ev, 0, sizeof(double) * n_pad * b->ncols, b->stream);
    if (e != cudaSuccess) {
        free_work(b);
        return bcuda(b, e, "batch event store");
    }
    double* out[4] = {b->d_ev, nullptr, nullptr, nullptr};
    if (b->kind == kKstar4D)
        for (int d = 1; d < 4; ++d) out[d] = b->d_ev + (size_t)d * n_pad;
    int st = gen_toys(b->kind, b->ranges, theta, counts, n_toys, seed, b->begin.data(), out, b->sm_count, b->stream);
    if (st != NLL_OK) {
        free_work(b);
        return bfail(b, st, "generation failed (invalid parameters or accept-reject did not converge)");
    }
    e = finish_store(b, basis, pos, true);
    if (e != cudaSuccess) return bcuda(b, e, "batch work arrays");
    b->loaded = true;
    b->err.clear();
    return NLL_OK;
}

int nll_batch_eval_grad(nll_batch* b, const double* thetas, double* nll_out, double* grad_out, int* status_out)
{
    if (!b) return NLL_ERR_ARG;
    if (!b->loaded) return bfail(b, NLL_ERR_STATE, "no toys loaded");
    if (!thetas || !nll_out || !grad_out) return bfail(b, NLL_ERR_ARG, "null argument");
    if (cudaSetDevice(b->device) != cudaSuccess) return bfail(b, NLL_ERR_CUDA, "cudaSetDevice failed");
    if (b->n_toys == 0) return NLL_OK;
    if (follow_user_stream(b) != cudaSuccess) return bfail(b, NLL_ERR_CUDA, "stream ordering failed");
    return eval_all(b, thetas, nll_out, grad_out, status_out, nullptr);
}

int nll_batch_set_schedule(nll_batch* b, int tile_events, int blocks_per_sm)
{
    if (!b) return NLL_ERR_ARG;
    if (tile_events < 0 || (tile_events > 0 && (tile_events < 128 || (tile_events & 1))))
        return bfail(b, NLL_ERR_ARG, "tile_events must be 0 or an even number >= 128");
    if (blocks_per_sm < 0 || blocks_per_sm > 32) return bfail(b, NLL_ERR_ARG, "blocks_per_sm out of range");
    b->tile_events = tile_events;
    if (blocks_per_sm) b->bps = blocks_per_sm;
    return NLL_OK;
}

int nll_batch_get_schedule(const nll_batch* b, int* tile_events, int* blocks_per_sm)
{
    if (!b) return NLL_ERR_ARG;
    if (tile_events) *tile_events = b->tile_events;
    if (blocks_per_sm) *blocks_per_sm = b->bps;
    return NLL_OK;
}

int nll_batch_num_toys(const nll_batch* b) { return b ? b->n_toys : -1; }

const char* nll_batch_last_error(const nll_batch* b) { return b ? b->err.c_str() : "null batch"; }

int nll_batch_autotune(nll_batch* b)
{
    if (!b) return NLL_ERR_ARG;
    if (!b->loaded || b->n_toys == 0) return bfail(b, NLL_ERR_STATE, "no toys loaded");
    if (cudaSetDevice(b->device) != cudaSuccess) return bfail(b, NLL_ERR_CUDA, "cudaSetDevice failed");
    // evaluate every toy at a valid interior point of the model: the mean of the ranges is
    // not one, so use the first toy's sample-independent default (mid-window Gaussian)
    const int np = b->npar;
    std::vector<double> th((size_t)b->n_toys * np);
    double base[18];
    const double ma = b->ranges[0], mb = b->ranges[1];
    if (b->kind == kMass1D) {
        const double v[4] = {0.5 * (ma + mb), 0.05 * (mb - ma), 0.0, 0.5};
        memcpy(base, v, sizeof v);
    } else {
        const double v[18] = {0.5 * (ma + mb), 0.05 * (mb - ma), 0.6, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0.5};
        memcpy(base, v, sizeof v);
    }
    for (int t = 0; t < b->n_toys; ++t) memcpy(&th[(size_t)t * np], base, sizeof(double) * np);
    std::vector<double> nll(b->n_toys), g((size_t)b->n_toys * np);
    const int tiles[] = {0, 256, 512, 1024, 2048, 4096};
    const int bpss[] = {1, 2, 4};
    // a result kept from an earlier process for the same device and workload (GBNLL_TUNE_CACHE)
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, b->device) != cudaSuccess) return bfail(b, NLL_ERR_CUDA, "device properties");
    int64_t events = 0;
    for (int t = 0; t < b->n_toys; ++t) events += b->end[t] - b->begin[t];
    int toys_class = 0, events_class = 0;
    while ((1 << (toys_class + 1)) <= b->n_toys) ++toys_class;
    while ((int64_t(1) << (events_class + 1)) <= events / b->n_toys) ++events_class;
    const std::string key = tune_cache_key(prop.name, b->sm_count, "batch", b->kind,
                                           (b->weighted ? 1 : 0) + (b->has_basis ? 2 : 0), toys_class, events_class);
    int kept[3];
    if (tune_cache_lookup(key, kept)) {
        bool tile_ok = false, bps_ok = false;
        for (int tile : tiles) tile_ok = tile_ok || tile == kept[0];
        for (int bps : bpss) bps_ok = bps_ok || bps == kept[1];
        if (tile_ok && bps_ok) {
            b->tile_events = kept[0];
            b->bps = kept[1];
            return NLL_OK;
        }
    }
    float best = 1e30f;
    int bt = b->tile_events, bb = b->bps;
    for (int tile : tiles)
        for (int bps : bpss) {
            b->tile_events = tile;
            b->bps = bps;
            float tot = 0.f;
            for (int rep = 0; rep < 3; ++rep) {
                float ms = 0.f;
                eval_all(b, th.data(), nll.data(), g.data(), nullptr, &ms);
                if (rep > 0) tot += ms;
            }
            if (tot < best) {
                best = tot;
                bt = tile;
                bb = bps;
            }
        }
    b->tile_events = bt;
    b->bps = bb;
    const int result[3] = {bt, bb, 0};
    tune_cache_store(key, result);
    return NLL_OK;
}

// memory that kernels on the batch's device can write: its own device memory, pinned or
// managed memory, or ordinary host memory where the device has pageable-memory access
static bool device_writable(nll_batch* b, const void* p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeDevice) return at.device == b->device;
    if (at.type == cudaMemoryTypeManaged || at.type == cudaMemoryTypeHost) return true;
    int pageable = 0;
    cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, b->device);
    return at.type == cudaMemoryTypeUnregistered && pageable != 0;
}

// The whole batched fit (nll_batch_fit and nll_batch_fit_arrays): leaves every toy's packed
// result (kResStride doubles, batch_pack_results) in b->h_res, or with `direct` writes the
// results into those arrays from the device; the configuration goes to *cfg_out.
static int batch_fit_core(nll_batch* b, const double* theta0, int shared_start, const double* lo, const double* hi,
                          const double* step, const int* fixed, const fit_options* opt_in, int* steps_out,
                          FitConfig* cfg_out, const ArrayOut* direct)
{
    if (!b) return NLL_ERR_ARG;
    if (!b->loaded) return bfail(b, NLL_ERR_STATE, "no toys loaded");
    if (!theta0) return bfail(b, NLL_ERR_ARG, "null argument");
    GBNLL_TRACE("nll_batch_fit");
    if (cudaSetDevice(b->device) != cudaSuccess) return bfail(b, NLL_ERR_CUDA, "cudaSetDevice failed");
    fit_options opt;
    if (opt_in)
        opt = *opt_in;
    else
        memset(&opt, 0, sizeof opt);
    if (!(opt.tol_edm > 0.0)) opt.tol_edm = 1e-8;
    if (opt.max_iter <= 0) opt.max_iter = 500;
    if (opt.strategy < 0 || opt.strategy > 5 || opt.strategy == 4 || opt.hessian < 0 || opt.hessian > 3)
        return bfail(b, NLL_ERR_ARG, "strategy must be 0..3 or 5 and hessian 0..3");
    const int n = b->n_toys, np = b->npar;
    if (n == 0) return NLL_OK;
    BatchDev d = make_dev(b);
    FitConfig& c = d.cfg;
    setup_config(c, np, lo, hi, step, fixed, opt);
    const int nf = c.nf;
    // start states on the device: only the start points and steps cross the link
    cudaError_t e = cudaSuccess;
    if (!b->d_init) e = gb_malloc(&b->budget, &b->d_init, sizeof(double) * ((size_t)n + 1) * kNP);
    if (e == cudaSuccess && !b->h_res) {
        e = cudaHostAlloc(&b->h_res, sizeof(double) * (size_t)n * kResStride, cudaHostAllocMapped);
        if (e == cudaSuccess) e = cudaHostGetDevicePointer(&b->d_res, b->h_res, 0);
    }
    if (e != cudaSuccess) return bcuda(b, e, "fit set-up buffers");
    const size_t nth = shared_start ? (size_t)np : (size_t)n * np;
    double* d_step = b->d_init + (size_t)n * kNP;
    *b->h_active = n;
    e = follow_user_stream(b);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_init, theta0, sizeof(double) * nth, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess && step)
        e = cudaMemcpyAsync(d_step, step, sizeof(double) * np, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) {
        batch_init_fits<<<n, 128, 0, b->stream>>>(b->d_fits, n, c, b->d_init, shared_start ? 1 : 0,
                                                  step ? d_step : nullptr);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return bcuda(b, e, "fit state set-up");
    int* d_steps = b->d_counters + 3;
    int* d_step_tp = b->d_counters + 4;
    d.step_tp = d_step_tp;
    batch_loop_init<<<1, 1, 0, b->stream>>>(d_steps, d_step_tp, d.tile_pairs);
    e = cudaGetLastError();
    if (e != cudaSuccess) return bcuda(b, e, "fit loop set-up");
    int steps_before = 0;  // steps run ahead of the loop's graph
    {
        GBNLL_TRACE("start matrices (queued)");
        if (opt.strategy == 2) {
            // start matrices from the analytic Hessian at every toy's start point, queued without a
            // wait (the fit loop follows on the same stream); the pass takes each toy's first step
            int st = ensure_hess_work(b);
            if (st != NLL_OK) return st;
            e = run_hess_core(target_of(b), b->hw, c, kHmStart, false, nullptr, 0, false, false);
            if (e != cudaSuccess) return bcuda(b, e, "start matrices");
        } else if (opt.strategy == 3 || opt.strategy == 5) {
            // Start matrices that give no NLL and gradient at the start point (from a subsample of
            // every toy's events, strategy 3, or in single precision, strategy 5): the pass runs on
            // the auxiliary stream beside the loop's first step, whose evaluation of the start points
            // (FP64 bound) overlaps the pass (bound by single-precision and shared-memory work, or
            // short); the step's update waits for the start matrices.  The pass takes at most two
            // blocks per SM, so that the evaluation's blocks find room.
            int st = ensure_hess_work(b);
            if (st != NLL_OK) return st;
            HessTarget Ta = target_of(b);
            Ta.stream = b->aux_stream;
            Ta.max_bps = 2;
            e = cudaEventRecord(b->ev_fork, b->stream);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(b->aux_stream, b->ev_fork, 0);
            if (e == cudaSuccess) e = launch_step_eval(d, variant_of(b), b->weighted, b->sm_count * b->bps, b->stream);
            if (opt.strategy == 3) {
                // the subsample's unit lists, then the whole toys' lists again for the later passes
                if (e == cudaSuccess)
                    e = hw_set_units(b->hw, b->begin, b->end, std::vector<int>(), b->aux_stream, false, true);
                if (e == cudaSuccess) e = run_hess_core(Ta, b->hw, c, kHmStart, false, nullptr, 0, false, false, true);
                if (e == cudaSuccess)
                    e = hw_set_units(b->hw, b->begin, b->end, std::vector<int>(), b->aux_stream, false, false);
            } else if (e == cudaSuccess) {
                e = run_hess_core(Ta, b->hw, c, kHmStart, false, nullptr, 0, false, false, false, true);
            }
            if (e == cudaSuccess) e = cudaEventRecord(b->ev_join, b->aux_stream);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->ev_join, 0);
            if (e == cudaSuccess) e = launch_step_update(d, b->stream);
            if (e != cudaSuccess) return bcuda(b, e, "start matrices");
            steps_before = 1;
        }
    }

    // The fit loop runs on the device: a CUDA graph with one while node whose body is a device
    // step (counter reset, prepare, evaluate, update) followed by a one-thread control kernel
    // that counts the step and keeps the loop going while some toy is still fitting (and the
    // step limit is not reached).  The graph is built once and kept while the batch's buffers
    // and the fit configuration stay the same; one launch runs the whole loop.
    const int eval_blocks = b->sm_count * b->bps;
    const int max_steps = opt.max_iter * 40 + 8;  // every line-search trial is one step
    const int shape[4] = {eval_blocks, max_steps, 0, variant_of(b)};
    if (!b->fit_exec || memcmp(&b->fit_dev, &d, sizeof d) != 0 || memcmp(b->fit_shape, shape, sizeof shape) != 0) {
        if (b->fit_exec) cudaGraphExecDestroy(b->fit_exec);
        if (b->fit_graph) cudaGraphDestroy(b->fit_graph);
        b->fit_exec = nullptr;
        b->fit_graph = nullptr;
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        cudaGraphConditionalHandle handle;
        e = cudaGraphCreate(&graph, 0);
        if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&handle, graph, 1u, cudaGraphCondAssignDefault);
        cudaGraphNodeParams np_ = {};
        cudaGraphNode_t node;
        if (e == cudaSuccess) {
            np_.type = cudaGraphNodeTypeConditional;
            np_.conditional.handle = handle;
            np_.conditional.type = cudaGraphCondTypeWhile;
            np_.conditional.size = 1;
            e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np_);
        }
        if (e == cudaSuccess) {
            cudaGraph_t body = np_.conditional.phGraph_out[0];
            e = cudaStreamBeginCaptureToGraph(b->stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                cudaError_t ec = launch_step(d, variant_of(b), b->weighted, eval_blocks, b->stream);
                if (ec == cudaSuccess) {
                    batch_loop_control<<<1, 1, 0, b->stream>>>(handle, d.n_active, d_steps, max_steps, d_step_tp,
                                                              n, d.tile_pairs);
                    ec = cudaGetLastError();
                }
                e = cudaStreamEndCapture(b->stream, &body);
                if (e == cudaSuccess) e = ec;
            }
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
        if (e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return bcuda(b, e, "fit graph");
        }
        b->fit_graph = graph;
        b->fit_exec = exec;
        b->fit_dev = d;
        memcpy(b->fit_shape, shape, sizeof shape);
    }
    int steps = 0;
    {
        GBNLL_TRACE("fit loop (device)");
        e = cudaGraphLaunch(b->fit_exec, b->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&steps, d_steps, sizeof(int), cudaMemcpyDeviceToHost, b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    }
    if (e != cudaSuccess) return bcuda(b, e, "fit loop");
    if (steps_out) *steps_out = steps + steps_before;
    if (opt.hessian >= 2) {
        GBNLL_TRACE("Newton polish");
        // analytic Hessian at every toy's final point: covariance, EDM, and Newton polish steps
        // (each pass evaluates the toys still polishing) until no toy proposes another step
        int st = ensure_hess_work(b);
        if (st != NLL_OK) return st;
        e = polish_core(target_of(b), b->hw, c, opt.hessian, false, n >= 64);
        if (e != cudaSuccess) return bcuda(b, e, "Newton polish");
    }
    if (direct)
        batch_write_arrays<<<n, 128, 0, b->stream>>>(b->d_fits, n, c, *direct);
    else
        batch_pack_results<<<n, 128, 0, b->stream>>>(b->d_fits, nullptr, n, np, nf, b->d_res);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "fit results");
    *cfg_out = c;
    return NLL_OK;
}

int nll_batch_fit(nll_batch* b, const double* theta0, int shared_start, const double* lo, const double* hi,
                  const double* step, const int* fixed, const fit_options* opt_in, fit_result* results, int* steps_out)
{
    if (b && !results) return bfail(b, NLL_ERR_ARG, "null argument");
    FitConfig c;
    memset(&c, 0, sizeof c);
    const int st = batch_fit_core(b, theta0, shared_start, lo, hi, step, fixed, opt_in, steps_out, &c, nullptr);
    if (st != NLL_OK || b->n_toys == 0) return st;
    int all = NLL_OK;
    for (int t = 0; t < b->n_toys; ++t) {
        fill_result_packed(b->h_res + (size_t)t * kResStride, c, results[t]);
        if (results[t].status != NLL_OK) all = NLL_ERR_NOT_CONVERGED;
    }
    return all;
}

int nll_batch_fit_arrays(nll_batch* b, const double* theta0, int shared_start, const double* lo, const double* hi,
                         const double* step, const int* fixed, const fit_options* opt_in, double* theta_out,
                         double* err_out, double* cov_out, double* nll_out, double* edm_out, int* n_eval_out,
                         int* n_iter_out, int* status_out, int* steps_out)
{
    FitConfig c;
    memset(&c, 0, sizeof c);
    // where the device can write every output (pinned, managed, or -- on a system with
    // pageable-memory access such as the Grace-Blackwell link -- ordinary host memory) the
    // results go there directly; else they are unpacked on the host from the packed buffer
    ArrayOut o{theta_out, err_out, cov_out, nll_out, edm_out, n_eval_out, n_iter_out, status_out};
    bool direct = b && status_out;
    const void* outs[8] = {theta_out, err_out, cov_out, nll_out, edm_out, n_eval_out, n_iter_out, status_out};
    for (int k = 0; k < 8 && direct; ++k)
        if (outs[k]) direct = device_writable(b, outs[k]);
    const int st = batch_fit_core(b, theta0, shared_start, lo, hi, step, fixed, opt_in, steps_out, &c,
                                  direct ? &o : nullptr);
    if (st != NLL_OK || b->n_toys == 0) return st;
    if (direct) {
        for (int t = 0; t < b->n_toys; ++t)
            if (status_out[t] != NLL_OK) return NLL_ERR_NOT_CONVERGED;
        return NLL_OK;
    }
    const int np = c.npar, nf = c.nf;
    int all = NLL_OK;
    for (int t = 0; t < b->n_toys; ++t) {
        const double* p = b->h_res + (size_t)t * kResStride;
        const double* tail = p + 2 * kNP + kNP * kNP;
        if (theta_out) memcpy(theta_out + (size_t)t * np, p, sizeof(double) * np);
        if (err_out) {
            double* e = err_out + (size_t)t * np;
            for (int k = 0; k < np; ++k) e[k] = 0.0;
            for (int i = 0; i < nf; ++i) e[c.idx[i]] = p[kNP + i];
        }
        if (cov_out) {
            double* v = cov_out + (size_t)t * np * np;
            memset(v, 0, sizeof(double) * np * np);
            for (int i = 0; i < nf; ++i)
                for (int j = 0; j < nf; ++j) v[c.idx[i] * np + c.idx[j]] = p[2 * kNP + i * nf + j];
        }
        if (nll_out) nll_out[t] = tail[0];
        if (edm_out) edm_out[t] = tail[1];
        if (n_eval_out) n_eval_out[t] = (int)tail[2];
        if (n_iter_out) n_iter_out[t] = (int)tail[3];
        const int status = (int)tail[4];
        if (status_out) status_out[t] = status;
        if (status != NLL_OK) all = NLL_ERR_NOT_CONVERGED;
    }
    return all;
}

int nll_batch_eval_hess(nll_batch* b, const double* thetas, int shared, double* nll_out, double* grad_out,
                        double* hess_out, double* w2_out, int* status_out)
{
    if (!b) return NLL_ERR_ARG;
    if (!b->loaded) return bfail(b, NLL_ERR_STATE, "no toys loaded");
    if (!thetas || !nll_out || !hess_out) return bfail(b, NLL_ERR_ARG, "null argument");
    if (cudaSetDevice(b->device) != cudaSuccess) return bfail(b, NLL_ERR_CUDA, "cudaSetDevice failed");
    const int n = b->n_toys, np = b->npar;
    if (n == 0) return NLL_OK;
    std::vector<double> th((size_t)n * np);
    for (int t = 0; t < n; ++t)
        for (int k = 0; k < np; ++k) th[(size_t)t * np + k] = thetas[(shared ? 0 : (size_t)t * np) + k];
    BatchDev d = make_dev(b);
    cudaError_t e = follow_user_stream(b);
    if (e != cudaSuccess) return bcuda(b, e, "stream order");
    int st = run_hess_pass(b, d.cfg, kHmEval, w2_out != nullptr, th.data());
    if (st != NLL_OK) return st;
    const size_t per = 1 + np + 2 * (size_t)np * np;
    std::vector<double> out(per * n);
    std::vector<int> sts(n);
    e = cudaMemcpyAsync(out.data(), b->hw.d_out, sizeof(double) * per * n, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sts.data(), b->hw.d_status, sizeof(int) * n, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "Hessian results");
    int first_bad = NLL_OK;
    for (int t = 0; t < n; ++t) {
        const double* o = out.data() + per * t;
        nll_out[t] = o[0];
        if (grad_out) memcpy(grad_out + (size_t)t * np, o + 1, sizeof(double) * np);
        memcpy(hess_out + (size_t)t * np * np, o + 1 + np, sizeof(double) * np * np);
        if (w2_out) memcpy(w2_out + (size_t)t * np * np, o + 1 + np + np * np, sizeof(double) * np * np);
        if (status_out) status_out[t] = sts[t];
        if (sts[t] != NLL_OK && first_bad == NLL_OK) first_bad = sts[t];
    }
    return first_bad;
}

}  // extern "C"
