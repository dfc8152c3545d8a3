// hess.cu -- analytic Hessian of the NLL and the squared-weight score matrix for sm_103a.
//
// Paper Sec. 2.1: with analytic derivatives the fitter also gets the Hessian (for the HESSE
// uncertainties and the Migrad start) and, for weighted fits, the Fisher information,
// whose sandwich H^-1 W H^-1 (W = sum_i w_i^2 s_i s_i^T, s_i = d ln P_i / dtheta) is the
// asymptotic covariance (Langenbruch, Eur. Phys. J. C 82 (2022) 393).
//
// Mathematics.  Both models are two-component mixtures P = f S + (1 - f) B with normalised
// components.  With the per-event shares ps = f S / P, pb = (1 - f) B / P (ps + pb = 1) and
// the component log-derivatives phi_a = d ln S / d a (signal parameters) or d ln B / d a
// (background parameters), the scores are s_a = ps phi_a, pb phi_a and
// s_f = ps / f - pb / (1 - f).  The NLL Hessian H = -sum w d^2 ln P splits as
//   a, b in the same component X:  -sum w ps pb phi_a phi_b - sum w p_X h_ab
//                                  (h_ab = d^2 ln X / da db - curvature of the component)
//   a, b in different components:   sum w s_a s_b
//   a = f, b in S (B):             -(+) sum w ps pb phi_b / (f (1 - f))
//   a = b = f:                      sum w s_f^2,
// and h is zero or a polynomial in d = m - mu for the mass terms, a constant for the
// exponential slope, and zero for the angular coefficients (the rate is linear in them,
// so there H_ab = sum w s_a s_b).  Every per-event product is formed without dividing by
// the angular rate or a Chebyshev factor (either may vanish inside the range): the
// background scores and cross terms carry the other factors instead of a quotient.
//
// GB300 mapping.  FP64 is the bound (~2 DFMA/clk/SM), so the kernel spends one FMA per
// slot per event and nothing else in its inner loop:
//   * a block of 128 threads stages the columns of 128 events (one thread per event) in
//     shared memory, column-major, ~60 KB for the 4D model (3 blocks per SM);
//   * each thread then owns up to three slots (column pairs, from the launch parameters)
//     and sums their products over the tile; thread l starts at event l and wraps, so a
//     half-warp's 64-bit reads fall in 16 different bank pairs whatever the columns;
//   * the grid is persistent (blocks take tiles b, b + B, ...); per-block slot sums go to
//     scratch and a second launch reduces them, one block per slot, in a fixed order
//     (deterministic, and spread over all SMs instead of one last block);
//   * a warp runs only as many slot rows as its lanes own (195 slots: 7 warp rows, not 8);
//   * unweighted, sum ln P is the logarithm of a running product per thread (one log per
//     thread, as in the fused kernel), added to its slot after the tiles;
//   * the staging uses the library's table-driven exponential and its reciprocal
//     (fp64_math.cuh), as the fused kernel does.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <mutex>
#include <vector>

#include "fp64_math.cuh"
#include "gbnll_internal.h"
#include "nll_device.cuh"

namespace gbnll {

__device__ double g_htab[kTabDoubles];  // exp and sin/cos tables, uploaded once per device

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
__device__ __forceinline__ void stage_event(const HArgs& a, int64_t e, double* z, int t, const double* tab,
                                            LogProd& lp)
{
    using L = HCols<KIND, W>;
    const HConst& c = a.c;
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
            angular_basis(xl, xk, __ldg(a.col[kColPhi] + ei), h, t2l, t2k, xp, t2p, tab + kExpTable);
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
        put(L::WLNP, ok ? w * log(P) : 0.0);
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

template <int KIND, int VAR, bool W>
__global__ void __launch_bounds__(kHessThreads) hess_kernel(const HArgs a)
{
    extern __shared__ double z[];
    __shared__ double s_tab[kTabDoubles];
    __shared__ double s_lnp[kHessThreads / 32];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    constexpr int ntab = (KIND == kKstar4D && VAR == kVarDirect) ? kTabDoubles : kExpTable;
    for (int j = t; j < ntab; j += kHessThreads) s_tab[j] = g_htab[j];
    __syncthreads();
    const int ns = a.nslots;
    // slots t, t + 128, t + 256 of this thread; the warp runs as many slot rows as its first
    // lane owns (slots past the end, in the last partial row only, go to unused accumulators)
    const int w0 = t & ~31;
    const int nrow = ns > w0 ? min(3, (ns - w0 + kHessThreads - 1) / kHessThreads) : 0;
    int ci[3], cj[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int s = t + k * kHessThreads;
        const int sc = s < ns ? s : 0;
        ci[k] = a.si[sc];
        cj[k] = a.sj[sc];
    }
    double acc[3] = {0.0, 0.0, 0.0};
    LogProd lp{1.0, 0};  // unweighted: product of this thread's densities
    const int64_t ntiles = (a.n + kHessThreads - 1) / kHessThreads;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        stage_event<KIND, VAR, W>(a, tile * kHessThreads + t, z, t, s_tab, lp);
        __syncthreads();
        if (nrow == 1)
            tile_slots<1>(z, ci, cj, acc, lane);
        else if (nrow == 2)
            tile_slots<2>(z, ci, cj, acc, lane);
        else if (nrow == 3)
            tile_slots<3>(z, ci, cj, acc, lane);
        __syncthreads();
    }
    if (!W) {
        // sum over the block of the threads' ln(products), fixed tree, into the ln P slot
        double v = logprod_value(lp);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) s_lnp[warp] = v;
        __syncthreads();
        const int ls = a.lnp_slot;
        if (ls >= 0 && t == (ls & (kHessThreads - 1))) {
            const double tot = (s_lnp[0] + s_lnp[1]) + (s_lnp[2] + s_lnp[3]);
            const int row = ls / kHessThreads;  // static indices keep acc in registers
            if (row == 0)
                acc[0] += tot;
            else if (row == 1)
                acc[1] += tot;
            else
                acc[2] += tot;
        }
    }
    const int nb = gridDim.x;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int s = t + k * kHessThreads;
        if (s < ns) a.partials[(size_t)s * nb + blockIdx.x] = acc[k];
    }
}

// Slot totals: block s sums the per-block partials of slot s (thread l takes blocks l,
// l + 128, ...), then a fixed butterfly per warp and the four warp sums in order.
__global__ void __launch_bounds__(kHessThreads) hess_reduce_kernel(const double* __restrict__ partials, int nb,
                                                                   double* __restrict__ out)
{
    __shared__ double s_w[kHessThreads / 32];
    const int t = threadIdx.x, lane = t & 31, s = blockIdx.x;
    const double* p = partials + (size_t)s * nb;
    double v = 0.0;
    for (int b = t; b < nb; b += kHessThreads) v += p[b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) s_w[t >> 5] = v;
    __syncthreads();
    if (t == 0) out[s] = (s_w[0] + s_w[1]) + (s_w[2] + s_w[3]);
}

// ------------------------------------------------------------------------------------
// Host: slot table and assembly (one piece of code serves both: the assembly is run once
// with a recording accessor to list the column pairs it reads, in first-use order)
// ------------------------------------------------------------------------------------
namespace {

struct Recorder {
    HessLayout* L;
    bool overflow = false;
    double operator()(int i, int j)
    {
        for (int s = 0; s < L->nslots; ++s)
            if (L->si[s] == i && L->sj[s] == j) return 0.0;
        if (L->nslots >= kHessMaxSlots) {
            overflow = true;
            return 0.0;
        }
        L->si[L->nslots] = (uint8_t)i;
        L->sj[L->nslots] = (uint8_t)j;
        ++L->nslots;
        return 0.0;
    }
};

struct Reader {
    const HessLayout* L;
    const double* sums;
    bool missing = false;
    double operator()(int i, int j)
    {
        for (int s = 0; s < L->nslots; ++s)
            if (L->si[s] == i && L->sj[s] == j) return sums[s];
        missing = true;
        return NAN;
    }
};

// Parameter classes: 0 mass shape (mu, sigma), 1 angular coefficient, 2 exponential slope,
// 3 Chebyshev coefficient, 4 signal fraction.
template <int KIND>
int pclass(int a)
{
    if (KIND == kMass1D) return a < 2 ? 0 : (a == 2 ? 2 : 4);
    if (a < 2) return 0;
    if (a < 10) return 1;
    if (a == 10) return 2;
    if (a < 17) return 3;
    return 4;
}

template <int KIND, bool W, class Get>
double assemble_t(const Hoist& Hh, double sum_wdm, bool want_w2, Get& S, double* nll, double* grad, double* Hm,
                  double* Wm)
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

template <class Get>
double assemble_any(int kind, bool weighted, const Hoist& H, double sum_wdm, bool want_w2, Get& S, double* nll,
                    double* grad, double* Hm, double* Wm)
{
    if (kind == kMass1D)
        return weighted ? assemble_t<kMass1D, true>(H, sum_wdm, want_w2, S, nll, grad, Hm, Wm)
                        : assemble_t<kMass1D, false>(H, sum_wdm, want_w2, S, nll, grad, Hm, Wm);
    return weighted ? assemble_t<kKstar4D, true>(H, sum_wdm, want_w2, S, nll, grad, Hm, Wm)
                    : assemble_t<kKstar4D, false>(H, sum_wdm, want_w2, S, nll, grad, Hm, Wm);
}

template <int KIND, bool W>
int ncols_of()
{
    return HCols<KIND, W>::NC;
}

}  // namespace

bool hess_layout(int kind, bool weighted, bool want_w2, HessLayout* L)
{
    memset(L, 0, sizeof *L);
    Hoist H;
    memset(&H, 0, sizeof H);
    H.f = 0.5;
    H.sigma = 1.0;
    double nll, grad[18], Hm[18 * 18], Wm[18 * 18];
    Recorder rec{L};
    assemble_any(kind, weighted, H, 0.0, want_w2, rec, &nll, grad, Hm, Wm);
    L->ncols = kind == kMass1D ? (weighted ? ncols_of<kMass1D, true>() : ncols_of<kMass1D, false>())
                               : (weighted ? ncols_of<kKstar4D, true>() : ncols_of<kKstar4D, false>());
    L->lnp_slot = -1;
    if (!weighted) {
        const int wl = kind == kMass1D ? HCols<kMass1D, false>::WLNP : HCols<kKstar4D, false>::WLNP;
        const int one = kind == kMass1D ? HCols<kMass1D, false>::ONE : HCols<kKstar4D, false>::ONE;
        for (int s = 0; s < L->nslots; ++s)
            if (L->si[s] == wl && L->sj[s] == one) L->lnp_slot = s;
        if (L->lnp_slot < 0) return false;
    }
    return !rec.overflow;
}

double hess_assemble(int kind, bool weighted, bool want_w2, const Hoist& H, double sum_wdm, const HessLayout& L,
                     const double* sums, double* nll, double* grad, double* hess, double* w2)
{
    Reader rd{&L, sums};
    double bad = assemble_any(kind, weighted, H, sum_wdm, want_w2, rd, nll, grad, hess, w2);
    return rd.missing ? NAN : bad;
}

void hess_fill_const(int kind, const Hoist& H, const double* theta, HConst* c)
{
    memset(c, 0, sizeof *c);
    c->mu = H.mu;
    c->b0 = H.b0;
    c->neg_b0s = -H.b0 * kExpArgScale;
    c->neg_als = -H.alpha * kExpArgScale;
    c->k0s = (H.lnb1 - H.alpha * (H.mu - H.ma)) * kExpArgScale;
    c->b2 = H.b2;
    c->inv_sigma = 1.0 / H.sigma;
    c->dlnN1_dmu = H.dlnN1_dmu;
    c->dlnN1_dsig = H.dlnN1_dsig;
    c->mu_ma = H.mu - H.ma;
    c->dlnN2t_dal = H.dlnN2t_dal;
    c->inv_f = 1.0 / H.f;
    c->inv_1mf = 1.0 / (1.0 - H.f);
    if (kind == kKstar4D) {
        for (int k = 0; k < 8; ++k) c->ang[k] = theta[2 + k];
        for (int j = 0; j < 3; ++j) {
            c->c1[j] = theta[11 + 2 * j];
            c->c2[j] = theta[12 + 2 * j];
            c->dl[j] = H.dlnNc_dc2[j];
        }
    }
}

template <int KIND, int VAR, bool W>
static size_t hess_smem()
{
    return (size_t)HCols<KIND, W>::NC * kHessThreads * sizeof(double);
}

template <int KIND, int VAR, bool W>
static cudaError_t launch_t(int blocks, cudaStream_t s, const HArgs& a)
{
    const size_t smem = hess_smem<KIND, VAR, W>();
    cudaError_t e = cudaFuncSetAttribute(hess_kernel<KIND, VAR, W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    hess_kernel<KIND, VAR, W><<<blocks, kHessThreads, smem, s>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    hess_reduce_kernel<<<a.nslots, kHessThreads, 0, s>>>(a.partials, blocks, a.out);
    return cudaGetLastError();
}

template <int KIND, int VAR, bool W>
static int occ_t()
{
    const size_t smem = hess_smem<KIND, VAR, W>();
    if (cudaFuncSetAttribute(hess_kernel<KIND, VAR, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, hess_kernel<KIND, VAR, W>, kHessThreads, smem) !=
        cudaSuccess)
        return 0;
    return nb;
}

namespace {
std::mutex g_htab_mutex;
bool g_htab_ready[64];

cudaError_t ensure_htab()
{
    int device = 0;
    cudaError_t e = cudaGetDevice(&device);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_htab_mutex);
    if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
    if (g_htab_ready[device]) return cudaSuccess;
    std::vector<double> tab(kTabDoubles);
    fill_device_tables(tab.data());
    e = cudaMemcpyToSymbol(g_htab, tab.data(), sizeof(double) * kTabDoubles);
    if (e == cudaSuccess) g_htab_ready[device] = true;
    return e;
}
}  // namespace

cudaError_t launch_hess(int kind, int variant, bool weighted, int blocks, cudaStream_t stream, const HArgs& a)
{
    if (a.nslots <= 0 || a.nslots > kHessMaxSlots || blocks <= 0) return cudaErrorInvalidValue;
    cudaError_t e = ensure_htab();
    if (e != cudaSuccess) return e;
    if (kind == kMass1D)
        return weighted ? launch_t<kMass1D, kVarPrecompute, true>(blocks, stream, a)
                        : launch_t<kMass1D, kVarPrecompute, false>(blocks, stream, a);
    if (variant == kVarDirect)
        return weighted ? launch_t<kKstar4D, kVarDirect, true>(blocks, stream, a)
                        : launch_t<kKstar4D, kVarDirect, false>(blocks, stream, a);
    return weighted ? launch_t<kKstar4D, kVarPrecompute, true>(blocks, stream, a)
                    : launch_t<kKstar4D, kVarPrecompute, false>(blocks, stream, a);
}

int hess_occupancy(int kind, int variant, bool weighted)
{
    if (kind == kMass1D) return weighted ? occ_t<kMass1D, kVarPrecompute, true>() : occ_t<kMass1D, kVarPrecompute, false>();
    if (variant == kVarDirect)
        return weighted ? occ_t<kKstar4D, kVarDirect, true>() : occ_t<kKstar4D, kVarDirect, false>();
    return weighted ? occ_t<kKstar4D, kVarPrecompute, true>() : occ_t<kKstar4D, kVarPrecompute, false>();
}

}  // namespace gbnll
