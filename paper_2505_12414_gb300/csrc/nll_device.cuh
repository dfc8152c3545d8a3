// nll_device.cuh -- per-event bodies, pair loads and fixed-order reductions shared by the
// single-sample kernels (kernels.cu) and the batched pseudo-experiment kernels (batch.cu).
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "fp64_math.cuh"
#include "gbnll_internal.h"

namespace gbnll {

// ----------------------------------------------------------------------------------
// Angular basis (paper Sec. 2.4.2, Eq. 3 regrouped by parameter):
//   A = h0 + FL hFL + S3 h3 + S4 h4 + S5 h5 + AFB h6 + S7 h7 + S8 h8 + S9 h9,
//   h0 = c sin^2 tK (3/4 + cos 2tl / 4), hFL = c cos^2 tK (1 - cos 2tl) - h0, ...
// with c = 9/(32 pi).  Also the Chebyshev inputs T2(ctl), T2(ctk), phi/pi, T2(phi/pi).
// sin tK and sin tl enter only as their product (one square root of the product of the
// squares, fsqrt), and sin/cos phi come from the table method (trig = the |cos|, |sin| table).
// ----------------------------------------------------------------------------------
__device__ __forceinline__ void angular_basis(double ctl, double ctk, double phi, double h[9], double& t2l,
                                              double& t2k, double& xp, double& t2p, const double* trig)
{
    const double c = 0x1.6eb167b830193p-4;   // 9/(32 pi)
    const double c2 = 0x1.6eb167b830193p-3;  // 2 c
    const double kInvPi = 0x1.45f306dc9c883p-2;
    const double sl2 = fma(-ctl, ctl, 1.0), sk2 = fma(-ctk, ctk, 1.0);  // sin^2 tl, sin^2 tK
    const double sksl = fsqrt(sk2 * sl2);                               // sin tK sin tl
    double sp, cp;
    fsincos_pi(phi, trig, sp, cp);
    t2l = fma(-2.0, sl2, 1.0);  // cos 2tl = 1 - 2 sin^2 tl
    t2k = fma(-2.0, sk2, 1.0);
    const double csk2 = c * sk2;
    const double h0 = csk2 * fma(0.25, t2l, 0.75);
    const double a = csk2 * sl2;            // c sin^2 tK sin^2 tl
    const double b = c2 * ctk * sksl;       // c sin 2tK sin tl
    const double bc = b * cp, bs = b * sp, ctl2 = ctl + ctl;
    h[0] = h0;
    h[1] = fma(fma(-2.0, csk2, c2), sl2, -h0);  // c cos^2 tK (1 - cos 2tl) - h0
    h[2] = a * fma(cp + cp, cp, -1.0);          // S3: a cos 2phi
    h[3] = ctl2 * bc;                           // S4: c sin 2tK sin 2tl cos phi
    h[4] = bc;                                  // S5
    h[5] = csk2 * (4.0 / 3.0) * ctl;            // AFB: 4/3 c sin^2 tK cos tl
    h[6] = bs;                                  // S7
    h[7] = ctl2 * bs;                           // S8
    h[8] = a * ((sp + sp) * cp);                // S9: a sin 2phi
    xp = phi * kInvPi;
    t2p = fma(xp + xp, xp, -1.0);
}

// The same basis without its constant factors, for evaluations that compute it per event
// (direct variant): h_k = c F_k q_k with c = 9/(32 pi) and F_k = direct_factor(k) (F_0 = 1),
//   q0 = sK^2 (1 - sl^2/2), q1 = 2 cK^2 sl^2 - q0, q2 = sK^2 sl^2 cos 2phi,
//   q3 = ctl q4, q4 = ctK sK sl cos phi, q5 = sK^2 ctl, q6 = ctK sK sl sin phi, q7 = ctl q6,
//   q8 = sK^2 sl^2 sin phi cos phi,
// which saves the multiplications by c, 2, 4 and 4/3 (the callers put c into the exponent
// and F_k into the coefficients and the gradient sums).
__device__ __forceinline__ void angular_basis_direct(double ctl, double ctk, double phi, double q[9], double& t2l,
                                                     double& t2k, double& xp, double& t2p, const double* trig)
{
    const double kInvPi = 0x1.45f306dc9c883p-2;
    const double sl2 = fma(-ctl, ctl, 1.0), sk2 = fma(-ctk, ctk, 1.0);
    const double a = sk2 * sl2;
    const double sksl = fsqrt(a);
    double sp, cp;
    fsincos_pi(phi, trig, sp, cp);
    t2l = fma(-2.0, sl2, 1.0);
    t2k = fma(-2.0, sk2, 1.0);
    const double q0 = fma(-0.5, a, sk2);
    const double ck2 = ctk * ctk;
    const double bq = ctk * sksl;
    const double q4 = bq * cp, q6 = bq * sp;
    q[0] = q0;
    q[1] = fma(ck2 + ck2, sl2, -q0);
    q[2] = a * fma(cp + cp, cp, -1.0);
    q[3] = ctl * q4;
    q[4] = q4;
    q[5] = sk2 * ctl;
    q[6] = q6;
    q[7] = ctl * q6;
    q[8] = a * (sp * cp);
    xp = phi * kInvPi;
    t2p = fma(xp + xp, xp, -1.0);
}

// Per-thread gradient sums of the direct variant back to the basis h_k: sum R E' q_k times F_k.
template <int K>
__device__ __forceinline__ void direct_unscale(double (&acc)[K])
{
#pragma unroll
    for (int k = 0; k < 8; ++k)
        if (direct_factor(k + 1) != 1.0) acc[4 + k] *= direct_factor(k + 1);
}

// ----------------------------------------------------------------------------------
// Per-event bodies.  acc[] slots as documented in gbnll_internal.h.  `valid` == false
// turns the event into an exact no-op (factor 1 in the product, R = 0 in every sum), so
// both events of a pair run in one basic block and their dependency chains interleave.
// ----------------------------------------------------------------------------------
template <bool W, bool GRAD>
__device__ __forceinline__ void event_mass(const KConst& c, double m, double w, bool valid, double* acc,
                                           LogProd& lp, int& bad, const double* tab)
{
    double d = m - c.mu;
    double E = fexp_scaled(fma(d, fma(c.neg_b0, d, c.neg_alpha), c.k0), tab);
    double P = E + c.b2;
    bad |= valid ? not_positive_normal(P) : 0;
    P = valid ? P : 1.0;
    if (W)
        acc[0] = fma(valid ? w : 0.0, flog(P, tab), acc[0]);
    else
        logprod_mul(lp, P);
    if (GRAD) {
        double R = frcp(P);
        if (W) R *= w;
        R = valid ? R : 0.0;
        double rs = R * E;
        acc[1] += rs;
        double rsd = rs * d;
        acc[2] += rsd;
        acc[3] = fma(rsd, d, acc[3]);
        acc[4] += R;
        acc[5] = fma(R, d, acc[5]);
    }
}

template <bool W, bool GRAD, bool DIR = false>
__device__ __forceinline__ void event_4d(const KConst& c, double m, const double h[9], double xl, double t2l,
                                         double xk, double t2k, double xp, double t2p, double w, bool valid,
                                         double* acc, LogProd& lp, int& bad, const double* tab)
{
    double d = m - c.mu;
    double E = fexp_scaled(fma(d, fma(c.neg_b0, d, c.neg_alpha), DIR ? c.k0d : c.k0), tab);
    double A = fma(DIR ? c.angd[0] : c.ang[0], h[1], h[0]);
#pragma unroll
    for (int k = 1; k < 8; ++k) A = fma(DIR ? c.angd[k] : c.ang[k], h[k + 1], A);
    double C1 = fma(c.cq[1], xl, fma(c.cq[2], t2l, c.cq[0]));
    double C2 = fma(c.cq[4], xk, fma(c.cq[5], t2k, c.cq[3]));
    double C3 = fma(c.cq[7], xp, fma(c.cq[8], t2p, c.cq[6]));
    double C12 = C1 * C2;
    double C = C12 * C3;
    double P = fma(A, E, C);
    bad |= valid ? not_positive_normal(P) : 0;
    P = valid ? P : 1.0;
    if (W)
        acc[0] = fma(valid ? w : 0.0, flog(P, tab), acc[0]);
    else
        logprod_mul(lp, P);
    if (GRAD) {
        double R = frcp(P);
        if (W) R *= w;
        R = valid ? R : 0.0;
        double rE = R * E;
        double rs = rE * A;
        acc[1] += rs;
        double rsd = rs * d;
        acc[2] += rsd;
        acc[3] = fma(rsd, d, acc[3]);
#pragma unroll
        for (int k = 0; k < 8; ++k) acc[4 + k] = fma(rE, h[k + 1], acc[4 + k]);
        // R C/C_j for the three background factors, and R C
        double u3 = R * C12;
        double rc3 = R * C3;
        double u1 = rc3 * C2;
        double u2 = rc3 * C1;
        double re = u3 * C3;
        acc[12] += re;
        acc[13] = fma(re, d, acc[13]);
        acc[14] = fma(u1, xl, acc[14]);
        acc[15] = fma(u1, t2l, acc[15]);
        acc[16] = fma(u2, xk, acc[16]);
        acc[17] = fma(u2, t2k, acc[17]);
        acc[18] = fma(u3, xp, acc[18]);
        acc[19] = fma(u3, t2p, acc[19]);
    }
}

// ----------------------------------------------------------------------------------
// Fixed-order reductions
// ----------------------------------------------------------------------------------

// Warp reduction of K slots by recursive halving: at each level a lane keeps the lower or
// upper part of the slots it holds (the lower part has ceil(n/2) of its n slots, the upper the
// rest, padded with a zero), sends the other part to lane ^ s and adds what it receives, so
// the warp spends ceil(K/2) + ceil(K/4) + ... FP64 additions (23 for 21 slots, 21 for 19)
// instead of 5 K.  On return each lane holds the warp total of slot reduce_slot_of<K>(lane)
// (-1: none).  The pairing is fixed, so the result is deterministic.
template <int K>
__device__ __forceinline__ int reduce_slot_of(int lane)
{
    // the split of each level is the same for all lanes: h = ceil(n/2) of the n = K, ceil(K/2),
    // ... slots the level starts from; a lane's group holds min(cnt, h) (lower) or
    // max(cnt - h, 0) (upper) of them
    int first = 0, cnt = K, n = K;
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
        const int h = (n + 1) >> 1;
        if (lane & s) {
            first += h;
            cnt = cnt > h ? cnt - h : 0;
        } else {
            cnt = cnt < h ? cnt : h;
        }
        n = h;
    }
    return cnt == 1 ? first : -1;
}

template <int K>
__device__ __forceinline__ double warp_reduce_slots(const double (&in)[K])
{
    static_assert(K <= 32, "at most 32 slots");
    const int lane = threadIdx.x & 31;
    double v[K];
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = in[k];
    constexpr int h16 = (K + 1) >> 1, h8 = (h16 + 1) >> 1, h4 = (h8 + 1) >> 1, h2 = (h4 + 1) >> 1;
    // one level: n slots held, h = ceil(n/2) kept (indices past n read as zero)
#define GBNLL_HALVE(S, N, H)                                                  \
    {                                                                         \
        const bool upper = (lane & (S)) != 0;                                 \
        _Pragma("unroll") for (int i = 0; i < (H); ++i)                       \
        {                                                                     \
            const double hi = (i + (H) < (N)) ? v[(i + (H)) % K] : 0.0;       \
            const double send = upper ? v[i] : hi;                            \
            const double keep = upper ? hi : v[i];                            \
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, (S));            \
        }                                                                     \
    }
    GBNLL_HALVE(16, K, h16)
    GBNLL_HALVE(8, h16, h8)
    GBNLL_HALVE(4, h8, h4)
    GBNLL_HALVE(2, h4, h2)
    GBNLL_HALVE(1, h2, 1)
#undef GBNLL_HALVE
    return v[0];
}

// Reduce K per-thread values over the block; the result is valid in threads 0..K-1.
template <int K>
__device__ __forceinline__ double block_reduce(const double (&v)[K], double* smem)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    double s = warp_reduce_slots<K>(v);
    const int slot = reduce_slot_of<K>(lane);
    if (slot >= 0) smem[warp * K + slot] = s;
    __syncthreads();
    double res = 0.0;
    if (threadIdx.x < K) {
        for (int w = 0; w < nwarps; ++w) res += smem[w * K + threadIdx.x];
    }
    __syncthreads();
    return res;
}

// Block partials -> scratch; the last block to arrive sums them in a fixed order into
// out[0..K) and resets the ticket for the next launch (used by the load-time statistics).
template <int K>
__device__ __forceinline__ void grid_reduce(const double (&v)[K], double* smem, double* partials,
                                            unsigned int* ticket, double* out)
{
    __shared__ int s_last;
    const int nb = gridDim.x;
    double bsum = block_reduce<K>(v, smem);
    if (threadIdx.x < K) partials[threadIdx.x * nb + blockIdx.x] = bsum;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(ticket, 1u) == (unsigned)(nb - 1));
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double acc[K];
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
#pragma unroll
        for (int k = 0; k < K; ++k) acc[k] += __ldcg(partials + k * nb + b);
    }
    double tot = block_reduce<K>(acc, smem);
    if (threadIdx.x < K) out[threadIdx.x] = tot;
    if (threadIdx.x == 0) *ticket = 0u;
}

// Block partials -> scratch, slot-major (partials[k * nb + block]); the final sums are
// taken by final_reduce_kernel, launched behind the fused kernel.
template <int K>
__device__ __forceinline__ void block_partials(const double (&v)[K], double* smem, double* partials)
{
    double bsum = block_reduce<K>(v, smem);
    if (threadIdx.x < K) partials[threadIdx.x * gridDim.x + blockIdx.x] = bsum;
}

// ----------------------------------------------------------------------------------
// The fused kernel
// ----------------------------------------------------------------------------------
__device__ __forceinline__ double2 ld2(const double* col, int64_t p)
{
    return __ldg(reinterpret_cast<const double2*>(col) + p);
}

// Inputs of one pair of consecutive events (one 128-bit load per column).
struct PairIn {
    double2 m, w, l, k, f;
    double2 h[9];
    double2 t2l, t2k, xp, t2p;
};

// 128-bit load of events 2p, 2p+1; with TAIL, a pair whose second event is past n loads the
// first event alone (the caller's buffer may end there) and repeats it.
template <bool TAIL>
__device__ __forceinline__ double2 ld2t(const double* col, int64_t p, bool whole)
{
    if (!TAIL || whole) return ld2(col, p);
    const double x = __ldg(col + 2 * p);
    return make_double2(x, x);
}

template <int KIND, int VAR, bool W, bool TAIL = false>
__device__ __forceinline__ void load_pair(const KArgs& a, int64_t p, PairIn& in)
{
    const bool whole = !TAIL || 2 * p + 1 < a.n;
    in.m = ld2t<TAIL>(a.col[kColM], p, whole);
    if (W) in.w = ld2t<TAIL>(a.w, p, whole);
    if (KIND == kKstar4D) {
        in.l = ld2t<TAIL>(a.col[kColCtl], p, whole);
        in.k = ld2t<TAIL>(a.col[kColCtk], p, whole);
        if (VAR == kVarPrecompute) {
#pragma unroll
            for (int j = 0; j < 9; ++j) in.h[j] = ld2(a.col[kColH0 + j], p);
            in.t2l = ld2(a.col[kColT2l], p);
            in.t2k = ld2(a.col[kColT2k], p);
            in.xp = ld2(a.col[kColXp], p);
            in.t2p = ld2(a.col[kColT2p], p);
        } else {
            in.f = ld2t<TAIL>(a.col[kColPhi], p, whole);
        }
    }
}

// Order key of a double (see order_key_host): integer-pipe range checks.
__device__ __forceinline__ long long order_key(double x)
{
    const long long b = __double_as_longlong(x);
    return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}

__device__ __forceinline__ int outside_key(double x, long long lo, long long hi)
{
    const long long k = order_key(x);
    return (k < lo) | (k > hi);
}

// In-place evaluation: sum w (m - ma) and the count of events outside the ranges (integer
// compares) for one pair; `second` masks the tail.
template <int KIND, int VAR, bool W>
__device__ __forceinline__ void inplace_pair(const KArgs& a, const PairIn& in, bool second, double& wdm,
                                             double& outside)
{
    const double wx = W ? in.w.x : 1.0, wy = W ? in.w.y : 1.0;
    const double dy = second ? in.m.y - a.ma : 0.0;
    wdm = fma(wx, in.m.x - a.ma, wdm);
    wdm = fma(wy, dy, wdm);
    int ox = outside_key(in.m.x, a.klo[0], a.khi[0]), oy = outside_key(in.m.y, a.klo[0], a.khi[0]);
    if (W) {
        ox |= outside_key(wx, a.klo[4], a.khi[4]);
        oy |= outside_key(wy, a.klo[4], a.khi[4]);
    }
    if (KIND == kKstar4D && VAR == kVarDirect) {
        ox |= outside_key(in.l.x, a.klo[1], a.khi[1]) | outside_key(in.k.x, a.klo[2], a.khi[2]) |
              outside_key(in.f.x, a.klo[3], a.khi[3]);
        oy |= outside_key(in.l.y, a.klo[1], a.khi[1]) | outside_key(in.k.y, a.klo[2], a.khi[2]) |
              outside_key(in.f.y, a.klo[3], a.khi[3]);
    }
    outside += (double)(ox + (second ? oy : 0));
}

template <int KIND, int VAR, bool W, bool GRAD>
__device__ __forceinline__ void process_pair(const KConst& c, const PairIn& in, bool second, double* acc,
                                             LogProd& lpx, LogProd& lpy, int& bad, const double* tab)
{
    const double wx = W ? in.w.x : 1.0, wy = W ? in.w.y : 1.0;
    if (KIND == kMass1D) {
        event_mass<W, GRAD>(c, in.m.x, wx, true, acc, lpx, bad, tab);
        event_mass<W, GRAD>(c, in.m.y, wy, second, acc, lpy, bad, tab);
    } else {
        double hx[9], hy[9];
        double t2lx, t2ly, t2kx, t2ky, xpx, xpy, t2px, t2py;
        if (VAR == kVarPrecompute) {
#pragma unroll
            for (int j = 0; j < 9; ++j) {
                hx[j] = in.h[j].x;
                hy[j] = in.h[j].y;
            }
            t2lx = in.t2l.x;
            t2ly = in.t2l.y;
            t2kx = in.t2k.x;
            t2ky = in.t2k.y;
            xpx = in.xp.x;
            xpy = in.xp.y;
            t2px = in.t2p.x;
            t2py = in.t2p.y;
        } else {  // factored basis: the caller applies direct_unscale to the gradient sums
            angular_basis_direct(in.l.x, in.k.x, in.f.x, hx, t2lx, t2kx, xpx, t2px, tab + kTrigOffset);
            angular_basis_direct(in.l.y, in.k.y, in.f.y, hy, t2ly, t2ky, xpy, t2py, tab + kTrigOffset);
        }
        constexpr bool DIR = VAR != kVarPrecompute;
        event_4d<W, GRAD, DIR>(c, in.m.x, hx, in.l.x, t2lx, in.k.x, t2kx, xpx, t2px, wx, true, acc, lpx, bad, tab);
        event_4d<W, GRAD, DIR>(c, in.m.y, hy, in.l.y, t2ly, in.k.y, t2ky, xpy, t2py, wy, second, acc, lpy, bad, tab);
    }
}

}  // namespace gbnll
