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
#include "batch_device.cuh"
#include "trace.h"
#include "tune_cache.h"

namespace gbnll {
namespace {


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
        LogProd lpx = logprod_one(), lpy = logprod_one();
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
    // 64 pairs: the smallest tile the work arrays are sized for (a smaller schedule tile stays)
    *step_tp = (4 * active <= n_toys) ? min(base_tp, max(base_tp / 4, 64)) : base_tp;
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
