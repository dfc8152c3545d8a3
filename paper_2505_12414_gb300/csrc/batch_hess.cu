// batch_hess.cu -- the analytic Hessian pass over many fits at once (batched toys and a
// server's slots; paper Sec. 2.1): the start matrices of the quasi-Newton steps (strategies
// 2, 3 and 5), the Newton polish passes and covariances (hessian 2 / 3), and
// nll_batch_eval_hess.
//   batch_hess_prep      (thread per toy)   the parameter-only terms of each toy's point
//   batch_hess_units     (persistent)       the per-event columns of (toy, 512-event) units
//                                           staged in shared memory, their slot products
//                                           summed per unit (batch_hess32_units: the same in
//                                           single precision, for start matrices)
//   batch_hess_totals    (warp per toy)     the units' sums in order
//   batch_hess_assemble  (thread per toy)   NLL, gradient, H and W from the totals
//   batch_hess_finish    (warp per toy)     start matrix, Newton step or results; for passes
//                                           over a few toys it also sums and assembles
// and on the host the work arrays, the unit lists and the polish loop.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "../../include/gbnll.h"
#include "batch_device.cuh"
#include "batch_internal.h"
#include "fp64_math.cuh"
#include "gbnll_internal.h"
#include "hess_device.cuh"
#include "nll_device.cuh"

namespace gbnll {
namespace {

// ---------------------------------------------------------------------------------
// analytic Hessian pass over all toys (paper Sec. 2.1): the start matrices of strategies
// 2, 3 and 5, the covariance of hessian 2 / 3, and nll_batch_eval_hess.  The per-event work is
// the single-sample Hessian pass (hess_device.cuh) over (toy, 512-event) units; then per toy
// the units' sums in order, the assembly of NLL, gradient, H (and W), and the mode's matrix
// work.
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
        LogProd lp = logprod_one();
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
            if (!W) {  // products across the warp, one logarithm per warp, into the ln P slot
                const LogProd wp = logprod_warp(lp);
                if (lane == 0) s_lnp[warp] = logprod_value(wp);
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

std::mutex g_btab_mutex;
bool g_btab_ready[64];

// this unit's copy of the device table, once per device
cudaError_t ensure_hess_btab()
{
    int device = 0;
    cudaError_t e = cudaGetDevice(&device);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_btab_mutex);
    if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
    if (g_btab_ready[device]) return cudaSuccess;
    std::vector<double> tab(kTabDoubles);
    fill_device_tables(tab.data());
    e = cudaMemcpyToSymbol(g_btab, tab.data(), sizeof(double) * kTabDoubles);
    if (e == cudaSuccess) g_btab_ready[device] = true;
    return e;
}

}  // namespace

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
    if (e == cudaSuccess) e = ensure_hess_btab();
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
