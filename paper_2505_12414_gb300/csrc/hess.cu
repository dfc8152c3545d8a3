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
//   * a warp runs only as many slot rows as its lanes own, and the few slots past the last
//     full warp row of the H table are summed by each event's staging thread (4D, 195 slots:
//     6 warp rows of FMAs per event instead of 7);
//   * unweighted, sum ln P is the logarithm of a running product per thread (one log per
//     thread, as in the fused kernel), added to its slot after the tiles;
//   * the staging uses the library's table-driven exponential and its reciprocal
//     (fp64_math.cuh), as the fused kernel does.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "fp64_math.cuh"
#include "gbnll_internal.h"
#include "hess_device.cuh"
#include "nll_device.cuh"

namespace gbnll {

__device__ double g_htab[kTabDoubles];  // exp and sin/cos tables, uploaded once per device

template <int KIND, int VAR, bool W>
__global__ void __launch_bounds__(kHessThreads) hess_kernel(const HArgs a)
{
    extern __shared__ double z[];
    __shared__ double s_tab[(KIND == kKstar4D && VAR == kVarDirect) ? kTabDoubles : (W ? kTrigOffset : kExpTable)];
    constexpr int TM = HessTailMax<KIND>::value;
    __shared__ double s_lnp[kHessThreads / 32];
    __shared__ double s_tred[(kHessThreads / 32) * TM];
    __shared__ uint8_t s_ti[TM], s_tj[TM];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    // the slot-total kernel behind this one may be scheduled now: it waits (griddepcontrol.wait)
    // for this grid to complete, so its launch latency overlaps the event loop
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    constexpr int ntab = (KIND == kKstar4D && VAR == kVarDirect) ? kTabDoubles : (W ? kTrigOffset : kExpTable);
    for (int j = t; j < ntab; j += kHessThreads) s_tab[j] = g_htab[j];
    const int ns = a.nslots;
    // Tail slots [tb, tb + tn) are summed by the staging thread of each event; when they end
    // the table the warp rows stop before them (195 slots: 6 rows instead of 7; the mass
    // model's table is all tail).
    const int tb = a.tail_begin, tn = a.tail_count;
    if (t < TM) {
        const int sr = t < tn ? tb + t : 0;
        s_ti[t] = a.sij[sr];
        s_tj[t] = a.sij[kHessMaxSlots + sr];
    }
    __syncthreads();
    const int ns_rows = (tn > 0 && tb + tn == ns) ? tb : ns;
    // slots t, t + 128, t + 256 of this thread; the warp runs as many slot rows as its first
    // lane owns (slots past the end, in the last partial row only, go to unused accumulators)
    const int w0 = t & ~31;
    const int nrow = ns_rows > w0 ? min(3, (ns_rows - w0 + kHessThreads - 1) / kHessThreads) : 0;
    double tacc[TM];
#pragma unroll
    for (int r = 0; r < TM; ++r) tacc[r] = 0.0;
    int ci[3], cj[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int s = t + k * kHessThreads;
        const int sc = s < ns ? s : 0;
        ci[k] = a.sij[sc];
        cj[k] = a.sij[kHessMaxSlots + sc];
    }
    double acc[3] = {0.0, 0.0, 0.0};
    LogProd lp = logprod_one();  // unweighted: product of this thread's densities
    const int64_t ntiles = (a.ev.n + kHessThreads - 1) / kHessThreads;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        stage_event<KIND, VAR, W>(a.ev, a.c, tile * kHessThreads + t, z, t, s_tab, lp);
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
    const int ls = a.lnp_slot;
    const bool lnp_in_tail = ls >= tb && ls < tb + tn;
    double lnp_tot = 0.0;
    if (!W) {
        // the threads' products multiplied across the warp (integer pipe), one logarithm per
        // warp, then the four warps in a fixed order, into the ln P slot
        const LogProd wp = logprod_warp(lp);
        if (lane == 0) s_lnp[warp] = logprod_value(wp);
        __syncthreads();
        lnp_tot = (s_lnp[0] + s_lnp[1]) + (s_lnp[2] + s_lnp[3]);
        if (ls >= 0 && !lnp_in_tail && t == (ls & (kHessThreads - 1))) {
            const double tot = lnp_tot;
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
    if (tn > 0) {  // tail slots: fixed tree over the block (slot tb + t in thread t)
        double tot = block_reduce<TM>(tacc, s_tred);
        if (t < tn) {
            if (!W && tb + t == ls) tot += lnp_tot;
            a.partials[(size_t)(tb + t) * nb + blockIdx.x] = tot;
        }
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int s = t + k * kHessThreads;
        if (s < ns && !(s >= tb && s < tb + tn)) a.partials[(size_t)s * nb + blockIdx.x] = acc[k];
    }
}

// Slot totals: block s sums the per-block partials of slot s (thread l takes blocks l,
// l + 128, ...), then a fixed butterfly per warp and the four warp sums in order; with
// `done` set it then stores seq into done[s] after a system-scope fence (the host polls
// these words).  Launched as a programmatic dependent of hess_kernel: griddepcontrol.wait
// returns once that grid has finished and its partials are visible.
__global__ void __launch_bounds__(kHessThreads) hess_reduce_kernel(const double* __restrict__ partials, int nb,
                                                                   double* __restrict__ out, unsigned int* done,
                                                                   unsigned int seq)
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    __shared__ double s_w[kHessThreads / 32];
    const int t = threadIdx.x, lane = t & 31, s = blockIdx.x;
    const double* p = partials + (size_t)s * nb;
    double v = 0.0;
    for (int b = t; b < nb; b += kHessThreads) v += p[b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) s_w[t >> 5] = v;
    __syncthreads();
    if (t == 0) {
        out[s] = (s_w[0] + s_w[1]) + (s_w[2] + s_w[3]);
        if (done) {
            __threadfence_system();
            reinterpret_cast<volatile unsigned int*>(done)[s] = seq;
        }
    }
}

// ------------------------------------------------------------------------------------
// Host: slot table and assembly (one piece of code serves both: the assembly is run once
// with a recording accessor to list the column pairs it reads, in first-use order)
// ------------------------------------------------------------------------------------
namespace {

struct Recorder {
    HessLayout* L;
    bool overflow = false;
    __host__ __device__ double operator()(int i, int j)  // host only in use; both for assemble_t
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

// slot sums by column pair through an inverse table (slot_of[i * 64 + j], 0xffff: none)
struct Reader {
    const uint16_t* slot_of;
    const double* sums;
    bool missing = false;
    __host__ __device__ double operator()(int i, int j)  // host only in use; both for assemble_t
    {
        const unsigned s = slot_of[i * 64 + j];
        if (s == 0xffffu) {
            missing = true;
            return NAN;
        }
        return sums[s];
    }
};

HessTerms terms_of(const Hoist& H)
{
    HessTerms T;
    T.alpha = H.alpha;
    T.f = H.f;
    T.sigma = H.sigma;
    T.b0 = H.b0;
    for (int k = 0; k < 3; ++k) {
        T.d2lnN1[k] = H.d2lnN1[k];
        T.dlnNc_dc2[k] = H.dlnNc_dc2[k];
    }
    T.d2lnN2t_dal2 = H.d2lnN2t_dal2;
    return T;
}

template <class Get>
double assemble_any(int kind, bool weighted, const Hoist& Hh, double sum_wdm, bool want_w2, Get& S, double* nll,
                    double* grad, double* Hm, double* Wm)
{
    const HessTerms H = terms_of(Hh);
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

static bool hess_layout_build(int kind, bool weighted, bool want_w2, HessLayout* L)
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
    // the H table's slots past its last full warp row (W slots are recorded after H's)
    int nh = L->nslots;
    if (want_w2) {
        HessLayout Lh;
        if (!hess_layout_build(kind, weighted, false, &Lh)) return false;
        nh = Lh.nslots;
    }
    const int r = nh % 32;
    if (kind == kMass1D && L->nslots <= kHessOwnMax) {  // every slot by the staging thread
        L->tail_begin = 0;
        L->tail_count = L->nslots;
    } else if (r > 0 && r <= kHessTailMax && !(L->lnp_slot >= nh - r && L->lnp_slot < nh)) {
        L->tail_begin = nh - r;
        L->tail_count = r;
    }
    return !rec.overflow;
}

namespace {
__device__ uint8_t g_hsij[8][2 * kHessMaxSlots];  // slot tables by layout key, per device
std::mutex g_hsij_mutex;
const uint8_t* g_hsij_addr[64][8];  // device address of each uploaded table (null: not yet)
}  // namespace

cudaError_t hess_slot_table(int kind, bool weighted, bool want_w2, const HessLayout& L, const uint8_t** out)
{
    int device = 0;
    cudaError_t e = cudaGetDevice(&device);
    if (e != cudaSuccess) return e;
    if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
    const int key = (kind == kMass1D ? 0 : 4) + (weighted ? 2 : 0) + (want_w2 ? 1 : 0);
    std::lock_guard<std::mutex> lock(g_hsij_mutex);
    if (!g_hsij_addr[device][key]) {
        uint8_t t[2 * kHessMaxSlots];
        memcpy(t, L.si, kHessMaxSlots);
        memcpy(t + kHessMaxSlots, L.sj, kHessMaxSlots);
        e = cudaMemcpyToSymbol(g_hsij, t, sizeof t, (size_t)key * sizeof t);
        if (e != cudaSuccess) return e;
        uint8_t* base = nullptr;
        e = cudaGetSymbolAddress((void**)&base, g_hsij);
        if (e != cudaSuccess) return e;
        g_hsij_addr[device][key] = base + (size_t)key * 2 * kHessMaxSlots;
    }
    *out = g_hsij_addr[device][key];
    return cudaSuccess;
}

// The slot table of (kind, weighted, W) is built once (recording the assembly is quadratic in
// the slot count) and copied out on every call.
// Layouts and their inverse maps (slot of each column pair), built once per (kind, weighted, W).
namespace {
std::mutex g_layout_mutex;
HessLayout g_layout[2][2][2];
uint16_t g_slot_of[2][2][2][64 * 64];
signed char g_layout_state[2][2][2];  // 0: not built, 1: built, -1: does not fit

signed char layout_state(int kind, bool weighted, bool want_w2)
{
    const int k = kind == kMass1D ? 0 : 1, w = weighted ? 1 : 0, x = want_w2 ? 1 : 0;
    std::lock_guard<std::mutex> lock(g_layout_mutex);
    signed char& st = g_layout_state[k][w][x];
    if (st == 0) {
        HessLayout& L = g_layout[k][w][x];
        st = hess_layout_build(kind, weighted, want_w2, &L) ? 1 : -1;
        if (st > 0) {
            uint16_t* so = g_slot_of[k][w][x];
            memset(so, 0xff, sizeof g_slot_of[k][w][x]);
            for (int s = 0; s < L.nslots; ++s) so[L.si[s] * 64 + L.sj[s]] = (uint16_t)s;
        }
    }
    return st;
}
}  // namespace

bool hess_layout(int kind, bool weighted, bool want_w2, HessLayout* L)
{
    if (layout_state(kind, weighted, want_w2) < 0) return false;
    *L = g_layout[kind == kMass1D ? 0 : 1][weighted ? 1 : 0][want_w2 ? 1 : 0];
    return true;
}

double hess_assemble(int kind, bool weighted, bool want_w2, const Hoist& H, double sum_wdm, const HessLayout& L,
                     const double* sums, double* nll, double* grad, double* hess, double* w2)
{
    if (layout_state(kind, weighted, want_w2) < 0) return NAN;
    (void)L;  // the cached inverse map of the same layout
    Reader rd{g_slot_of[kind == kMass1D ? 0 : 1][weighted ? 1 : 0][want_w2 ? 1 : 0], sums};
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

// Per device and kernel instance: the dynamic shared-memory attribute is set once, and the
// occupancy (resident blocks per SM) is computed once; both cost host API calls that would
// otherwise add to every pass (small samples are latency-bound).
constexpr int kHessInstances = 6;
template <int KIND, int VAR, bool W>
constexpr int hess_instance()
{
    return KIND == kMass1D ? (W ? 1 : 0) : (VAR == kVarDirect ? (W ? 3 : 2) : (W ? 5 : 4));
}
namespace {
std::mutex g_hinst_mutex;
signed char g_hinst_occ[64][kHessInstances];  // 0: not set up yet; else occupancy + 1 (0 -> error)
}  // namespace

template <int KIND, int VAR, bool W>
static int setup_t()
{
    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess || device < 0 || device >= 64) return -1;
    constexpr int slot = hess_instance<KIND, VAR, W>();
    std::lock_guard<std::mutex> lock(g_hinst_mutex);
    signed char& c = g_hinst_occ[device][slot];
    if (c == 0) {
        const size_t smem = hess_smem<KIND, VAR, W>();
        int nb = 0;
        if (cudaFuncSetAttribute(hess_kernel<KIND, VAR, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
                cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, hess_kernel<KIND, VAR, W>, kHessThreads, smem) !=
                cudaSuccess)
            return -1;  // not cached: the next call tries again
        c = (signed char)std::min(nb + 1, 127);
    }
    return c - 1;
}

template <int KIND, int VAR, bool W>
static cudaError_t launch_t(int blocks, cudaStream_t s, const HArgs& a)
{
    const size_t smem = hess_smem<KIND, VAR, W>();
    if (setup_t<KIND, VAR, W>() < 0) return cudaErrorInvalidValue;
    cudaError_t e;
    hess_kernel<KIND, VAR, W><<<blocks, kHessThreads, smem, s>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(a.nslots);
    cfg.blockDim = dim3(kHessThreads);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, hess_reduce_kernel, (const double*)a.partials, blocks, a.out, a.done, a.seq);
}

template <int KIND, int VAR, bool W>
static int occ_t()
{
    return std::max(setup_t<KIND, VAR, W>(), 0);
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
