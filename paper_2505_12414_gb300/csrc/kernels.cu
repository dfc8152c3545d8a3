// kernels.cu -- fused FP64 NLL + gradient kernels for sm_103a.
//
// Hot path of the unbinned maximum-likelihood fit (paper Sec. 2.1, Eq. 1): for every
// event, evaluate the normalised density with the parameter-only terms hoisted into a
// per-launch constant block (paper Sec. 2.4.1) and, for the 4D model, optionally the
// event-only angular basis read from memory (paper Sec. 2.4.2); take the logarithm;
// accumulate the few per-event sums from which the host assembles the gradient; reduce
// warp -> block -> grid in a fixed order.
//
// GB300 specifics that shape the code:
//  * FP64 throughput is scarce (about 1.2 TFLOP/s against about 7 TB/s of HBM), so the
//    per-event work is arranged to minimise FP64 instructions:
//      - the density is factored as P = exp(alpha (m - ma)) * Ptilde,
//        Ptilde = A(angles) exp(-b0 d^2 - alpha d + k0) + C(background), so one
//        exponential per event serves both mixture components;
//      - for unweighted samples sum_i ln Ptilde_i is taken as the logarithm of a running
//        product whose binary exponent is split off with integer instructions each event
//        (one logarithm per thread instead of one per event); sum_i alpha (m_i - ma) is
//        a constant of the sample, computed once at load;
//      - the exponential is a table-driven implementation (P. T. P. Tang, ACM TOMS 15
//        (1989) 144) with a 1024-entry table of 2^(j/1024) held in shared memory and an
//        economised cubic; the hoisted constants carry the argument scale 1024/ln2, so the
//        reduction is exact and costs 7 FP64 instructions; the reciprocal 1/Ptilde starts from the hardware
//        approximation rcp.approx.ftz.f64 and takes one cubically convergent correction
//        y (1 + e + e^2), e = 1 - x y;
//      - validity checks and the exponent bookkeeping use the integer pipe only.
//  * Events are SoA FP64 columns read with 128-bit (double2) coalesced loads; each
//    thread handles two consecutive events per iteration of a grid-stride loop, in one
//    basic block (the ragged tail masks the second event arithmetically, no branch), so
//    the two events' dependency chains interleave in the FP64 pipe.
//  * Warp reductions halve the slot count per shuffle level (ceil(K/2) + ceil(K/4) + ...
//    FP64 adds per warp: 23 for the 21 slots of the 4D gradient, 9 for the mass model's 7)
//    instead of a shuffle tree per slot.
//  * The grid is a small multiple of the SM count; block partial sums are written to a
//    scratch buffer and final_reduce_kernel, launched behind the fused kernel as a
//    programmatic dependent, adds them in a fixed order (one block per slot), so results
//    are bitwise reproducible for a given launch shape.

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <mutex>

#include "fp64_math.cuh"
#include "gbnll_internal.h"
#include "nll_device.cuh"

namespace gbnll {

__device__ double g_exp2tab[kTabDoubles];  // exp and sin/cos tables (fill_device_tables), once per device

// Work split: block b owns the contiguous pair range [b P / B, (b+1) P / B) (P pairs, B
// blocks), which its threads walk with a block-sized stride (coalesced).  Every block,
// hence every SM, gets the same work to within one pair.
// IP (in place): the columns are the caller's buffers (device or host memory the device
// reads), so the tail pair may not be read whole, and the kernel also sums w (m - ma) and
// counts events outside the ranges (slots KB-1 and KB; the bad count moves to the last slot).
// Registers: up to 255 (a 256-thread block still fits the register file).  In place, the
// kernel waits on host memory over NVLink-C2C: at most 168 registers (52-80 B spilled) let 12
// warps per SM (3 x 128) hide that latency instead of 8; measured 4 % faster per in-place step
// than the 242 registers the compiler otherwise takes (144 and 128: slower).
template <int KIND, int VAR, bool W, bool GRAD, bool IP = false>
__global__ void __maxnreg__(IP ? 168 : 255) fused_nll_kernel(const KArgs a)
{
    constexpr int KB = !GRAD ? kAccNll : (KIND == kMass1D ? kAcc1D : kAcc4D);
    constexpr int K = KB + (IP ? kAccInPlace : 0);
    __shared__ double s_tab[(KIND == kKstar4D && VAR == kVarDirect) ? kTabDoubles : (W ? kTrigOffset : kExpTable)];
    __shared__ double s_red[8 * K];

    // the final-sum kernel behind this one may be scheduled now: it waits (griddepcontrol.wait)
    // for this grid to complete, so its launch latency overlaps the event loop
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int64_t n = a.n;
    const int64_t npairs = (n + 1) >> 1;
    const int64_t begin = npairs * blockIdx.x / gridDim.x;
    const int64_t end = npairs * (blockIdx.x + 1) / gridDim.x;
    int64_t p = begin + threadIdx.x;

    // The table's loads are issued first and the first pair's behind them, so the block's
    // first barrier does not wait for the pair data; the sin/cos part of the table is
    // staged only where the angular basis is computed here.
    constexpr int ntab = (KIND == kKstar4D && VAR == kVarDirect) ? kTabDoubles : (W ? kTrigOffset : kExpTable);
    constexpr int nper = ntab / 64;  // per thread at the smallest block (64 threads)
    double tv[nper];
#pragma unroll
    for (int i = 0; i < nper; ++i) {
        const int j = threadIdx.x + i * blockDim.x;
        if (j < ntab) tv[i] = g_exp2tab[j];
    }
    PairIn in;
    if (p < end) load_pair<KIND, VAR, W, IP>(a, p, in);
#pragma unroll
    for (int i = 0; i < nper; ++i) {
        const int j = threadIdx.x + i * blockDim.x;
        if (j < ntab) s_tab[j] = tv[i];
    }
    __syncthreads();

    double acc[K];
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = 0.0;
    LogProd lpx = logprod_one(), lpy = logprod_one();
    int bad = 0;
    const KConst& c = a.c;

    // The direct variant reads few columns (4, +1 weight) and spends long on each pair: its next
    // pair's loads are issued before the current pair is processed (double-buffered in
    // registers), so their latency -- long from host memory -- overlaps the arithmetic.  The
    // precompute variant's 16 columns would not fit a second buffer; its loads are issued after.
    constexpr bool kAhead = VAR == kVarDirect;
    while (p < end) {
        const int64_t pn = p + blockDim.x;
        PairIn nx;
        if (kAhead && pn < end) load_pair<KIND, VAR, W, IP>(a, pn, nx);
        process_pair<KIND, VAR, W, GRAD>(c, in, (2 * p + 1) < n, acc, lpx, lpy, bad, s_tab);
        if (IP) inplace_pair<KIND, VAR, W>(a, in, (2 * p + 1) < n, acc[KB - 1], acc[KB]);
        p = pn;
        if (kAhead)
            in = nx;
        else if (p < end)
            load_pair<KIND, VAR, W, IP>(a, p, in);
    }
    if (!W) {
        // one logarithm per warp: multiply the running products across the warp first
        double lw = logprod_value(logprod_warp(logprod_combine(lpx, lpy)));
        acc[0] = (threadIdx.x & 31) == 0 ? lw : 0.0;
    }
    acc[K - 1] = (double)bad;
    if (KIND == kKstar4D && VAR == kVarDirect && GRAD) direct_unscale<K>(acc);
    block_partials<K>(acc, s_red, a.partials);
}

// Final sums of a fused launch: block k adds slot k's nb block partials in a fixed order
// (thread t takes blocks t, t + 64, ...; then a shuffle tree and the two warps), writes
// out[k] and, with `done` set, stores seq into done[k] after a system-scope fence, so a host
// thread polling done[0..K) reads complete results.  It is launched as a programmatic
// dependent of the fused kernel, which lets it be scheduled as soon as every fused block has
// started (griddepcontrol.launch_dependents at the top of the fused kernel):
// griddepcontrol.wait then returns once that grid has finished and its partials are visible,
// where a plain stream-ordered launch would start several microseconds later.  Spreading the K slots over
// K blocks (K SMs) keeps this step off the single-SM FP64 bottleneck a last-block reduction
// has, and needs no ticket or grid-wide fence in the fused kernel.
__global__ void __launch_bounds__(64) final_reduce_kernel(const double* partials, int nb, double* out,
                                                          unsigned int* done, unsigned int seq)
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    __shared__ double s_hi;
    const double* pk = partials + (int64_t)blockIdx.x * nb;
    double r = 0.0;
#pragma unroll 4
    for (int b = threadIdx.x; b < nb; b += 64) r += __ldcg(pk + b);
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    if (threadIdx.x == 32) s_hi = r;
    __syncthreads();
    if (threadIdx.x == 0) {
        out[blockIdx.x] = r + s_hi;
        if (done) {
            __threadfence_system();
            reinterpret_cast<volatile unsigned int*>(done)[blockIdx.x] = seq;
        }
    }
}

// ----------------------------------------------------------------------------------
// Load-time statistics and range validation: sum w, sum w (m - ma), events outside.  With
// dst pointers set, the kernel also stores what it reads there: columns in host memory that the
// device reads in place (pinned memory, or pageable memory with ATS) arrive in the event store
// in the same pass, with no copy-engine transfer or host-side staging copy.
// ----------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) stats_kernel(const SArgs a)
{
    __shared__ double s_red[8 * 3];
    double v[3] = {0.0, 0.0, 0.0};
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
        double w = a.w ? a.w[i] : 1.0;
        if (a.dst_w) a.dst_w[i] = w;
        bool outside = !(w >= 0.0 && w <= 1.0e300);  // also catches NaN
        for (int d = 0; d < a.ndim; ++d) {
            double x = a.col[d][i];
            if (a.dst[d]) a.dst[d][i] = x;
            outside |= !(x >= a.lo[d] && x <= a.hi[d]);
        }
        double m = a.col[0][i];
        v[0] += w;
        v[1] = fma(w, m - a.lo[0], v[1]);
        v[2] += outside ? 1.0 : 0.0;
    }
    grid_reduce<3>(v, s_red, a.partials, a.ticket, a.out);
}

// ----------------------------------------------------------------------------------
// Event-only precompute of the angular basis (paper Sec. 2.4.2), once per sample.
// ----------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) basis_kernel(const BArgs a)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
        double h[9], t2l, t2k, xp, t2p;
        angular_basis(a.ctl[i], a.ctk[i], a.phi[i], h, t2l, t2k, xp, t2p, g_exp2tab + kTrigOffset);
#pragma unroll
        for (int j = 0; j < 9; ++j) a.out[j][i] = h[j];
        a.out[9][i] = t2l;
        a.out[10][i] = t2k;
        a.out[11][i] = xp;
        a.out[12][i] = t2p;
    }
}

// ----------------------------------------------------------------------------------
// launchers
// ----------------------------------------------------------------------------------
int num_acc(int kind, bool grad) { return !grad ? kAccNll : (kind == kMass1D ? kAcc1D : kAcc4D); }

template <int KIND, int VAR, bool IP>
static int occ_kv(bool weighted, bool grad, int threads)
{
    int nb = 0;
    if (weighted) {
        if (grad)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fused_nll_kernel<KIND, VAR, true, true, IP>, threads, 0);
        else
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fused_nll_kernel<KIND, VAR, true, false, IP>, threads, 0);
    } else {
        if (grad)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fused_nll_kernel<KIND, VAR, false, true, IP>, threads, 0);
        else
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fused_nll_kernel<KIND, VAR, false, false, IP>, threads, 0);
    }
    return nb;
}

int fused_occupancy(int kind, int variant, bool weighted, bool grad, int threads, bool in_place)
{
    if (in_place) {  // in place: mass model, or the 4D direct variant (nothing precomputed)
        if (kind == kMass1D) return occ_kv<kMass1D, kVarPrecompute, true>(weighted, grad, threads);
        return occ_kv<kKstar4D, kVarDirect, true>(weighted, grad, threads);
    }
    if (kind == kMass1D) return occ_kv<kMass1D, kVarPrecompute, false>(weighted, grad, threads);
    if (variant == kVarDirect) return occ_kv<kKstar4D, kVarDirect, false>(weighted, grad, threads);
    return occ_kv<kKstar4D, kVarPrecompute, false>(weighted, grad, threads);
}

template <int KIND, int VAR, bool IP>
static cudaError_t launch_kv(bool weighted, bool grad, int blocks, int threads, cudaStream_t s, const KArgs& a)
{
    if (weighted) {
        if (grad)
            fused_nll_kernel<KIND, VAR, true, true, IP><<<blocks, threads, 0, s>>>(a);
        else
            fused_nll_kernel<KIND, VAR, true, false, IP><<<blocks, threads, 0, s>>>(a);
    } else {
        if (grad)
            fused_nll_kernel<KIND, VAR, false, true, IP><<<blocks, threads, 0, s>>>(a);
        else
            fused_nll_kernel<KIND, VAR, false, false, IP><<<blocks, threads, 0, s>>>(a);
    }
    return cudaGetLastError();
}

static cudaError_t launch_final(int nslots, int nb, cudaStream_t stream, const KArgs& a)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nslots);
    cfg.blockDim = dim3(64);
    cfg.stream = stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, final_reduce_kernel, (const double*)a.partials, nb, a.out, a.done, a.seq);
}

// The fused kernel (block partials) and, behind it, the final per-slot sums into a.out.
cudaError_t launch_fused(int kind, int variant, bool weighted, bool grad, int blocks, int threads,
                         cudaStream_t stream, const KArgs& a, bool in_place)
{
    if (threads > 256 || threads < 64 || (threads & 31) || blocks < 1) return cudaErrorInvalidValue;
    cudaError_t e;
    if (in_place) {
        if (kind == kMass1D)
            e = launch_kv<kMass1D, kVarPrecompute, true>(weighted, grad, blocks, threads, stream, a);
        else if (variant != kVarDirect)
            return cudaErrorInvalidValue;
        else
            e = launch_kv<kKstar4D, kVarDirect, true>(weighted, grad, blocks, threads, stream, a);
    } else if (kind == kMass1D) {
        e = launch_kv<kMass1D, kVarPrecompute, false>(weighted, grad, blocks, threads, stream, a);
    } else if (variant == kVarDirect) {
        e = launch_kv<kKstar4D, kVarDirect, false>(weighted, grad, blocks, threads, stream, a);
    } else {
        e = launch_kv<kKstar4D, kVarPrecompute, false>(weighted, grad, blocks, threads, stream, a);
    }
    if (e != cudaSuccess) return e;
    return launch_final(num_acc(kind, grad) + (in_place ? kAccInPlace : 0), blocks, stream, a);
}

cudaError_t launch_stats(int blocks, int threads, cudaStream_t stream, const SArgs& a)
{
    stats_kernel<<<blocks, threads, 0, stream>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_basis(int blocks, int threads, cudaStream_t stream, const BArgs& a)
{
    // the basis takes sin/cos phi from the table: present on every device it runs on
    cudaError_t e = ensure_device_tables();
    if (e != cudaSuccess) return e;
    basis_kernel<<<blocks, threads, 0, stream>>>(a);
    return cudaGetLastError();
}

namespace {
std::mutex g_tab_mutex;
bool g_tab_ready[64];
}  // namespace

cudaError_t ensure_device_tables()
{
    int device = 0;
    cudaError_t e = cudaGetDevice(&device);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_tab_mutex);
    if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
    if (g_tab_ready[device]) return cudaSuccess;
    static double tab[kTabDoubles];
    fill_device_tables(tab);
    e = cudaMemcpyToSymbol(g_exp2tab, tab, kTabDoubles * sizeof(double));
    if (e == cudaSuccess) g_tab_ready[device] = true;
    return e;
}

// ----------------------------------------------------------------------------------
// Static scratch for callers that cannot allocate device memory (nll_eval_grad_4d_noalloc).
// One array per process and device, holding the block partials of the in-place 4D launch
// ([kAccModel][kNoAllocMaxBlocks]) and its final sums (32 slots).  Nothing in it has to start
// at zero: every launch writes each partial and each sum it later reads.
// ----------------------------------------------------------------------------------
constexpr int kNoAllocDoubles = kAccModel * kNoAllocMaxBlocks + 32;
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

cudaError_t noalloc_scratch_setup(int device, NoAllocScratch* out)
{
    static std::mutex mu;
    static double* base[64] = {nullptr};
    if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (!base[device]) {
        // host code only sees a stand-in for the symbol: look up its device address, with
        // `device` current, once per device
        double* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress((void**)&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        base[device] = ptr;
    }
    out->partials = base[device];
    out->out = base[device] + (size_t)kAccModel * kNoAllocMaxBlocks;
    out->max_blocks = kNoAllocMaxBlocks;
    return cudaSuccess;
}

}  // namespace gbnll
