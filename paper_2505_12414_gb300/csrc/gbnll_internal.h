// gbnll_internal.h -- structures shared by the CUDA kernels (kernels.cu) and the host
// runtime (runtime.cu).  Not part of the public C ABI (include/gbnll.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <string>

namespace gbnll {

constexpr int kMass1D = 1;
constexpr int kKstar4D = 2;

// Angular-part variants of the 4D kernel (paper Sec. 2.4.2).
constexpr int kVarPrecompute = 1;  // read the event-only basis built at load
constexpr int kVarDirect = 2;      // recompute the basis from the angles per evaluation

// Columns of the structure-of-arrays event store.  Every column holds n_pad doubles and
// starts on a 256-byte boundary.
enum Col : int {
    kColM = 0,     // mass
    kColCtl = 1,   // cos theta_l          (4D)
    kColCtk = 2,   // cos theta_K          (4D)
    kColPhi = 3,   // phi                  (4D)
    kColH0 = 4,    // basis: h0, hFL, h_S3 .. h_S9  (9 columns, 4D precompute)
    kColT2l = 13,  // 2 ctl^2 - 1
    kColT2k = 14,  // 2 ctk^2 - 1
    kColXp = 15,   // phi / pi
    kColT2p = 16,  // 2 (phi/pi)^2 - 1
    kNumCols = 17
};

// Accumulator slots of the fused kernels.  Every slot is an FP64 sum over events
// (slot 0 = sum of w ln Ptilde; the last slot counts invalid densities).
//   mass model : lnp, R s, R s d, R s d^2, R, R d, bad
//   4D model   : lnp, R s, R s d, R s d^2, R E h_k (8: FL, S3..S9), R C, R C d,
//                R C/C1 {x1, T2(x1)}, R C/C2 {x2, T2(x2)}, R C/C3 {x3, T2(x3)}, bad
//   NLL only   : lnp, bad
// with d = m - mu, E the Gaussian factor, R = w / Ptilde, s = A E, C the background
// factor (see kernels.cu for the factorisation).
constexpr int kAcc1D = 7;
constexpr int kAcc4D = 21;
constexpr int kAccNll = 2;
constexpr int kAccMax = 21;
// In-place evaluation (events read where the caller keeps them, nothing stored at load) adds
// two sums the load-time statistics supply otherwise: sum w (m - ma) and the count of events
// outside the observable ranges or with invalid weights.
constexpr int kAccInPlace = 2;
constexpr int kAccModel = kAccMax + kAccInPlace;  // slots of a model's own reduction buffers

// Per-launch constant block: every parameter-only term the per-event work needs
// (paper Sec. 2.4.1: terms that depend on the parameters only are computed once per
// parameter point on the host and passed to the kernel).
struct KConst {
    double mu;         // Gaussian mean
    double neg_b0;     // -S/(2 sigma^2)          (S = N/ln2, the exponential's argument scale)
    double neg_alpha;  // -S alpha
    double k0;         // S (ln b1 - alpha (mu - ma)); scaled exponent = d (neg_b0 d + neg_alpha) + k0
    double b2;         // mass model: background constant (1-f) / Ntilde2
    double ang[8];     // FL, S3, S4, S5, AFB, S7, S8, S9
    double cq[9];      // background factors: C_j = cq[3j] + cq[3j+1] x_j + cq[3j+2] T2(x_j)
    // 4D, angular basis computed per evaluation (direct variant), which drops the basis'
    // constant factors: h_k = c F_k q_k with c = 9/(32 pi) (direct_factor gives F_k), so
    // A = c (q_0 + sum_k ang_k F_k q_k); c goes into the exponent, F_k into the coefficients.
    double k0d;        // S (ln b1 + ln c - alpha (mu - ma))
    double angd[8];    // ang[k] F_{k+1}
};

// F_k of the direct variant's basis (k = 1..8: FL, S3, S4, S5, AFB, S7, S8, S9).
__host__ __device__ constexpr double direct_factor(int k)
{
    return k == 3 || k == 7 ? 4.0 : (k == 4 || k == 6 || k == 8) ? 2.0 : k == 5 ? 4.0 / 3.0 : 1.0;
}
constexpr double kLnBasisC = -2.41324121131290733843909748479889;  // ln(9 / (32 pi))

struct KArgs {
    const double* col[kNumCols];  // device column pointers (unused ones NULL)
    const double* w;              // weights or NULL
    int64_t n;                    // events
    KConst c;
    double* partials;             // [K][max_blocks] per-block sums (K = slots of the launch)
    unsigned int* ticket;         // grid-completion counter, 0 between launches
    double* out;                  // [K] final sums
    unsigned int* done;           // or NULL: completion word, set to seq once out is written
    unsigned int seq;
    // in-place evaluation only: ma, and order keys of [lo, hi] per observable and of the
    // weights' range [-0, 1e300] (slot 4); see order_key in nll_device.cuh
    double ma;
    long long klo[5], khi[5];
};

// Load-time statistics: sum w, sum w (m - ma), count of events outside the ranges.
struct SArgs {
    const double* col[4];
    const double* w;
    double* dst[4];  // non-null: the kernel also stores col[d] there (a copy read in place)
    double* dst_w;   // the same for w
    int64_t n;
    int ndim;
    double lo[4], hi[4];
    double* partials;
    unsigned int* ticket;
    double* out;  // [3]
};

struct BArgs {  // basis precompute
    const double* ctl;
    const double* ctk;
    const double* phi;
    double* out[13];  // h0, hFL, h_S3..h_S9, T2l, T2k, xp, T2p
    int64_t n;
};

// Host-side parameter-only terms of one parameter point (runtime.cu): the kernel constant
// block and the derivative constants of the gradient assembly.
struct Hoist {
    KConst k;
    double mu, sigma, alpha, f, ma;
    double b0, b2, lnb1;
    double dlnN1_dmu, dlnN1_dsig, dlnN2t_dal;
    double dlnNc_dc2[3];
    double d2lnN1[3];     // d^2 ln N1 / (dmu dmu, dmu dsigma, dsigma dsigma)
    double d2lnN2t_dal2;  // d^2 ln Ntilde2 / dalpha^2 (= variance of m under exp(alpha m))
};
int hoist_core(int kind, const double* ranges, const double* th, bool grad, Hoist& H, std::string* err);
void assemble_core(int kind, const Hoist& H, double sum_wdm, const double* S, double* nll_out, double* grad_out);

// Device memory of the library's objects (models, batches, servers) is counted against a
// per-object limit read at creation from the environment variable GBNLL_DEVICE_ALLOC_LIMIT
// (bytes; unset or 0: no limit), so that running out of device memory can be provoked from
// the host in tests: an allocation past the limit fails as cudaMalloc fails
// (cudaErrorMemoryAllocation) and allocates nothing.  gb_free returns the bytes to the
// object's count.
struct DevBudget {
    size_t limit = 0;  // 0: no limit
    size_t used = 0;
};
size_t dev_budget_limit_from_env();
cudaError_t gb_malloc_bytes(DevBudget* budget, void** p, size_t bytes);
template <class T>
inline cudaError_t gb_malloc(DevBudget* budget, T** p, size_t bytes)
{
    return gb_malloc_bytes(budget, reinterpret_cast<void**>(p), bytes);
}
void gb_free(void* p);

// Launchers (kernels.cu).  They return the launch's cudaError_t.
cudaError_t launch_fused(int kind, int variant, bool weighted, bool grad, int blocks, int threads,
                         cudaStream_t stream, const KArgs& a, bool in_place = false);
cudaError_t launch_stats(int blocks, int threads, cudaStream_t stream, const SArgs& a);
cudaError_t launch_basis(int blocks, int threads, cudaStream_t stream, const BArgs& a);
// The exp and sin/cos table of kernels.cu's kernels (fill_device_tables) on the current device,
// uploaded at the first call per device.
cudaError_t ensure_device_tables();
int num_acc(int kind, bool grad);

// On-device generation (gen.cu): toy t gets counts[t] events from stream (seed, t) at
// column positions out_pos[t]...; returns an nll_status.
int gen_toys(int kind, const double* ranges, const double* theta, const int64_t* counts, int n_toys, uint64_t seed,
             const int64_t* out_pos, double* const* out, int sm_count, cudaStream_t stream);
// per-toy sum of (m - ma) over [begin, end) (device arrays), fixed order
cudaError_t toy_sums(const double* m, const int64_t* d_begin, const int64_t* d_end, double ma, int n_toys,
                     double* d_out, cudaStream_t stream);

// Analytic Hessian (hess.cu).  One kernel stages per-event columns (scores and the few
// products the second derivatives need) in shared memory and sums column products
// ("slots") over events; the host assembles NLL, gradient, Hessian and W = sum w^2 s s^T
// from the slot sums and the parameter-only terms.
constexpr int kHessThreads = 128;   // threads per block = events per shared-memory tile
constexpr int kHessMaxSlots = 384;  // at most 3 slots per thread
constexpr int kHessMaxBlocksPerSm = 4;

struct HConst {
    double mu, b0, neg_b0s, neg_als, k0s, b2, inv_sigma;  // *s: times the exponential's scale
    double dlnN1_dmu, dlnN1_dsig, mu_ma, dlnN2t_dal, inv_f, inv_1mf;
    double ang[8];
    double c1[3], c2[3], dl[3];  // Chebyshev coefficients and d ln Nc_j / d c2_j
};

struct HEv {  // the sample as the Hessian pass reads it
    const double* col[kNumCols];
    const double* w;
    int64_t n;  // events with index < n are real (global index)
};

struct HArgs {
    HEv ev;
    HConst c;
    int nslots;
    int lnp_slot;          // unweighted: slot that receives the block's sum of ln P (else -1)
    int tail_begin, tail_count;  // slots summed while staging (HessLayout)
    double* partials;      // [kHessMaxSlots][blocks], reduced by a second launch
    double* out;           // [nslots]
    unsigned int* done;    // or NULL: completion words [nslots], set to seq once out[s] is written
    unsigned int seq;
    // column pair of each slot: sij[s] and sij[kHessMaxSlots + s], a device table of the layout
    // (hess_slot_table), so that the launch parameters stay small
    const uint8_t* sij;
};


// The Hessian table's few slots past its last full warp row (tail_count <= kHessTailMax, the
// same with or without the W slots after them) are summed by the thread that stages each
// event instead of costing a whole warp row of FMAs per event.  The mass model's table (at most
// kHessOwnMax slots) is summed that way entirely: each thread accumulates its own events'
// products, all threads busy and no tile phase, where a warp row would leave most lanes idle.
constexpr int kHessTailMax = 4;
constexpr int kHessOwnMax = 32;
template <int KIND>
struct HessTailMax {
    static constexpr int value = KIND == kMass1D ? kHessOwnMax : kHessTailMax;
};
struct HessLayout {
    int nslots = 0, ncols = 0, lnp_slot = -1;
    int tail_begin = 0, tail_count = 0;
    uint8_t si[kHessMaxSlots], sj[kHessMaxSlots];
};
// Slot table for (kind, weighted, with W); returns false if it does not fit.
bool hess_layout(int kind, bool weighted, bool want_w2, HessLayout* L);
// Device copy of a layout's slot table on the current device (uploaded once per device and
// layout); *out receives its address.
cudaError_t hess_slot_table(int kind, bool weighted, bool want_w2, const HessLayout& L, const uint8_t** out);
void hess_fill_const(int kind, const Hoist& H, const double* theta, HConst* c);
// Assemble from the slot sums; returns the count of events with a non-positive density.
double hess_assemble(int kind, bool weighted, bool want_w2, const Hoist& H, double sum_wdm, const HessLayout& L,
                     const double* sums, double* nll, double* grad, double* hess, double* w2);
cudaError_t launch_hess(int kind, int variant, bool weighted, int blocks, cudaStream_t stream, const HArgs& a);
int hess_occupancy(int kind, int variant, bool weighted);  // resident blocks per SM

// Static device scratch of nll_eval_grad_4d_noalloc (kernels.cu).
constexpr int kNoAllocMaxBlocks = 1024;
struct NoAllocScratch {
    double* partials;  // [kAccModel][max_blocks]
    double* out;       // [32] final sums
    int max_blocks;
};
// Device addresses of the scratch on `device` (which must be current); set up once per device.
cudaError_t noalloc_scratch_setup(int device, NoAllocScratch* out);
// True when p is host memory that kernels on `device` read in place: pinned or registered host
// memory, or ordinary pageable memory where the device reports pageable memory access (ATS over
// NVLink-C2C).
bool host_read_in_place(int device, const void* p);
int fused_occupancy(int kind, int variant, bool weighted, bool grad, int threads,
                    bool in_place = false);  // resident blocks/SM
// Order key of a double: key(x) <= key(y) iff x <= y for non-NaN x, y (-0 < +0); NaNs fall
// outside any finite interval.  Host copy of the device function in nll_device.cuh.
inline long long order_key_host(double x)
{
    long long b;
    memcpy(&b, &x, sizeof b);
    return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}

}  // namespace gbnll
