// runtime.cu -- host side of the C ABI declared in include/gbnll.h.
//
// Per minimiser step (paper Sec. 2.1 and 2.4.1) an evaluation
//   1. validates theta and computes the parameter-only terms on the host (normalisations,
//      their logarithms and derivatives) into the per-launch constant block,
//   2. launches one fused kernel that evaluates every event, its log-density and the
//      per-event gradient sums and reduces them on the device,
//   3. copies the handful of sums back and assembles NLL and gradient on the host.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/gbnll.h"
#include "fp64_math.cuh"
#include "gbnll_internal.h"
#include "trace.h"
#include "tune_cache.h"
#include "minimise.h"

using namespace gbnll;

namespace {

const double kPi = 3.14159265358979323846;

const char* kNames1D[4] = {"mu", "sigma", "alpha", "fsig"};
const char* kNames4D[18] = {"mu",     "sigma",  "FL",     "S3",     "S4",     "S5",
                            "AFB",    "S7",     "S8",     "S9",     "alpha",  "c1_ctl",
                            "c2_ctl", "c1_ctk", "c2_ctk", "c1_phi", "c2_phi", "fsig"};

int ensure_exp2_table(int device)
{
    if (device < 0 || device >= 64) return NLL_ERR_ARG;
    return ensure_device_tables() == cudaSuccess ? NLL_OK : NLL_ERR_CUDA;  // current device
}

}  // namespace

struct nll_model {
    DevBudget budget;  // device memory of this model (limit from GBNLL_DEVICE_ALLOC_LIMIT)
    int kind = 0;
    int ndim = 0;
    int npar = 0;
    int device = 0;
    int sm_count = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    double ranges[8] = {0};

    // event store
    int64_t n = 0, n_pad = 0;
    bool loaded = false, weighted = false, has_basis = false;
    int ncols = 0;           // event columns allocated before the weights
    double* d_ev = nullptr;  // kNumCols columns of n_pad doubles (only the used ones allocated)
    double* d_w = nullptr;
    size_t ev_bytes = 0;     // bytes used by the current sample
    size_t ev_capacity = 0;  // bytes allocated at d_ev
    double sum_w = 0.0, sum_wdm = 0.0;
    // in-place sample (on_device = 2): the caller's buffers, read by every evaluation
    bool in_place = false;
    const double* ip_col[4] = {nullptr, nullptr, nullptr, nullptr};
    const double* ip_w = nullptr;

    // reduction scratch and results
    int max_blocks = 0;
    double* d_partials = nullptr;
    unsigned int* d_ticket = nullptr;
    double* d_out = nullptr;  // device alias of h_out
    double* h_out = nullptr;  // mapped pinned host memory, written by the kernels
    // completion words after the kAccModel result slots, one per slot: an evaluation launch
    // stores its sequence number in word k once slot k is written, and the host polls them
    unsigned int* h_done = nullptr;
    unsigned int* d_done = nullptr;
    unsigned int seq = 0;

    // launch shape
    int bps = 2, threads = 256, variant = 0;
    // resident blocks per SM of the fused kernel, by [variant - 1][grad][threads / 64 - 1]
    // (0: not asked yet, -1: the occupancy query gave nothing)
    int occ[2][2][4] = {};

    // profiling
    bool profiling = false;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    mutable double last_ms = -1.0;
    mutable bool ms_pending = false;  // ev0/ev1 bracket a launch whose time is not read yet

    // analytic Hessian scratch (allocated at the first nll_eval_hess)
    double* d_hpart = nullptr;          // [kHessMaxSlots][hess_max_blocks]
    double* h_hout = nullptr;           // mapped pinned [kHessMaxSlots], then kHessMaxSlots completion words
    double* d_hout = nullptr;
    unsigned int* h_hdone = nullptr;
    unsigned int* d_hdone = nullptr;
    int hess_max_blocks = 0;

    // last valid constant block (for autotuning)
    bool have_last = false;
    Hoist last;

    std::string err;
};

namespace {

int fail(nll_model* m, int status, const char* fmt, ...)
{
    if (m) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        m->err = buf;
    }
    return status;
}

int fail_text(std::string* err, int status, const char* fmt, ...)
{
    if (err) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        *err = buf;
    }
    return status;
}

int cuda_fail(nll_model* m, cudaError_t e, const char* what)
{
    return fail(m, e == cudaErrorMemoryAllocation ? NLL_ERR_OOM : NLL_ERR_CUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

const double* colptr(const nll_model* m, int c) { return m->d_ev ? m->d_ev + (size_t)c * m->n_pad : nullptr; }

// column c and the weights as the kernels read them (the event store, or the caller's buffers)
const double* evcol(const nll_model* m, int c)
{
    if (m->in_place) return c < m->ndim ? m->ip_col[c] : nullptr;
    return c < m->ncols ? colptr(m, c) : nullptr;
}
const double* evw(const nll_model* m) { return !m->weighted ? nullptr : (m->in_place ? m->ip_w : m->d_w); }

// N1 = 1/2 [erf(za) - erf(zb)] with za = (mu-ma)/(sqrt2 sigma), zb = (mu-mb)/(sqrt2 sigma)
// (paper Eq. 2); evaluated with erfc on the side where both arguments share a sign.
double gauss_norm(double za, double zb)
{
    if (zb > 0.0) return 0.5 * (erfc(zb) - erfc(za));
    if (za < 0.0) return 0.5 * (erfc(-za) - erfc(-zb));
    return 0.5 * (erf(za) - erf(zb));
}

// Parameter-only terms (paper Sec. 2.4.1).  The density is written as
//   P(x) = exp(alpha (m - ma)) * Ptilde,
//   Ptilde = A(angles) exp(-b0 d^2 - alpha d + k0) + b2 prod_j Cbar_j(x_j),
// d = m - mu, b0 = 1/(2 sigma^2), k0 = ln b1 - alpha (mu - ma),
// b1 = fsig / (sqrt(2 pi) sigma N1), b2 = (1 - fsig) / (Ntilde2 prod_j Nc_j),
// Ntilde2 = exp(-alpha ma) N2 = expm1(alpha (mb - ma)) / alpha  (mb - ma at alpha = 0),
// Cbar_j = 1 + c1_j x_j + c2_j (2 x_j^2 - 1), Nc_j = (2 - 2/3 c2_j) (times pi for phi).
}  // namespace

namespace gbnll {

namespace {
std::mutex g_alloc_mutex;
std::unordered_map<void*, std::pair<DevBudget*, size_t>>& alloc_registry()
{
    static std::unordered_map<void*, std::pair<DevBudget*, size_t>> reg;
    return reg;
}
}  // namespace

size_t dev_budget_limit_from_env()
{
    const char* v = getenv("GBNLL_DEVICE_ALLOC_LIMIT");
    if (!v || !*v) return 0;
    char* end = nullptr;
    const unsigned long long x = strtoull(v, &end, 10);
    return (end && *end == '\0') ? (size_t)x : 0;
}

cudaError_t gb_malloc_bytes(DevBudget* budget, void** p, size_t bytes)
{
    *p = nullptr;
    std::lock_guard<std::mutex> lock(g_alloc_mutex);
    if (budget && budget->limit && budget->used + bytes > budget->limit) return cudaErrorMemoryAllocation;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        return e;
    }
    alloc_registry()[*p] = {budget, bytes};
    if (budget) budget->used += bytes;
    return cudaSuccess;
}

void gb_free(void* p)
{
    if (!p) return;
    {
        std::lock_guard<std::mutex> lock(g_alloc_mutex);
        auto& reg = alloc_registry();
        auto it = reg.find(p);
        if (it != reg.end()) {
            if (it->second.first) it->second.first->used -= it->second.second;
            reg.erase(it);
        }
    }
    cudaFree(p);
}

int hoist_core(int kind, const double* ranges, const double* th, bool grad, Hoist& H, std::string* err)
{
    memset(&H, 0, sizeof H);
    const int npar = kind == kMass1D ? 4 : 18;
    for (int k = 0; k < npar; ++k)
        if (!isfinite(th[k])) return fail_text(err, NLL_ERR_ARG, "parameter %d (%s) is not finite", k,
                                           kind == kMass1D ? kNames1D[k] : kNames4D[k]);
    const double ma = ranges[0], mb = ranges[1], D = mb - ma;
    double mu = th[0], sigma = th[1];
    double alpha = kind == kMass1D ? th[2] : th[10];
    double f = kind == kMass1D ? th[3] : th[17];
    if (!(sigma > 0.0)) return fail_text(err, NLL_ERR_ARG, "sigma must be > 0 (got %g)", sigma);
    if (grad ? !(f > 0.0 && f < 1.0) : !(f >= 0.0 && f <= 1.0))
        return fail_text(err, NLL_ERR_ARG, "fsig must be in %s (got %g)", grad ? "(0, 1)" : "[0, 1]", f);
    double za = (mu - ma) / (sqrt(2.0) * sigma), zb = (mu - mb) / (sqrt(2.0) * sigma);
    double N1 = gauss_norm(za, zb);
    if (!(N1 > 1e-300)) return fail_text(err, NLL_ERR_ARG, "Gaussian normalisation underflows (mu=%g sigma=%g)", mu, sigma);
    double ea = exp(-za * za), eb = exp(-zb * zb);
    H.dlnN1_dmu = (ea - eb) / (sqrt(2.0 * kPi) * sigma * N1);
    H.dlnN1_dsig = -(za * ea - zb * eb) / (sqrt(kPi) * sigma * N1);
    double t = alpha * D;
    double Nt2;
    if (alpha == 0.0) {
        Nt2 = D;
        H.dlnN2t_dal = 0.5 * D;
    } else {
        Nt2 = expm1(t) / alpha;
        // d ln Ntilde2 / d alpha = D (1/(1 - e^-t) - 1/t)
        if (fabs(t) > 1e-3)
            H.dlnN2t_dal = D * (-1.0 / expm1(-t) - 1.0 / t);
        else
            H.dlnN2t_dal = D * (0.5 + t / 12.0 - t * t * t / 720.0 + t * t * t * t * t / 30240.0);
    }
    // second derivatives (analytic Hessian): d2 ln N1 = N1''/N1 - (N1'/N1)^2 with
    //   N1''_mumu = -(za ea - zb eb) / (sqrt(pi) sigma^2),
    //   N1''_musigma = (ea (2 za^2 - 1) - eb (2 zb^2 - 1)) / (sqrt(2 pi) sigma^2),
    //   N1''_sigmasigma = 2 (za ea (1 - za^2) - zb eb (1 - zb^2)) / (sqrt(pi) sigma^2)
    {
        const double s2 = sigma * sigma;
        H.d2lnN1[0] = -(za * ea - zb * eb) / (sqrt(kPi) * s2 * N1) - H.dlnN1_dmu * H.dlnN1_dmu;
        H.d2lnN1[1] = (ea * (2.0 * za * za - 1.0) - eb * (2.0 * zb * zb - 1.0)) / (sqrt(2.0 * kPi) * s2 * N1) -
                      H.dlnN1_dmu * H.dlnN1_dsig;
        H.d2lnN1[2] = 2.0 * (za * ea * (1.0 - za * za) - zb * eb * (1.0 - zb * zb)) / (sqrt(kPi) * s2 * N1) -
                      H.dlnN1_dsig * H.dlnN1_dsig;
    }
    // d^2 ln Ntilde2 / d alpha^2 = D^2 v(|t|), v(a) = 1/a^2 - e^-a / (1 - e^-a)^2: the variance of
    // (m - ma)/D under exp(t (m - ma)/D).  Below |t| = 1/2, its power series from the expansion
    // of coth, v = sum_n (2n-1) B_2n a^(2n-2) / (2n)!, through a^16.
    {
        const double a = fabs(t);
        double v;
        if (a < 0.5) {
            static const double c[9] = {1.0 / 12.0,
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
            for (int k = 7; k >= 0; --k) v = fma(v, a2, c[k]);
        } else {
            const double em = expm1(-a);
            v = 1.0 / (a * a) - exp(-a) / (em * em);
        }
        H.d2lnN2t_dal2 = D * D * v;
    }
    double b0 = 1.0 / (2.0 * sigma * sigma);
    double lnb1 = (f > 0.0) ? log(f) - 0.5 * log(2.0 * kPi) - log(sigma) - log(N1) : -INFINITY;
    H.lnb1 = lnb1;
    double b2 = (1.0 - f) / Nt2;
    if (kind == kKstar4D) {
        for (int j = 0; j < 3; ++j) {
            double c2 = th[12 + 2 * j];
            double nc = 2.0 - (2.0 / 3.0) * c2;
            if (!(nc > 0.0)) return fail_text(err, NLL_ERR_ARG, "Chebyshev normalisation %d is not positive", j);
            H.dlnNc_dc2[j] = (-2.0 / 3.0) / nc;
            b2 /= nc * (j == 2 ? kPi : 1.0);
        }
    }
    // exponent range of the per-event exponential: -b0 d^2 - alpha (m - ma) + ln b1 <= |alpha| D + ln b1
    if (fabs(alpha) * D + std::max(lnb1, 0.0) > 700.0)
        return fail_text(err, NLL_ERR_ARG, "parameter point outside the exponent range (|alpha|(mb-ma)=%g, ln b1=%g)",
                    fabs(alpha) * D, lnb1);
    H.mu = mu;
    H.sigma = sigma;
    H.alpha = alpha;
    H.f = f;
    H.ma = ma;
    H.b0 = b0;
    H.b2 = b2;
    KConst& k = H.k;
    const double S = kExpArgScale;  // the kernels' exponential takes its argument times S
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
    return NLL_OK;
}

}  // namespace gbnll

namespace gbnll {
bool host_read_in_place(int device, const void* p)
{
    static std::atomic<int> attr[64];  // 0: not asked, 1: no pageable access, 2: access
    if (device < 0 || device >= 64 || !p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    // pinned or registered: read in place where the device addresses it at the host pointer
    if (at.type == cudaMemoryTypeHost) return at.devicePointer == p;
    if (at.type != cudaMemoryTypeUnregistered) return false;
    int a = attr[device].load(std::memory_order_relaxed);
    if (a == 0) {
        int pageable = 0;
        if (cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, device) != cudaSuccess) {
            cudaGetLastError();
            pageable = 0;
        }
        a = pageable ? 2 : 1;
        attr[device].store(a, std::memory_order_relaxed);
    }
    return a == 2;
}
}  // namespace gbnll

namespace {

int hoist(nll_model* m, const double* th, bool grad, Hoist& H)
{
    return hoist_core(m->kind, m->ranges, th, grad, H, &m->err);
}

// Resident blocks per SM of the fused kernel that a launch at this shape would run (cached).
int fused_resident(nll_model* m, int variant, bool grad, int threads)
{
    if (variant < 1 || variant > 2 || threads < 64 || threads > 256 || threads % 64) return -1;
    int& o = m->occ[variant - 1][grad ? 1 : 0][threads / 64 - 1];
    if (o == 0) {
        const int r = fused_occupancy(m->kind, variant, m->weighted, grad, threads, m->in_place);
        o = r > 0 ? r : -1;
    }
    return o;
}

// Blocks of a fused launch: bps per SM, at most the blocks one wave holds (the kernel strides
// over the pairs, so blocks past the resident ones would only wait for a second wave), and no
// more than the pairs need.
int launch_blocks(const nll_model* m, int bps, int threads)
{
    int64_t npairs = (m->n + 1) / 2;
    int64_t need = (npairs + threads - 1) / threads;
    int64_t b = std::min<int64_t>((int64_t)m->sm_count * bps, std::max<int64_t>(need, 1));
    return (int)std::min<int64_t>(b, m->max_blocks);
}

int effective_variant(const nll_model* m)
{
    if (m->kind != kKstar4D) return kVarPrecompute;
    if (m->variant == NLL_VARIANT_DIRECT) return kVarDirect;
    if (m->variant == NLL_VARIANT_PRECOMPUTE) return m->has_basis ? kVarPrecompute : -1;
    return m->has_basis ? kVarPrecompute : kVarDirect;
}

unsigned int next_seq(nll_model* m)
{
    if (++m->seq == 0u) m->seq = 1u;  // 0 is the words' initial value
    return m->seq;
}

int run_fused(nll_model* m, const Hoist& H, bool grad, int bps, int threads, int variant, bool record)
{
    KArgs a;
    memset(&a, 0, sizeof a);
    for (int c = 0; c < kNumCols; ++c) a.col[c] = evcol(m, c);
    a.w = evw(m);
    a.n = m->n;
    a.c = H.k;
    if (m->in_place) {
        a.ma = m->ranges[0];
        for (int d = 0; d < m->ndim; ++d) {
            a.klo[d] = order_key_host(m->ranges[2 * d]);
            a.khi[d] = order_key_host(m->ranges[2 * d + 1]);
        }
        a.klo[4] = order_key_host(-0.0);
        a.khi[4] = order_key_host(1.0e300);
    }
    a.partials = m->d_partials;
    a.ticket = m->d_ticket;
    a.out = m->d_out;
    if (record) {
        a.done = m->d_done;
        a.seq = next_seq(m);
    }
    // A sample too small to give every SM a block at this block size runs in 64-thread blocks:
    // the events' FP64 work then spreads over up to four times as many SMs (an SM's FP64 pipe,
    // not the launch, bounds a small evaluation).
    if (threads > 64 && (m->n + 1) / 2 < (int64_t)m->sm_count * threads) threads = 64;
    const int resident = fused_resident(m, variant, grad, threads);
    int blocks = launch_blocks(m, resident > 0 && resident < bps ? resident : bps, threads);
    cudaError_t e;
    if (record && m->profiling) cudaEventRecord(m->ev0, m->stream);
    e = launch_fused(m->kind, variant, m->weighted, grad, blocks, threads, m->stream, a, m->in_place);
    if (e != cudaSuccess) return cuda_fail(m, e, "fused kernel launch");
    if (record && m->profiling) cudaEventRecord(m->ev1, m->stream);
    return NLL_OK;
}

}  // namespace

namespace gbnll {
// NLL and gradient from the kernel sums S (slots of gbnll_internal.h) and the constants.
void assemble_core(int kind, const Hoist& H, double sum_wdm, const double* S, double* nll_out, double* grad_out)
{
    const bool grad = grad_out != nullptr;
    const int npar = kind == kMass1D ? 4 : 18;
    // ln L = alpha sum w (m - ma) + sum w ln Ptilde
    double lnL = H.alpha * sum_wdm + S[0];
    *nll_out = -lnL;
    if (!grad) return;
    const double two_b0 = 2.0 * H.b0, dma = H.mu - H.ma;
    double dL[18] = {0};
    // mass shape: d ln s / d mu = 2 b0 d - dlnN1/dmu ; d ln s / d sigma = 2 b0 d^2 / sigma - 1/sigma - dlnN1/dsigma
    dL[0] = two_b0 * S[2] - H.dlnN1_dmu * S[1];
    dL[1] = two_b0 / H.sigma * S[3] - (1.0 / H.sigma + H.dlnN1_dsig) * S[1];
    if (kind == kMass1D) {
        double sre = H.b2 * S[4], sred = H.b2 * S[5];
        dL[2] = sred + dma * sre - H.dlnN2t_dal * sre;
        dL[3] = S[1] / H.f - sre / (1.0 - H.f);
    } else {
        for (int k = 0; k < 8; ++k) dL[2 + k] = S[4 + k];
        double sre = S[12], sred = S[13];
        dL[10] = sred + dma * sre - H.dlnN2t_dal * sre;
        dL[11] = H.b2 * S[14];
        dL[12] = H.b2 * S[15] - H.dlnNc_dc2[0] * sre;
        dL[13] = S[16];
        dL[14] = S[17] - H.dlnNc_dc2[1] * sre;
        dL[15] = S[18];
        dL[16] = S[19] - H.dlnNc_dc2[2] * sre;
        dL[17] = S[1] / H.f - sre / (1.0 - H.f);
    }
    for (int k = 0; k < npar; ++k) grad_out[k] = -dL[k];
}

}  // namespace gbnll

namespace {

// Waits for a launch numbered seq with K result slots: polls the K mapped completion words,
// which the final-sum kernels set after a system-scope fence once each slot's result is in
// host memory (this returns a few microseconds before the stream would report the launch
// complete), and asks the stream every 1024 polls whether it failed or went idle without
// setting them.
cudaError_t wait_words(cudaStream_t stream, const unsigned int* words, unsigned int seq, int K)
{
    int k = 0;
    for (unsigned int it = 1;; ++it) {
        while (k < K && __atomic_load_n(words + k, __ATOMIC_ACQUIRE) == seq) ++k;
        if (k == K) return cudaSuccess;
        if ((it & 1023u) == 0u) {
            cudaError_t q = cudaStreamQuery(stream);
            if (q == cudaErrorNotReady) continue;
            if (q != cudaSuccess) return q;
            while (k < K && __atomic_load_n(words + k, __ATOMIC_ACQUIRE) == seq) ++k;
            return k == K ? cudaSuccess : cudaErrorLaunchFailure;  // stream idle, words not set
        }
    }
}


int eval_impl(nll_model* m, const double* theta, int n_params, double* nll_out, double* grad_out)
{
    if (!m) return NLL_ERR_ARG;
    const bool grad = grad_out != nullptr;
    if (!theta || !nll_out) return fail(m, NLL_ERR_ARG, "null theta or output");
    if (n_params != m->npar) return fail(m, NLL_ERR_ARG, "expected %d parameters, got %d", m->npar, n_params);
    if (!m->loaded) return fail(m, NLL_ERR_STATE, "no events loaded");
    GBNLL_TRACE(grad ? "nll_eval_grad" : "nll_eval");
    Hoist H;
    int st;
    {
        GBNLL_TRACE("hoist");
        st = hoist(m, theta, grad, H);
    }
    if (st != NLL_OK) return st;
    m->last = H;
    m->have_last = true;
    const int KB = num_acc(m->kind, grad);
    const int K = KB + (m->in_place ? kAccInPlace : 0);
    double S[kAccModel] = {0};
    if (m->n > 0) {
        int var = effective_variant(m);
        if (var < 0) return fail(m, NLL_ERR_STATE, "precompute variant requested but no basis was built");
        if (cudaSetDevice(m->device) != cudaSuccess) return fail(m, NLL_ERR_CUDA, "cudaSetDevice failed");
        {
            GBNLL_TRACE("launch");
            st = run_fused(m, H, grad, m->bps, m->threads, var, true);
        }
        if (st != NLL_OK) return st;
        cudaError_t e;
        {
            GBNLL_TRACE("wait for the sums");
            e = wait_words(m->stream, m->h_done, m->seq, K);
        }
        if (e != cudaSuccess) return cuda_fail(m, e, "evaluation");
        if (m->profiling) {  // the kernel time is read when asked for (nll_last_kernel_ms)
            m->ms_pending = true;
            m->last_ms = -1.0;
        }
        memcpy(S, m->h_out, K * sizeof(double));
    }
    if (m->in_place) {  // the statistics a copied load computes once come with every evaluation
        if (S[KB] != 0.0) {
            *nll_out = INFINITY;
            if (grad)
                for (int k = 0; k < m->npar; ++k) grad_out[k] = NAN;
            return fail(m, NLL_ERR_ARG, "%.0f event(s) outside the observable ranges or with invalid weights", S[KB]);
        }
        m->sum_wdm = S[KB - 1];
    }
    double bad = S[K - 1];
    if (bad != 0.0 || !isfinite(S[0])) {
        *nll_out = INFINITY;
        if (grad)
            for (int k = 0; k < m->npar; ++k) grad_out[k] = NAN;
        return fail(m, NLL_ERR_NONPOSITIVE_PDF, "density not positive for %.0f thread(s) of events", bad);
    }
    assemble_core(m->kind, H, m->sum_wdm, S, nll_out, grad ? grad_out : nullptr);
    return NLL_OK;
}

int ensure_hess_scratch(nll_model* m)
{
    if (m->d_hpart) return NLL_OK;
    m->hess_max_blocks = m->sm_count * kHessMaxBlocksPerSm;
    cudaError_t e = gb_malloc(&m->budget, &m->d_hpart, sizeof(double) * kHessMaxSlots * (size_t)m->hess_max_blocks);
    if (e == cudaSuccess)
        e = cudaHostAlloc(&m->h_hout, (sizeof(double) + sizeof(unsigned int)) * kHessMaxSlots, cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer(&m->d_hout, m->h_hout, 0);
    if (e == cudaSuccess) {
        m->h_hdone = reinterpret_cast<unsigned int*>(m->h_hout + kHessMaxSlots);
        m->d_hdone = reinterpret_cast<unsigned int*>(m->d_hout + kHessMaxSlots);
        for (int k = 0; k < kHessMaxSlots; ++k) m->h_hdone[k] = 0u;
    }
    if (e != cudaSuccess) {
        if (m->d_hpart) gb_free(m->d_hpart);
        if (m->h_hout) cudaFreeHost(m->h_hout);
        m->d_hpart = m->h_hout = m->d_hout = nullptr;
        return cuda_fail(m, e, "Hessian scratch");
    }
    return NLL_OK;
}

int hess_impl(nll_model* m, const double* theta, int n_params, double* nll_out, double* grad_out, double* hess_out,
              double* w2_out)
{
    if (!m) return NLL_ERR_ARG;
    if (!theta || !nll_out || !hess_out) return fail(m, NLL_ERR_ARG, "null theta or output");
    if (n_params != m->npar) return fail(m, NLL_ERR_ARG, "expected %d parameters, got %d", m->npar, n_params);
    if (!m->loaded) return fail(m, NLL_ERR_STATE, "no events loaded");
    if (m->in_place && m->n > 0) {  // range check and sum w (m - ma) come with an evaluation
        double f, g[18];
        int st0 = eval_impl(m, theta, n_params, &f, g);
        if (st0 != NLL_OK) {
            *nll_out = f;
            return st0;
        }
    }
    GBNLL_TRACE("nll_eval_hess");
    Hoist H;
    int st;
    {
        GBNLL_TRACE("hoist");
        st = hoist(m, theta, true, H);
    }
    if (st != NLL_OK) return st;
    const bool want_w2 = w2_out != nullptr;
    HessLayout L;
    if (!hess_layout(m->kind, m->weighted, want_w2, &L)) return fail(m, NLL_ERR_ARG, "Hessian slot table overflow");
    double sums[kHessMaxSlots];
    for (int k = 0; k < kHessMaxSlots; ++k) sums[k] = 0.0;
    if (m->n > 0) {
        int var = effective_variant(m);
        if (var < 0) return fail(m, NLL_ERR_STATE, "precompute variant requested but no basis was built");
        if (cudaSetDevice(m->device) != cudaSuccess) return fail(m, NLL_ERR_CUDA, "cudaSetDevice failed");
        st = ensure_hess_scratch(m);
        if (st != NLL_OK) return st;
        static_assert(sizeof(HArgs) <= 4096, "kernel parameters");
        HArgs a;
        memset(&a, 0, sizeof a);
        for (int c = 0; c < kNumCols; ++c) a.ev.col[c] = evcol(m, c);
        a.ev.w = evw(m);
        a.ev.n = m->n;
        hess_fill_const(m->kind, H, theta, &a.c);
        a.nslots = L.nslots;
        a.lnp_slot = L.lnp_slot;
        a.tail_begin = L.tail_begin;
        a.tail_count = L.tail_count;
        a.partials = m->d_hpart;
        a.out = m->d_hout;
        a.done = m->d_hdone;
        a.seq = next_seq(m);
        cudaError_t et = hess_slot_table(m->kind, m->weighted, want_w2, L, &a.sij);
        if (et != cudaSuccess) return cuda_fail(m, et, "Hessian slot table");
        int occ = std::min(std::max(hess_occupancy(m->kind, var, m->weighted), 1), kHessMaxBlocksPerSm);
        const int64_t ntiles = (m->n + kHessThreads - 1) / kHessThreads;
        int blocks = (int)std::min<int64_t>(ntiles, (int64_t)m->sm_count * occ);
        blocks = std::min(blocks, m->hess_max_blocks);
        if (m->profiling) cudaEventRecord(m->ev0, m->stream);
        cudaError_t e;
        {
            GBNLL_TRACE("launch");
            e = launch_hess(m->kind, var, m->weighted, blocks, m->stream, a);
        }
        if (e != cudaSuccess) return cuda_fail(m, e, "Hessian kernel launch");
        if (m->profiling) cudaEventRecord(m->ev1, m->stream);
        {
            GBNLL_TRACE("wait for the sums");
            e = wait_words(m->stream, m->h_hdone, a.seq, L.nslots);
        }
        if (e != cudaSuccess) return cuda_fail(m, e, "Hessian evaluation");
        if (m->profiling) {  // the kernel time is read when asked for (nll_last_kernel_ms)
            m->ms_pending = true;
            m->last_ms = -1.0;
        }
        memcpy(sums, m->h_hout, sizeof(double) * L.nslots);
    }
    const int np = m->npar;
    double nll, grad[18], Hm[18 * 18], Wm[18 * 18];
    double bad;
    {
        GBNLL_TRACE("assemble");
        bad = hess_assemble(m->kind, m->weighted, want_w2, H, m->sum_wdm, L, sums, &nll, grad, Hm, Wm);
    }
    if (bad != bad) return fail(m, NLL_ERR_ARG, "Hessian slot table incomplete");
    if (bad != 0.0 || !isfinite(nll)) {
        *nll_out = INFINITY;
        for (int k = 0; k < np; ++k) {
            if (grad_out) grad_out[k] = NAN;
            for (int j = 0; j < np; ++j) {
                hess_out[k * np + j] = NAN;
                if (w2_out) w2_out[k * np + j] = NAN;
            }
        }
        return fail(m, NLL_ERR_NONPOSITIVE_PDF, "density not positive for %.0f event(s)", bad);
    }
    *nll_out = nll;
    if (grad_out) memcpy(grad_out, grad, sizeof(double) * np);
    memcpy(hess_out, Hm, sizeof(double) * np * np);
    if (w2_out) memcpy(w2_out, Wm, sizeof(double) * np * np);
    return NLL_OK;
}

// forget the sample; the allocation is kept for reuse unless `release`
void reset_events(nll_model* m, bool release)
{
    if (release && m->d_ev) {
        gb_free(m->d_ev);
        m->d_ev = nullptr;
        m->ev_capacity = 0;
    }
    m->d_w = nullptr;
    m->loaded = m->weighted = m->has_basis = false;
    m->in_place = false;
    memset(m->occ, 0, sizeof m->occ);  // the next load may pick other kernels (weights, in place)
    for (int d = 0; d < 4; ++d) m->ip_col[d] = nullptr;
    m->ip_w = nullptr;
    m->n = m->n_pad = 0;
    m->ncols = 0;
}

void free_events(nll_model* m) { reset_events(m, true); }

// Range check and sums of the loaded events (stats_kernel); dst/dst_w (may be null) receive
// the columns read from host memory in place.
int run_stats(nll_model* m, const double* const* cols, double* const* dst, const double* w, double* dst_w, int64_t n,
              double out[3])
{
    SArgs s;
    memset(&s, 0, sizeof s);
    for (int d = 0; d < m->ndim; ++d) {
        s.col[d] = cols[d];
        s.dst[d] = dst ? dst[d] : nullptr;
        s.lo[d] = m->ranges[2 * d];
        s.hi[d] = m->ranges[2 * d + 1];
    }
    s.w = w;
    s.dst_w = dst_w;
    s.n = n;
    s.ndim = m->ndim;
    s.partials = m->d_partials;
    s.ticket = m->d_ticket;
    s.out = m->d_out;
    int blocks = (int)std::min<int64_t>(std::max<int64_t>((n + 255) / 256, 1), (int64_t)m->sm_count * 2);
    blocks = std::min(blocks, m->max_blocks);
    cudaError_t e = launch_stats(blocks, 256, m->stream, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) return cuda_fail(m, e, "load statistics");
    memcpy(out, m->h_out, 3 * sizeof(double));
    return NLL_OK;
}

}  // namespace

// ------------------------------------------------------------------------------------
// C ABI
// ------------------------------------------------------------------------------------
extern "C" {

int nll_create_model(int kind, const double* obs_ranges, int device, uintptr_t cuda_stream, nll_model** out)
{
    if (!out) return NLL_ERR_ARG;
    *out = nullptr;
    if ((kind != NLL_MODEL_MASS1D && kind != NLL_MODEL_KSTARMUMU4D) || !obs_ranges) return NLL_ERR_ARG;
    double ma = obs_ranges[0], mb = obs_ranges[1];
    if (!(isfinite(ma) && isfinite(mb) && ma < mb)) return NLL_ERR_ARG;
    if (kind == NLL_MODEL_KSTARMUMU4D) {
        const double want[6] = {-1.0, 1.0, -1.0, 1.0, -kPi, kPi};
        for (int i = 0; i < 6; ++i)
            if (fabs(obs_ranges[2 + i] - want[i]) > 1e-12) return NLL_ERR_ARG;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return NLL_ERR_CUDA;
    if (cudaSetDevice(device) != cudaSuccess) return NLL_ERR_CUDA;
    nll_model* m = new nll_model();
    m->budget.limit = dev_budget_limit_from_env();
    m->kind = kind;
    m->ndim = kind == NLL_MODEL_MASS1D ? 1 : 4;
    m->npar = kind == NLL_MODEL_MASS1D ? 4 : 18;
    m->device = device;
    memcpy(m->ranges, obs_ranges, sizeof(double) * 2 * m->ndim);
    if (kind == NLL_MODEL_KSTARMUMU4D) {
        m->ranges[6] = -kPi;
        m->ranges[7] = kPi;
    }
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
        delete m;
        return NLL_ERR_CUDA;
    }
    m->sm_count = prop.multiProcessorCount;
    m->max_blocks = m->sm_count * 32;
    int st = ensure_exp2_table(device);
    if (st != NLL_OK) {
        delete m;
        return st;
    }
    cudaError_t e = cudaSuccess;
    m->stream = (cudaStream_t)cuda_stream;  // 0: CUDA's default stream
    m->own_stream = false;
    if (e == cudaSuccess) e = gb_malloc(&m->budget, &m->d_partials, sizeof(double) * kAccModel * m->max_blocks);
    if (e == cudaSuccess) e = gb_malloc(&m->budget, &m->d_ticket, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemset(m->d_ticket, 0, sizeof(unsigned int));
    // results land in mapped pinned host memory: the grid's last block writes them there
    if (e == cudaSuccess)
        e = cudaHostAlloc(&m->h_out, sizeof(double) * kAccModel + sizeof(unsigned int) * kAccModel, cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer(&m->d_out, m->h_out, 0);
    if (e == cudaSuccess) {
        m->h_done = reinterpret_cast<unsigned int*>(m->h_out + kAccModel);
        m->d_done = reinterpret_cast<unsigned int*>(m->d_out + kAccModel);
        for (int k = 0; k < kAccModel; ++k) m->h_done[k] = 0u;
    }
    if (e == cudaSuccess) e = cudaEventCreate(&m->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&m->ev1);
    if (e != cudaSuccess) {
        int code = e == cudaErrorMemoryAllocation ? NLL_ERR_OOM : NLL_ERR_CUDA;
        nll_destroy(m);
        return code;
    }
    *out = m;
    return NLL_OK;
}

void nll_destroy(nll_model* m)
{
    if (!m) return;
    cudaSetDevice(m->device);
    if (m->stream) cudaStreamSynchronize(m->stream);
    free_events(m);
    if (m->d_partials) gb_free(m->d_partials);
    if (m->d_ticket) gb_free(m->d_ticket);
    if (m->h_out) cudaFreeHost(m->h_out);  // d_out is its device alias
    if (m->d_hpart) gb_free(m->d_hpart);
    if (m->h_hout) cudaFreeHost(m->h_hout);
    if (m->ev0) cudaEventDestroy(m->ev0);
    if (m->ev1) cudaEventDestroy(m->ev1);
    if (m->own_stream && m->stream) cudaStreamDestroy(m->stream);
    delete m;
}

}  // extern "C"

namespace {
// In-place sample: check that the device can read every buffer (device memory of this
// device, pinned or registered host memory, or any host memory where the device reads
// pageable memory) and that the 128-bit loads are aligned; store nothing.
int check_readable(nll_model* m, const double* p, const char* what)
{
    if (((uintptr_t)p & 15u) != 0) return fail(m, NLL_ERR_ARG, "%s is not 16-byte aligned", what);
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(m, NLL_ERR_ARG, "%s: pointer attributes unavailable", what);
    }
    if (at.type == cudaMemoryTypeDevice && at.device == m->device) return NLL_OK;
    if (at.type == cudaMemoryTypeManaged || at.type == cudaMemoryTypeHost) return NLL_OK;
    int pageable = 0;
    cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, m->device);
    if (at.type == cudaMemoryTypeUnregistered && pageable) return NLL_OK;
    return fail(m, NLL_ERR_ARG, "%s is not memory the device can read in place", what);
}

int load_in_place(nll_model* m, const double* const* columns, const double* weights, int64_t n_events)
{
    if (n_events > 0) {
        static const char* names[4] = {"column 0", "column 1", "column 2", "column 3"};
        for (int d = 0; d < m->ndim; ++d) {
            int st = check_readable(m, columns[d], names[d]);
            if (st != NLL_OK) return st;
        }
        if (weights) {
            int st = check_readable(m, weights, "weights");
            if (st != NLL_OK) return st;
        }
        for (int d = 0; d < m->ndim; ++d) m->ip_col[d] = columns[d];
        m->ip_w = weights;
    }
    m->in_place = true;
    m->n = n_events;
    m->n_pad = n_events;
    m->ncols = m->ndim;
    m->weighted = weights != nullptr;
    m->sum_w = m->sum_wdm = 0.0;  // sum w (m - ma) comes with every evaluation
    m->has_basis = false;
    m->loaded = true;
    m->err.clear();
    return NLL_OK;
}
}  // namespace

extern "C" {

int nll_load_events(nll_model* m, const double* const* columns, const double* weights, int64_t n_events,
                    int on_device, int precompute)
{
    if (!m) return NLL_ERR_ARG;
    if (n_events < 0 || (n_events > 0 && !columns)) return fail(m, NLL_ERR_ARG, "bad event count or columns");
    for (int d = 0; d < m->ndim && n_events > 0; ++d)
        if (!columns[d]) return fail(m, NLL_ERR_ARG, "column %d is NULL", d);
    if (on_device < 0 || on_device > 2) return fail(m, NLL_ERR_ARG, "on_device must be 0, 1 or 2");
    if (cudaSetDevice(m->device) != cudaSuccess) return fail(m, NLL_ERR_CUDA, "cudaSetDevice failed");
    if (on_device == 2) {
        // nothing of the model's is written, and every evaluation has finished when it
        // returned, so no wait for the stream: the caller's earlier work keeps running
        reset_events(m, false);
        return load_in_place(m, columns, weights, n_events);
    }
    cudaStreamSynchronize(m->stream);  // an evaluation may not run on the store being replaced
    reset_events(m, false);
    const bool basis = (m->kind == kKstar4D) && precompute;
    const int64_t n_pad = std::max<int64_t>((n_events + 63) / 64 * 64, 64);
    // columns: mass model m [+ w]; 4D: m, ctl, ctk, phi [+ basis 13] [+ w]
    int ncols = m->kind == kMass1D ? 1 : (basis ? kNumCols : 4);
    int nalloc = ncols + (weights ? 1 : 0);
    size_t bytes = sizeof(double) * (size_t)n_pad * nalloc;
    cudaError_t e = cudaSuccess;
    if (bytes > m->ev_capacity) {
        reset_events(m, true);
        e = gb_malloc(&m->budget, &m->d_ev, bytes);
        if (e != cudaSuccess) {
            m->d_ev = nullptr;
            return cuda_fail(m, e, "event store allocation");
        }
        m->ev_capacity = bytes;
    }
    m->ev_bytes = bytes;
    m->n_pad = n_pad;
    m->ncols = ncols;
    if (n_events < n_pad) {  // zero the padding tail of every column
        for (int c = 0; c < nalloc && e == cudaSuccess; ++c)
            e = cudaMemsetAsync(m->d_ev + (size_t)c * n_pad + n_events, 0,
                                sizeof(double) * (size_t)(n_pad - n_events), m->stream);
    }
    // Host columns the device reads in place (pinned memory, or pageable memory with ATS) are
    // stored by the statistics kernel as it reads them -- one pass over NVLink-C2C, measured
    // faster than the copy engines for pinned columns; the rest by cudaMemcpyAsync.
    cudaMemcpyKind kindc = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const double* src[4] = {nullptr, nullptr, nullptr, nullptr};
    double* dst[4] = {nullptr, nullptr, nullptr, nullptr};
    const double* src_w = nullptr;
    double* dst_w = nullptr;
    for (int d = 0; d < m->ndim && e == cudaSuccess && n_events > 0; ++d) {
        double* to = m->d_ev + (size_t)d * n_pad;
        if (!on_device && host_read_in_place(m->device, columns[d])) {
            src[d] = columns[d];
            dst[d] = to;
        } else {
            src[d] = to;
            e = cudaMemcpyAsync(to, columns[d], sizeof(double) * n_events, kindc, m->stream);
        }
    }
    if (weights) {
        m->d_w = m->d_ev + (size_t)ncols * n_pad;
        src_w = m->d_w;
        if (e == cudaSuccess && n_events > 0) {
            if (!on_device && host_read_in_place(m->device, weights)) {
                src_w = weights;
                dst_w = m->d_w;
            } else {
                e = cudaMemcpyAsync(m->d_w, weights, sizeof(double) * n_events, kindc, m->stream);
            }
        }
    }
    if (e != cudaSuccess) {
        free_events(m);
        return cuda_fail(m, e, "event copy");
    }
    m->n = n_events;
    m->weighted = weights != nullptr;
    double stats[3] = {0.0, 0.0, 0.0};
    if (n_events > 0) {
        int st = run_stats(m, src, dst, src_w, dst_w, n_events, stats);
        if (st != NLL_OK) {
            free_events(m);
            return st;
        }
        if (stats[2] != 0.0) {
            free_events(m);
            return fail(m, NLL_ERR_ARG, "%.0f event(s) outside the observable ranges or with invalid weights",
                        stats[2]);
        }
    }
    m->sum_w = stats[0];
    m->sum_wdm = stats[1];
    if (basis && n_events > 0) {
        BArgs b;
        b.ctl = colptr(m, kColCtl);
        b.ctk = colptr(m, kColCtk);
        b.phi = colptr(m, kColPhi);
        for (int j = 0; j < 13; ++j) b.out[j] = m->d_ev + (size_t)(kColH0 + j) * n_pad;
        b.n = n_events;
        int blocks = (int)std::min<int64_t>((n_events + 255) / 256, (int64_t)m->sm_count * 8);
        e = launch_basis(std::max(blocks, 1), 256, m->stream, b);
        if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
        if (e != cudaSuccess) {
            free_events(m);
            return cuda_fail(m, e, "basis precompute");
        }
    }
    m->has_basis = basis;
    m->loaded = true;
    m->err.clear();
    return NLL_OK;
}

int nll_eval(nll_model* m, const double* theta, int n_params, double* nll_out)
{
    return eval_impl(m, theta, n_params, nll_out, nullptr);
}

int nll_eval_grad(nll_model* m, const double* theta, int n_params, double* nll_out, double* grad_out)
{
    if (m && !grad_out) return fail(m, NLL_ERR_ARG, "null gradient output");
    return eval_impl(m, theta, n_params, nll_out, grad_out);
}

int fit_minimise(nll_model* m, const double* theta0, const double* lo, const double* hi, const double* step,
                 const int* fixed, int n_params, const fit_options* opt, fit_result* out)
{
    if (!m || !out) return NLL_ERR_ARG;
    if (n_params != m->npar) return fail(m, NLL_ERR_ARG, "expected %d parameters", m->npar);
    Objective obj = [m, n_params](const double* th, double* f, double* g) {
        return nll_eval_grad(m, th, n_params, f, g);
    };
    HessianFn hs = [m, n_params](const double* th, double* f, double* g, double* H, double* W) {
        return nll_eval_hess(m, th, n_params, f, g, H, W);
    };
    return bfgs_minimise(obj, n_params, theta0, lo, hi, step, fixed, opt, out, &hs);
}

int nll_eval_hess(nll_model* m, const double* theta, int n_params, double* nll_out, double* grad_out,
                  double* hess_out, double* w2_out)
{
    return hess_impl(m, theta, n_params, nll_out, grad_out, hess_out, w2_out);
}

int nll_hess_num_slots(int kind, int weighted, int want_w2)
{
    if (kind != NLL_MODEL_MASS1D && kind != NLL_MODEL_KSTARMUMU4D) return -1;
    HessLayout L;
    return hess_layout(kind, weighted != 0, want_w2 != 0, &L) ? L.nslots : -1;
}

int nll_num_params(const nll_model* m) { return m ? m->npar : -1; }

const char* nll_param_name(const nll_model* m, int i)
{
    if (!m || i < 0 || i >= m->npar) return "";
    return m->kind == kMass1D ? kNames1D[i] : kNames4D[i];
}

const char* nll_last_error(const nll_model* m) { return m ? m->err.c_str() : "null model"; }

int nll_set_launch(nll_model* m, int blocks_per_sm, int threads_per_block, int variant)
{
    if (!m) return NLL_ERR_ARG;
    if (blocks_per_sm < 0 || blocks_per_sm > 32) return fail(m, NLL_ERR_ARG, "blocks_per_sm out of range");
    if (threads_per_block != 0 &&
        (threads_per_block < 64 || threads_per_block > 256 || (threads_per_block % 64) != 0))
        return fail(m, NLL_ERR_ARG, "threads_per_block must be 64, 128, 192 or 256");
    if (variant < 0 || variant > 2) return fail(m, NLL_ERR_ARG, "unknown variant");
    if (blocks_per_sm) m->bps = blocks_per_sm;
    if (threads_per_block) m->threads = threads_per_block;
    if (variant) m->variant = variant;
    return NLL_OK;
}

int nll_get_launch(const nll_model* m, int* blocks_per_sm, int* threads_per_block, int* variant, int* sm_count)
{
    if (!m) return NLL_ERR_ARG;
    if (blocks_per_sm) *blocks_per_sm = m->bps;
    if (threads_per_block) *threads_per_block = m->threads;
    if (variant) *variant = effective_variant(m);
    if (sm_count) *sm_count = m->sm_count;
    return NLL_OK;
}

int nll_autotune(nll_model* m)
{
    if (!m) return NLL_ERR_ARG;
    if (!m->loaded || !m->have_last || m->n == 0)
        return fail(m, NLL_ERR_STATE, "autotune needs loaded events and one prior evaluation");
    if (cudaSetDevice(m->device) != cudaSuccess) return fail(m, NLL_ERR_CUDA, "cudaSetDevice failed");
    m->ms_pending = false;  // the sweep below re-records ev0/ev1
    m->last_ms = -1.0;
    // candidate shapes: for each block size, one wave of resident blocks and one block fewer per
    // SM (launches never exceed one wave)
    std::vector<std::pair<int, int>> shapes;
    bool grad_ok = m->last.f > 0.0 && m->last.f < 1.0;
    for (int thr : {64, 128, 192, 256}) {
        int occ = fused_occupancy(m->kind, effective_variant(m) < 0 ? kVarDirect : effective_variant(m), m->weighted,
                                  grad_ok, thr, m->in_place);
        if (occ <= 0) continue;
        shapes.push_back({std::min(occ, 32), thr});
        if (occ > 1) shapes.push_back({std::min(occ - 1, 32), thr});
    }
    std::vector<int> variants;
    if (m->kind == kKstar4D && m->has_basis && m->variant == NLL_VARIANT_AUTO) {
        variants.push_back(kVarPrecompute);
        variants.push_back(kVarDirect);
    } else {
        variants.push_back(effective_variant(m));
    }
    bool grad = grad_ok;
    // a result kept from an earlier process for the same device and workload (GBNLL_TUNE_CACHE)
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, m->device) != cudaSuccess) return fail(m, NLL_ERR_CUDA, "device properties");
    int size_class = 0;
    while ((int64_t(1) << (size_class + 1)) <= m->n) ++size_class;
    const std::string key = tune_cache_key(prop.name, m->sm_count, "fused", m->kind,
                                           variants.size() > 1 ? -1 : variants[0],
                                           (m->weighted ? 1 : 0) + (grad ? 2 : 0) + (m->in_place ? 4 : 0), size_class);
    int kept[3];
    if (tune_cache_lookup(key, kept)) {
        bool valid = kept[0] >= 1 && kept[0] <= 32 && kept[1] >= 64 && kept[1] <= 1024 && kept[1] % 64 == 0;
        bool var_ok = false;
        for (int v : variants) var_ok = var_ok || v == kept[2];
        if (valid && var_ok) {
            m->bps = kept[0];
            m->threads = kept[1];
            if (variants.size() > 1) m->variant = kept[2] == kVarDirect ? NLL_VARIANT_DIRECT : NLL_VARIANT_PRECOMPUTE;
            return NLL_OK;
        }
    }
    float best = 1e30f;
    int best_bps = m->bps, best_thr = m->threads, best_var = variants[0];
    for (int var : variants)
        for (auto& sh : shapes) {
            float tot = 0.f;
            for (int rep = 0; rep < 4; ++rep) {
                cudaEventRecord(m->ev0, m->stream);
                int st = run_fused(m, m->last, grad, sh.first, sh.second, var, false);
                if (st != NLL_OK) return st;
                cudaEventRecord(m->ev1, m->stream);
                cudaError_t e = cudaEventSynchronize(m->ev1);
                if (e != cudaSuccess) return cuda_fail(m, e, "autotune");
                float ms;
                cudaEventElapsedTime(&ms, m->ev0, m->ev1);
                if (rep > 0) tot += ms;  // first launch of a shape is a warm-up
            }
            if (tot < best) {
                best = tot;
                best_bps = sh.first;
                best_thr = sh.second;
                best_var = var;
            }
        }
    m->bps = best_bps;
    m->threads = best_thr;
    if (variants.size() > 1) m->variant = best_var == kVarDirect ? NLL_VARIANT_DIRECT : NLL_VARIANT_PRECOMPUTE;
    const int result[3] = {best_bps, best_thr, best_var};
    tune_cache_store(key, result);
    return NLL_OK;
}

int nll_set_profiling(nll_model* m, int on)
{
    if (!m) return NLL_ERR_ARG;
    m->profiling = on != 0;
    m->last_ms = -1.0;
    m->ms_pending = false;
    return NLL_OK;
}

int nll_last_kernel_ms(const nll_model* m, double* ms)
{
    if (!m || !ms) return NLL_ERR_ARG;
    if (m->ms_pending) {
        m->ms_pending = false;
        float t = 0.f;
        if (cudaEventSynchronize(m->ev1) == cudaSuccess && cudaEventElapsedTime(&t, m->ev0, m->ev1) == cudaSuccess)
            m->last_ms = t;
    }
    if (m->last_ms < 0.0) return NLL_ERR_STATE;
    *ms = m->last_ms;
    return NLL_OK;
}

int nll_precomputed_basis(nll_model* m, double* out)
{
    if (!m || !out) return NLL_ERR_ARG;
    if (!m->has_basis) return fail(m, NLL_ERR_STATE, "no precomputed basis");
    if (cudaSetDevice(m->device) != cudaSuccess) return fail(m, NLL_ERR_CUDA, "cudaSetDevice failed");
    std::vector<double> col((size_t)m->n);
    for (int j = 0; j < 13; ++j) {
        cudaError_t e = cudaMemcpyAsync(col.data(), colptr(m, kColH0 + j), sizeof(double) * m->n,
                                        cudaMemcpyDeviceToHost, m->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
        if (e != cudaSuccess) return cuda_fail(m, e, "basis copy");
        for (int64_t i = 0; i < m->n; ++i) out[i * 13 + j] = col[i];
    }
    return NLL_OK;
}

// ------------------------------------------------------------------------------------
// No-allocation evaluation for callers that cannot call cudaMalloc.  The paper has no
// counterpart.  One launch of the fused kernel's in-place 4D instance (direct angular
// variant, tail-safe loads, range check and sum w (m - ma) in the same pass) and its final
// sums; the block partials and the sums live in a static device array (kernels.cu), and the
// sample stays in the caller's device buffers.
// ------------------------------------------------------------------------------------
int nll_eval_grad_4d_noalloc(const double* obs_ranges, const double* const* dev_columns, const double* dev_weights,
                             int64_t n_events, const double* theta, int n_params, int blocks, uintptr_t cuda_stream,
                             double* nll_out, double* grad_out)
{
    if (!obs_ranges || !theta || !nll_out || !grad_out || n_events < 0 || n_params != 18) return NLL_ERR_ARG;
    if (blocks < 0 || blocks > kNoAllocMaxBlocks) return NLL_ERR_ARG;  // beyond the static scratch
    if (!(isfinite(obs_ranges[0]) && isfinite(obs_ranges[1]) && obs_ranges[0] < obs_ranges[1])) return NLL_ERR_ARG;
    const double want[6] = {-1.0, 1.0, -1.0, 1.0, -kPi, kPi};
    for (int i = 0; i < 6; ++i)
        if (fabs(obs_ranges[2 + i] - want[i]) > 1e-12) return NLL_ERR_ARG;
    if (n_events > 0) {
        if (!dev_columns) return NLL_ERR_ARG;
        for (int d = 0; d < 4; ++d)
            if (!dev_columns[d] || ((uintptr_t)dev_columns[d] & 15)) return NLL_ERR_ARG;
        if (dev_weights && ((uintptr_t)dev_weights & 15)) return NLL_ERR_ARG;
    }
    int device = 0, sms = 0;
    if (cudaGetDevice(&device) != cudaSuccess) return NLL_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return NLL_ERR_CUDA;
    int st = ensure_exp2_table(device);
    if (st != NLL_OK) return st;
    NoAllocScratch sc;
    if (noalloc_scratch_setup(device, &sc) != cudaSuccess) return NLL_ERR_CUDA;

    nll_model m;  // parameter layout and ranges for the hoisting; owns nothing
    m.kind = kKstar4D;
    m.ndim = 4;
    m.npar = 18;
    m.device = device;
    for (int i = 0; i < 8; ++i) m.ranges[i] = obs_ranges[i];
    m.ranges[6] = -kPi;
    m.ranges[7] = kPi;
    Hoist H;
    st = hoist(&m, theta, true, H);
    if (st != NLL_OK) return st;
    if (n_events == 0) {
        *nll_out = 0.0;
        for (int k = 0; k < 18; ++k) grad_out[k] = 0.0;
        return NLL_OK;
    }
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    const int64_t npairs = (n_events + 1) / 2;

    KArgs a;
    memset(&a, 0, sizeof a);
    for (int d = 0; d < 4; ++d) a.col[d] = dev_columns[d];
    a.w = dev_weights;
    a.n = n_events;
    a.c = H.k;
    a.ma = m.ranges[0];
    for (int d = 0; d < 4; ++d) {
        a.klo[d] = order_key_host(m.ranges[2 * d]);
        a.khi[d] = order_key_host(m.ranges[2 * d + 1]);
    }
    a.klo[4] = order_key_host(-0.0);
    a.khi[4] = order_key_host(1.0e300);
    a.partials = sc.partials;
    a.out = sc.out;  // no completion words: the call synchronises the stream
    const int threads = 128;
    int nb = blocks ? blocks
                    : (int)std::min<int64_t>((int64_t)sms * 2, std::max<int64_t>((npairs + threads - 1) / threads, 1));
    constexpr int KB = kAcc4D, K = kAcc4D + kAccInPlace;
    double S[K];
    cudaError_t e = launch_fused(kKstar4D, kVarDirect, dev_weights != nullptr, true, nb, threads, stream, a, true);
    if (e == cudaSuccess) e = cudaMemcpyAsync(S, sc.out, sizeof S, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return NLL_ERR_CUDA;

    // slot KB counts events outside the ranges (or with invalid weights), slot KB - 1 holds
    // sum w (m - ma), the last slot the invalid densities; assembly as for a 4D model
    if (S[KB] != 0.0) {
        *nll_out = INFINITY;
        for (int k = 0; k < 18; ++k) grad_out[k] = NAN;
        return NLL_ERR_ARG;
    }
    if (S[K - 1] != 0.0 || !isfinite(S[0])) {
        *nll_out = INFINITY;
        for (int k = 0; k < 18; ++k) grad_out[k] = NAN;
        return NLL_ERR_NONPOSITIVE_PDF;
    }
    assemble_core(kKstar4D, H, S[KB - 1], S, nll_out, grad_out);
    return NLL_OK;
}

}  // extern "C"
