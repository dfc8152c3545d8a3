// gen.cu -- on-device generation of pseudo-experiments (paper Sec. 2.5).
//
// The paper generates toys by accept-reject on the accelerator, with every parameter fixed
// during generation so that parameter-only terms fold into constants (Sec. 2.5), and seeds
// one generator per work item.  Here every event is produced by one thread from a
// counter-based SplitMix64 stream (Steele, Lea & Flood, OOPSLA 2014): draw j of try k of
// event i of a toy is mix(state0 + (i 2^17 + 8 k + j + 1) * gamma), where state0 is the toy's
// stream state.  An event never depends on how many events or threads there are, so the
// output is deterministic and needs no scan: event i lands at position i of its toy.
//   * component: signal with probability fsig (draw 0 of try 0);
//   * signal mass: Box-Muller normal, retried while outside the window;
//   * background mass: inverse of the truncated exponential's distribution function;
//   * signal angles (4D): uniform in the box, accepted with probability A / Amax, Amax the
//     paper's accept-reject bound 9/(32 pi) (4 + sum|S_i| + 4/3 |AFB|) (appendix, get_max);
//     terms whose coefficients are zero are folded away (no phi, no sin theta needed);
//   * background angles (4D): uniform, accepted with probability prod C_j / prod max C_j.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "../../include/gbnll.h"
#include "fp64_math.cuh"
#include "gbnll_internal.h"

namespace gbnll {
namespace {

// exp, log and sin/cos tables (fill_device_tables), uploaded once per device; the generation
// kernel reads the logarithm's part through the read-only cache
__device__ double g_gtab[kTabDoubles];
std::mutex g_gtab_mutex;
bool g_gtab_ready[64];

cudaError_t ensure_gen_tables()
{
    int device = 0;
    cudaError_t e = cudaGetDevice(&device);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_gtab_mutex);
    if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
    if (g_gtab_ready[device]) return cudaSuccess;
    static double tab[kTabDoubles];
    fill_device_tables(tab);
    e = cudaMemcpyToSymbol(g_gtab, tab, kTabDoubles * sizeof(double));
    if (e == cudaSuccess) g_gtab_ready[device] = true;
    return e;
}

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;
constexpr int kMaxTries = 4096;  // per event and stage; P(no acceptance) < 1e-180 at 10 %
const double kPiG = 3.14159265358979323846;

__host__ __device__ __forceinline__ uint64_t sm64_mix(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// stream state of (seed, stream), as the host generator derives it
__host__ __device__ __forceinline__ uint64_t stream_state(uint64_t seed, uint64_t stream)
{
    return sm64_mix(seed ^ sm64_mix(stream * kGamma + 1));
}

// double in (0, 1) from 64 random bits: ((x >> 11) + 1/2) 2^-53, as one conversion and one
// fma (the fma rounds k 2^-53 + 2^-54 once, which is (k + 1/2) rounded, then scaled exactly)
__device__ __forceinline__ double u01(uint64_t x) { return fma((double)(x >> 11), 0x1p-53, 0x1p-54); }

struct GenConst {
    int kind;
    double ma, mb, mu, sigma, alpha, em1;  // em1 = expm1(alpha (mb - ma))
    double inv_alpha;                      // 1 / alpha (0 when alpha is 0)
    int bg_log1p;                          // |em1| < 1/16: background mass from log1p (see gen_kernel)
    double fsig;
    double ang[8];                         // FL, S3, S4, S5, AFB, S7, S8, S9
    double amax;                           // accept-reject bound of the angular rate
    int fold_phi, fold_sin;                // phi-dependent / sin(theta)-odd terms all zero
    double cheb[6], cmax;
};

struct GenArgs {
    GenConst g;
    const int64_t* toy_first;  // [n_toys + 1] first output event of each toy (output positions)
    const int64_t* toy_count;  // [n_toys] events per toy
    const uint64_t* toy_state; // [n_toys] stream states
    int n_toys;
    int64_t total;             // sum of counts
    const int64_t* out_pos;    // [n_toys] position of each toy's event 0 in the columns
    double* out[4];
    int* fail;                 // set when an event ran out of tries
};

// angular rate of paper Eq. 3 with the generation-time folding of zero coefficients
__device__ double angular_rate(const GenConst& g, double ctl, double ctk, double phi)
{
    const double c = 9.0 / (32.0 * kPiG);
    double cl2 = ctl * ctl, ck2 = ctk * ctk, sl2 = 1.0 - cl2, sk2 = 1.0 - ck2;
    double cos2l = 2.0 * cl2 - 1.0;
    double FL = g.ang[0];
    double r = (1.0 - FL) * 0.75 * sk2 + FL * ck2 + (1.0 - FL) * 0.25 * sk2 * cos2l - FL * ck2 * cos2l +
               g.ang[4] * (4.0 / 3.0) * sk2 * ctl;
    if (!g.fold_phi) {
        double sp, cp;
        sincospi(phi * (1.0 / kPiG), &sp, &cp);
        double c2p = 2.0 * cp * cp - 1.0, s2p = 2.0 * sp * cp;
        r += g.ang[1] * sk2 * sl2 * c2p + g.ang[7] * sk2 * sl2 * s2p;
        if (!g.fold_sin) {
            double sl = sqrt(sl2), sk = sqrt(sk2);
            double s2k = 2.0 * sk * ctk, s2l = 2.0 * sl * ctl;
            r += g.ang[2] * s2k * s2l * cp + g.ang[3] * s2k * sl * cp + g.ang[5] * s2k * sl * sp +
                 g.ang[6] * s2k * s2l * sp;
        }
    }
    return c * r;
}

__global__ void __launch_bounds__(256) gen_kernel(GenArgs a)
{
    const GenConst& g = a.g;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < a.total; e += stride) {
        // toy of output event e (binary search over the first-event offsets)
        int lo = 0, hi = a.n_toys;
        while (hi - lo > 1) {
            int mid = (lo + hi) >> 1;
            if (a.toy_first[mid] <= e) lo = mid; else hi = mid;
        }
        const int t = lo;
        const int64_t i = e - a.toy_first[t];
        const uint64_t base = a.toy_state[t] + ((uint64_t)i << 17) * kGamma;
        auto draw = [&](int k, int j) { return u01(sm64_mix(base + (uint64_t)(8 * k + j + 1) * kGamma)); };
        const bool sig = draw(0, 0) < g.fsig;
        const double D = g.mb - g.ma;
        double m = g.ma, ctl = 0.0, ctk = 0.0, phi = 0.0;
        bool ok = false;
        int k = 1;
        // Draw (1, 0) is the Box-Muller radius draw of the first signal try and the
        // inverse-distribution draw of a background mass: one logarithm, taken by the whole
        // warp, serves both (log(1 + u em1) for the background: 1 + u em1 lies in
        // [exp(alpha (mb - ma)), 1] and is formed with one rounding, which costs no accuracy
        // that matters unless |em1| is small; then log1p takes the background, a branch that
        // is uniform because em1 is a constant of the launch).  The logarithm is the
        // table-driven one of fp64_math.cuh: its arguments here are at least 2^-53 (u draws
        // lie in [2^-53, 1 - 2^-53] and em1 > -1), so always positive normals.
        const double u1 = draw(1, 0);
        const double lg1 = g.bg_log1p ? (sig ? flog(u1, g_gtab) : log1p(u1 * g.em1))
                                      : flog(sig ? u1 : fma(u1, g.em1, 1.0), g_gtab);
        if (sig) {
            double lg = lg1;
            for (; k < kMaxTries; ++k) {  // Box-Muller, truncated to the window
                if (k > 1) lg = flog(draw(k, 0), g_gtab);
                double z = sqrt(-2.0 * lg) * cospi(2.0 * draw(k, 1));
                m = g.mu + g.sigma * z;
                if (m >= g.ma && m <= g.mb) {
                    ok = true;
                    break;
                }
            }
            if (g.kind == kKstar4D && ok) {
                ok = false;
                for (++k; k < 2 * kMaxTries; ++k) {
                    ctl = 2.0 * draw(k, 0) - 1.0;
                    ctk = 2.0 * draw(k, 1) - 1.0;
                    phi = kPiG * (2.0 * draw(k, 2) - 1.0);
                    if (draw(k, 3) * g.amax < angular_rate(g, ctl, ctk, phi)) {
                        ok = true;
                        break;
                    }
                }
            }
        } else {
            m = g.alpha == 0.0 ? fma(u1, D, g.ma) : fma(lg1, g.inv_alpha, g.ma);
            m = fmin(fmax(m, g.ma), g.mb);
            ok = true;
            if (g.kind == kKstar4D) {
                ok = false;
                for (k = 2; k < kMaxTries; ++k) {
                    double x[3], prod = 1.0;
                    for (int j = 0; j < 3; ++j) {
                        x[j] = 2.0 * draw(k, j) - 1.0;
                        prod *= 1.0 + g.cheb[2 * j] * x[j] + g.cheb[2 * j + 1] * (2.0 * x[j] * x[j] - 1.0);
                    }
                    if (draw(k, 3) * g.cmax < prod) {
                        ctl = x[0];
                        ctk = x[1];
                        phi = kPiG * x[2];
                        ok = true;
                        break;
                    }
                }
            }
        }
        if (!ok) atomicOr(a.fail, 1);
        const int64_t pos = a.out_pos[t] + i;
        a.out[0][pos] = m;
        if (g.kind == kKstar4D) {
            a.out[1][pos] = ctl;
            a.out[2][pos] = ctk;
            a.out[3][pos] = phi;
        }
    }
}

__global__ void uniforms_kernel(uint64_t state, int64_t n, double* out)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        out[k] = u01(sm64_mix(state + (uint64_t)(k + 1) * kGamma));
}

}  // namespace

// folded generation constants; false if theta is not a valid generation point
static bool gen_setup(int kind, const double* ranges, const double* th, GenConst& g)
{
    memset(&g, 0, sizeof g);
    g.kind = kind;
    g.ma = ranges[0];
    g.mb = ranges[1];
    const int np = kind == kMass1D ? 4 : 18;
    for (int k = 0; k < np; ++k)
        if (!std::isfinite(th[k])) return false;
    g.mu = th[0];
    g.sigma = th[1];
    g.alpha = kind == kMass1D ? th[2] : th[10];
    g.fsig = kind == kMass1D ? th[3] : th[17];
    if (!(g.sigma > 0.0) || !(g.fsig >= 0.0 && g.fsig <= 1.0)) return false;
    g.em1 = expm1(g.alpha * (g.mb - g.ma));
    g.inv_alpha = g.alpha == 0.0 ? 0.0 : 1.0 / g.alpha;
    g.bg_log1p = fabs(g.em1) < 0.0625 ? 1 : 0;
    if (kind == kKstar4D) {
        double sum = 0.0;
        for (int j = 0; j < 8; ++j) g.ang[j] = th[2 + j];
        for (int j = 1; j < 8; ++j) sum += (j == 4 ? 4.0 / 3.0 : 1.0) * fabs(g.ang[j]);
        g.amax = 9.0 / (32.0 * kPiG) * (4.0 + sum);
        g.fold_phi = g.ang[1] == 0.0 && g.ang[2] == 0.0 && g.ang[3] == 0.0 && g.ang[5] == 0.0 && g.ang[6] == 0.0 &&
                     g.ang[7] == 0.0;
        g.fold_sin = g.ang[2] == 0.0 && g.ang[3] == 0.0 && g.ang[5] == 0.0 && g.ang[6] == 0.0;
        g.cmax = 1.0;
        for (int j = 0; j < 6; ++j) g.cheb[j] = th[11 + j];
        for (int j = 0; j < 3; ++j) {
            double c1 = g.cheb[2 * j], c2 = g.cheb[2 * j + 1];
            if (!(2.0 - (2.0 / 3.0) * c2 > 0.0)) return false;
            g.cmax *= 1.0 + fabs(c1) + fabs(c2);
        }
    }
    return true;
}

// generation of n_toys toys into columns (positions out_pos[t] .. + counts[t]); host arrays in
static cudaError_t gen_launch(const GenConst& g, const int64_t* counts, const uint64_t* states, const int64_t* out_pos,
                       int n_toys, double* const* out, int sm_count, cudaStream_t stream, int* failed)
{
    std::vector<int64_t> first(n_toys + 1, 0);
    for (int t = 0; t < n_toys; ++t) first[t + 1] = first[t] + counts[t];
    const int64_t total = first[n_toys];
    *failed = 0;
    if (total == 0) return cudaSuccess;
    cudaError_t et = ensure_gen_tables();
    if (et != cudaSuccess) return et;
    int64_t *d_first = nullptr, *d_count = nullptr, *d_pos = nullptr;
    uint64_t* d_state = nullptr;
    int* d_fail = nullptr;
    cudaError_t e = cudaMalloc(&d_first, sizeof(int64_t) * (n_toys + 1));
    if (e == cudaSuccess) e = cudaMalloc(&d_count, sizeof(int64_t) * n_toys);
    if (e == cudaSuccess) e = cudaMalloc(&d_pos, sizeof(int64_t) * n_toys);
    if (e == cudaSuccess) e = cudaMalloc(&d_state, sizeof(uint64_t) * n_toys);
    if (e == cudaSuccess) e = cudaMalloc(&d_fail, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_first, first.data(), sizeof(int64_t) * (n_toys + 1), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_count, counts, sizeof(int64_t) * n_toys, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_pos, out_pos, sizeof(int64_t) * n_toys, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_state, states, sizeof(uint64_t) * n_toys, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_fail, 0, sizeof(int), stream);
    if (e == cudaSuccess) {
        GenArgs a;
        memset(&a, 0, sizeof a);
        a.g = g;
        a.toy_first = d_first;
        a.toy_count = d_count;
        a.toy_state = d_state;
        a.n_toys = n_toys;
        a.total = total;
        a.out_pos = d_pos;
        for (int d = 0; d < 4; ++d) a.out[d] = out[d];
        a.fail = d_fail;
        int blocks = (int)std::min<int64_t>((total + 255) / 256, (int64_t)sm_count * 16);
        gen_kernel<<<blocks, 256, 0, stream>>>(a);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(failed, d_fail, sizeof(int), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (d_first) cudaFree(d_first);
    if (d_count) cudaFree(d_count);
    if (d_pos) cudaFree(d_pos);
    if (d_state) cudaFree(d_state);
    if (d_fail) cudaFree(d_fail);
    return e;
}

uint64_t gen_stream_state(uint64_t seed, uint64_t stream) { return stream_state(seed, stream); }

namespace {
// sum (m - ma) over each toy's events [begin, end), one block per toy, fixed order
__global__ void __launch_bounds__(256) toy_sums_kernel(const double* m, const int64_t* begin, const int64_t* end,
                                                       double ma, double* out)
{
    __shared__ double s[256];
    const int t = blockIdx.x;
    double v = 0.0;
    for (int64_t i = begin[t] + threadIdx.x; i < end[t]; i += blockDim.x) v += m[i] - ma;
    s[threadIdx.x] = v;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[t] = s[0];
}
}  // namespace

int gen_toys(int kind, const double* ranges, const double* theta, const int64_t* counts, int n_toys, uint64_t seed,
             const int64_t* out_pos, double* const* out, int sm_count, cudaStream_t stream)
{
    GenConst g;
    if (!gen_setup(kind, ranges, theta, g)) return NLL_ERR_ARG;
    std::vector<uint64_t> states(n_toys);
    for (int t = 0; t < n_toys; ++t) states[t] = stream_state(seed, (uint64_t)t);
    int failed = 0;
    cudaError_t e = gen_launch(g, counts, states.data(), out_pos, n_toys, out, sm_count, stream, &failed);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? NLL_ERR_OOM : NLL_ERR_CUDA;
    return failed ? NLL_ERR_NOT_CONVERGED : NLL_OK;
}

cudaError_t toy_sums(const double* m, const int64_t* d_begin, const int64_t* d_end, double ma, int n_toys,
                     double* d_out, cudaStream_t stream)
{
    if (n_toys == 0) return cudaSuccess;
    toy_sums_kernel<<<n_toys, 256, 0, stream>>>(m, d_begin, d_end, ma, d_out);
    return cudaGetLastError();
}

}  // namespace gbnll

using namespace gbnll;

extern "C" {

int nll_generate(int kind, const double* obs_ranges, const double* theta, int64_t n_events, uint64_t seed,
                 uint64_t stream, int device, uintptr_t cuda_stream, double* const* dev_columns)
{
    if ((kind != NLL_MODEL_MASS1D && kind != NLL_MODEL_KSTARMUMU4D) || !obs_ranges || !theta || n_events < 0)
        return NLL_ERR_ARG;
    const int ndim = kind == NLL_MODEL_MASS1D ? 1 : 4;
    if (n_events > 0 && !dev_columns) return NLL_ERR_ARG;
    for (int d = 0; d < ndim && n_events > 0; ++d)
        if (!dev_columns[d]) return NLL_ERR_ARG;
    double ranges[8] = {obs_ranges[0], obs_ranges[1], -1.0, 1.0, -1.0, 1.0, -kPiG, kPiG};
    if (!(ranges[0] < ranges[1])) return NLL_ERR_ARG;
    GenConst g;
    if (!gen_setup(kind, ranges, theta, g)) return NLL_ERR_ARG;
    if (cudaSetDevice(device) != cudaSuccess) return NLL_ERR_CUDA;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    uint64_t st = stream_state(seed, stream);
    int64_t pos = 0;
    double* out[4] = {dev_columns[0], ndim > 1 ? dev_columns[1] : nullptr, ndim > 1 ? dev_columns[2] : nullptr,
                      ndim > 1 ? dev_columns[3] : nullptr};
    int failed = 0;
    cudaError_t e = gen_launch(g, &n_events, &st, &pos, 1, out, sms, (cudaStream_t)cuda_stream, &failed);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? NLL_ERR_OOM : NLL_ERR_CUDA;
    return failed ? NLL_ERR_NOT_CONVERGED : NLL_OK;
}

int nll_diag_uniforms(uint64_t seed, uint64_t stream, int64_t n, int device, double* host_out)
{
    if (n < 0 || (n > 0 && !host_out)) return NLL_ERR_ARG;
    if (n == 0) return NLL_OK;
    if (cudaSetDevice(device) != cudaSuccess) return NLL_ERR_CUDA;
    double* d = nullptr;
    if (cudaMalloc(&d, sizeof(double) * n) != cudaSuccess) return NLL_ERR_OOM;
    uniforms_kernel<<<(int)std::min<int64_t>((n + 255) / 256, 4096), 256>>>(stream_state(seed, stream), n, d);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpy(host_out, d, sizeof(double) * n, cudaMemcpyDeviceToHost);
    cudaFree(d);
    return e == cudaSuccess ? NLL_OK : NLL_ERR_CUDA;
}

}  // extern "C"
