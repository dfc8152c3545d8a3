// calibrate.cu -- FP64 throughput calibration on the current GPU (diagnostic entry point).
//
// The fused kernels are bound by the FP64 pipe, so their roofline is the FP64 issue rate.
// nll_calibrate_fp64 measures it with independent DFMA chains, and measures CUDA's own
// exp(), log() and 1.0/x and this library's fexp / frcp in the same way, so that the cost
// of a transcendental can be expressed in DFMA issue slots on the running GPU.
#include <cuda_runtime.h>
#include <math.h>

#include "../../include/gbnll.h"
#include "fp64_math.cuh"

namespace {

constexpr int kChains = 8;

__device__ double g_cal_tab[gbnll::kTabDoubles];

template <int OP>
__global__ void __launch_bounds__(256) cal_kernel(double* out, int iters, double a)
{
    __shared__ double s_tab[gbnll::kExpTable];
    for (int j = threadIdx.x; j < gbnll::kExpTable; j += blockDim.x) s_tab[j] = g_cal_tab[j];
    __syncthreads();
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 0.5 + 1e-3 * (c + (gid & 7));
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            if (OP == 0) x[c] = fma(x[c], a, 0.25);            // DFMA
            if (OP == 1) x[c] = exp(-x[c]);                    // CUDA exp
            if (OP == 2) x[c] = 1.0 / (x[c] + 1.0);            // CUDA division (+1 DADD)
            if (OP == 3) x[c] = log(x[c] + 3.0);               // CUDA log (+1 DADD)
            if (OP == 4) x[c] = gbnll::fexp_scaled(-x[c], s_tab);  // library exp
            if (OP == 5) x[c] = gbnll::frcp(x[c] + 1.0);       // library reciprocal (+1 DADD)
        }
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    out[gid] = s;
}

template <int OP>
cudaError_t time_op(double* out, int blocks, int iters, double a, float* ms)
{
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) return e;
    cal_kernel<OP><<<blocks, 256>>>(out, iters, a);  // warm-up
    cudaEventRecord(e0);
    for (int r = 0; r < 3; ++r) cal_kernel<OP><<<blocks, 256>>>(out, iters, a);
    cudaEventRecord(e1);
    e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventElapsedTime(ms, e0, e1);
    *ms /= 3.0f;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return e;
}

cudaError_t upload_table()
{
    static double tab[gbnll::kTabDoubles];
    gbnll::fill_device_tables(tab);
    return cudaMemcpyToSymbol(g_cal_tab, tab, sizeof tab);
}

__global__ void __launch_bounds__(256) diag_kernel(int fn, const double* x, double* y, int64_t n)
{
    __shared__ double s_tab[gbnll::kTabDoubles];
    for (int j = threadIdx.x; j < gbnll::kTabDoubles; j += blockDim.x) s_tab[j] = g_cal_tab[j];
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double v;
        if (fn == 0) {
            v = gbnll::fexp_scaled(x[i], s_tab);
        } else if (fn == 1) {
            v = gbnll::frcp(x[i]);
        } else if (fn == 4) {
            v = gbnll::flog(x[i], s_tab);
        } else if (fn == 5) {
            v = gbnll::frcp_approx(x[i]);
        } else if (fn == 6) {
            v = gbnll::frcp_newton(x[i]);
        } else if (fn == 7) {
            v = gbnll::fsqrt(x[i]);
        } else {
            double sv, cv;
            gbnll::fsincos_pi(x[i], s_tab + gbnll::kTrigOffset, sv, cv);
            v = fn == 2 ? sv : cv;
        }
        y[i] = v;
    }
}

}  // namespace

extern "C" int nll_diag_math(int device, int fn, const double* x, double* y, int64_t n)
{
    if (fn < 0 || fn > 7 || n < 0 || (n > 0 && (!x || !y))) return NLL_ERR_ARG;
    if (n == 0) return NLL_OK;
    if (cudaSetDevice(device) != cudaSuccess) return NLL_ERR_CUDA;
    if (upload_table() != cudaSuccess) return NLL_ERR_CUDA;
    double *dx = nullptr, *dy = nullptr;
    if (cudaMalloc(&dx, sizeof(double) * n) != cudaSuccess) return NLL_ERR_OOM;
    if (cudaMalloc(&dy, sizeof(double) * n) != cudaSuccess) {
        cudaFree(dx);
        return NLL_ERR_OOM;
    }
    cudaError_t e = cudaMemcpy(dx, x, sizeof(double) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        int blocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
        diag_kernel<<<blocks, 256>>>(fn, dx, dy, n);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(y, dy, sizeof(double) * n, cudaMemcpyDeviceToHost);
    cudaFree(dx);
    cudaFree(dy);
    return e == cudaSuccess ? NLL_OK : NLL_ERR_CUDA;
}

extern "C" int nll_calibrate_fp64(int device, double* rates)
{
    if (!rates) return NLL_ERR_ARG;
    if (cudaSetDevice(device) != cudaSuccess) return NLL_ERR_CUDA;
    cudaDeviceProp p;
    if (cudaGetDeviceProperties(&p, device) != cudaSuccess) return NLL_ERR_CUDA;
    if (upload_table() != cudaSuccess) return NLL_ERR_CUDA;
    const int blocks = p.multiProcessorCount * 8;
    double* out = nullptr;
    if (cudaMalloc(&out, sizeof(double) * blocks * 256) != cudaSuccess) return NLL_ERR_OOM;
    const int it_fast = 4096, it_slow = 256;
    float ms[6] = {0};
    cudaError_t e = time_op<0>(out, blocks, it_fast, 0.999999, &ms[0]);
    if (e == cudaSuccess) e = time_op<1>(out, blocks, it_slow, 0.0, &ms[1]);
    if (e == cudaSuccess) e = time_op<2>(out, blocks, it_slow, 0.0, &ms[2]);
    if (e == cudaSuccess) e = time_op<3>(out, blocks, it_slow, 0.0, &ms[3]);
    if (e == cudaSuccess) e = time_op<4>(out, blocks, it_slow, 0.0, &ms[4]);
    if (e == cudaSuccess) e = time_op<5>(out, blocks, it_slow, 0.0, &ms[5]);
    cudaFree(out);
    if (e != cudaSuccess) return NLL_ERR_CUDA;
    const double per = (double)blocks * 256 * kChains;
    const int iters[6] = {it_fast, it_slow, it_slow, it_slow, it_slow, it_slow};
    for (int i = 0; i < 6; ++i) rates[i] = per * iters[i] / (ms[i] * 1e-3);
    return NLL_OK;
}
