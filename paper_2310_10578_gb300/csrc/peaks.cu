// peaks.cu -- measured FP32 FFMA and SFU (MUFU) throughput of the current
// device: the denominators of the evaluation's ALU roofline.
//
// Each thread runs independent dependency chains (enough of them to hide the
// pipeline latency) for a fixed number of iterations on registers; the grid
// fills every SM with 8 resident blocks; the time is taken with CUDA events
// around one launch after a warm-up launch.  FFMA: 2 flops per instruction.
// SFU: one ex2.approx.f32 per operation (the special-function unit's
// exponential), written as inline PTX.
#include "internal.h"

namespace creep {

namespace {

constexpr int PK_CHAINS = 8;
constexpr int PK_THREADS = 256;

__global__ void __launch_bounds__(PK_THREADS) k_ffma(float *out, int iters, float a, float b) {
    float x[PK_CHAINS];
#pragma unroll
    for (int k = 0; k < PK_CHAINS; ++k) x[k] = threadIdx.x * 1e-3f + k;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < PK_CHAINS; ++k) x[k] = fmaf(x[k], a, b);
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < PK_CHAINS; ++k) s += x[k];
    if (s == 12345.678f) out[blockIdx.x] = s;         // keeps the chains live; never true in practice
}

__device__ __forceinline__ float ex2_approx(float v) {
    float r;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}

__global__ void __launch_bounds__(PK_THREADS) k_mufu(float *out, int iters, float a) {
    float x[PK_CHAINS];
#pragma unroll
    for (int k = 0; k < PK_CHAINS; ++k) x[k] = threadIdx.x * 1e-6f + k * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < PK_CHAINS; ++k) x[k] = ex2_approx(x[k]) * a;   // stays near 1: 2^x * a, x ~ 0
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < PK_CHAINS; ++k) s += x[k];
    if (s == 12345.678f) out[blockIdx.x] = s;
}

}  // namespace

}  // namespace creep

using namespace creep;

extern "C" int rt_alu_peaks(double *ffma_tflops, double *mufu_gops, void *stream) {
    if (!ffma_tflops || !mufu_gops) {
        set_error("rt_alu_peaks: NULL argument");
        return RT_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    float *out = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&out, sizeof(float) * 8 * (size_t)nsm);
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    const int grid = 8 * nsm, iters_f = 1 << 16, iters_m = 1 << 13;
    float ms_f = 0.0f, ms_m = 0.0f;
    if (e == cudaSuccess) {
        k_ffma<<<grid, PK_THREADS, 0, st>>>(out, iters_f / 16, 0.999999f, 1e-7f);      // warm-up
        cudaEventRecord(t0, st);
        k_ffma<<<grid, PK_THREADS, 0, st>>>(out, iters_f, 0.999999f, 1e-7f);
        cudaEventRecord(t1, st);
        e = cudaEventSynchronize(t1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms_f, t0, t1);
    }
    if (e == cudaSuccess) {
        k_mufu<<<grid, PK_THREADS, 0, st>>>(out, iters_m / 16, 0.5f);
        cudaEventRecord(t0, st);
        k_mufu<<<grid, PK_THREADS, 0, st>>>(out, iters_m, 0.5f);
        cudaEventRecord(t1, st);
        e = cudaEventSynchronize(t1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms_m, t0, t1);
    }
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    cudaFree(out);
    if (e != cudaSuccess) {
        set_error(std::string("rt_alu_peaks: ") + cudaGetErrorString(e));
        return RT_ERR_CUDA;
    }
    const double threads = (double)grid * PK_THREADS;
    *ffma_tflops = 2.0 * PK_CHAINS * (double)iters_f * threads / (ms_f * 1e-3) / 1e12;
    *mufu_gops = (double)PK_CHAINS * (double)iters_m * threads / (ms_m * 1e-3) / 1e9;
    return RT_OK;
}

// ---------------------------------------------------------------------------
// Measured L2 read bandwidth: a 32 MiB buffer (well inside the L2) read by
// every SM, 16 B a thread per access through L2 only (ld.global.cg: no L1
// reuse), several passes after a warm-up pass that brings it into the L2.
namespace creep {
namespace {
__global__ void __launch_bounds__(PK_THREADS) k_l2_read(const float4 *__restrict__ buf, size_t n, int passes,
                                                        float *out) {
    float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (int p = 0; p < passes; ++p)
        for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
            const float4 v = __ldcg(buf + i);
            s.x += v.x; s.y += v.y; s.z += v.z; s.w += v.w;
        }
    if (s.x + s.y + s.z + s.w == 12345.678f) out[blockIdx.x] = s.x;   // keeps the loads live
}
}  // namespace
}  // namespace creep

extern "C" int rt_l2_peak(double *l2_gbs, void *stream) {
    if (!l2_gbs) {
        set_error("rt_l2_peak: NULL argument");
        return RT_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = (size_t)32 << 20, n = bytes / sizeof(float4);
    const int passes = 16;
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    float4 *buf = nullptr;
    float *out = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&buf, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&out, sizeof(float) * 8 * (size_t)nsm);
    if (e == cudaSuccess) e = cudaMemsetAsync(buf, 0, bytes, st);
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    float ms = 0.0f;
    const int grid = 8 * nsm;
    if (e == cudaSuccess) {
        k_l2_read<<<grid, PK_THREADS, 0, st>>>(buf, n, 1, out);             // warm-up: the buffer into L2
        cudaEventRecord(t0, st);
        k_l2_read<<<grid, PK_THREADS, 0, st>>>(buf, n, passes, out);
        cudaEventRecord(t1, st);
        e = cudaEventSynchronize(t1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
    }
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    cudaFree(buf);
    cudaFree(out);
    if (e != cudaSuccess) {
        set_error(std::string("rt_l2_peak: ") + cudaGetErrorString(e));
        return RT_ERR_CUDA;
    }
    *l2_gbs = (double)bytes * passes / (ms * 1e-3) / 1e9;
    return RT_OK;
}
