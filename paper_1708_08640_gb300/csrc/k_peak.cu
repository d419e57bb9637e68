// The FP32 CUDA-core roof of this GPU, measured: every SM runs long chains of independent
// FMAs (scalar FFMA, and the packed two-lane FFMA2 of the sm_100 family), timed with CUDA
// events on a private stream.  The FP32 form's kernels are bound by this pipe; their roofline
// fractions are taken against the larger of the two rates.
#include <cuda_runtime.h>

#include "s3cmtf.h"

namespace {

constexpr int kChains = 16;      // independent accumulators per thread
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) k_peak_ffma(float* out, int iters, float b, float c) {
    float a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = (float)(threadIdx.x + k);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == 12345.678f) out[blockIdx.x] = s;   // keeps the chains live; never true for the inputs
}

__global__ void __launch_bounds__(kThreads) k_peak_ffma2(float* out, int iters, float b, float c) {
    float2 a[kChains / 2];
#pragma unroll
    for (int k = 0; k < kChains / 2; ++k) a[k] = make_float2((float)(threadIdx.x + k), (float)k);
    const float2 bb = make_float2(b, b), cc = make_float2(c, c);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < kChains / 2; ++k) a[k] = __ffma2_rn(a[k], bb, cc);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains / 2; ++k) s += a[k].x + a[k].y;
    if (s == 12345.678f) out[blockIdx.x] = s;
}

template <typename K>
cudaError_t time_kernel(K kernel, int grid, int iters, cudaStream_t st, float* out, float* ms) {
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e != cudaSuccess) return e;
    e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        cudaEventDestroy(e0);
        return e;
    }
    // b, c keep every value finite and away from the sentinel: a <- a * 0.999 + 0.001
    kernel<<<grid, kThreads, 0, st>>>(out, iters, 0.999f, 0.001f);   // warm-up
    e = cudaGetLastError();
    float best = 0.f;
    for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
        e = cudaEventRecord(e0, st);
        if (e == cudaSuccess) kernel<<<grid, kThreads, 0, st>>>(out, iters, 0.999f, 0.001f);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float t = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
        if (e == cudaSuccess && (rep == 0 || t < best)) best = t;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms = best;
    return e;
}

}  // namespace

extern "C" int s3_measure_fp32_peak(double* ffma_tflops, double* ffma2_tflops, double* sm_mhz) {
    int dev = 0, sms = 0, clk_khz = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return S3_ERR_CUDA;
    if (cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, dev) != cudaSuccess) clk_khz = 0;
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return S3_ERR_CUDA;
    // a small sink for the stores that keep the chains live (never taken for these inputs)
    float* out = nullptr;
    const int grid = sms * 8;                 // 8 CTAs of 256 threads per SM: 64 warps
    if (cudaMalloc(&out, sizeof(float) * grid) != cudaSuccess) {
        cudaStreamDestroy(st);
        return S3_ERR_OOM;
    }
    const int iters = 1 << 11;   // 20 GFLOP a launch: about 0.26 ms at 80 TFLOP/s
    float ms1 = 0.f, ms2 = 0.f;
    cudaError_t e = time_kernel(k_peak_ffma, grid, iters, st, out, &ms1);
    if (e == cudaSuccess) e = time_kernel(k_peak_ffma2, grid, iters, st, out, &ms2);
    cudaFree(out);
    cudaStreamDestroy(st);
    if (e != cudaSuccess || ms1 <= 0.f || ms2 <= 0.f) return S3_ERR_CUDA;
    const double flops = 2.0 * (double)grid * kThreads * (double)iters * kChains;
    if (ffma_tflops) *ffma_tflops = flops / (ms1 * 1e-3) / 1e12;
    if (ffma2_tflops) *ffma2_tflops = flops / (ms2 * 1e-3) / 1e12;
    if (sm_mhz) *sm_mhz = clk_khz / 1000.0;
    return S3_OK;
}
