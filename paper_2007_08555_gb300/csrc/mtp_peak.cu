// Measured FP32 FMA throughput of the current device (instrumentation for the ALU roofline of the
// evaluation kernels; the paper has no counterpart).  Every thread runs kChains independent
// chains of fused multiply-adds (enough independent work to cover the FMA latency at full
// occupancy); the grid fills every SM with 2048 threads.  Timed with CUDA events on a private
// stream, median of the repeats.
#include <cuda_runtime.h>
#include <algorithm>
#include <vector>
#include "../../include/mtp.h"

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 32;
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) k_ffma_peak(float* out, int iters, float seed) {
    float a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = seed + 0.001f * (float)(threadIdx.x + k);
    const float mul = 0.999999f, add = 1e-7f * seed;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], mul, add);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == 12345.678f) out[0] = s;  // keeps the chains live; never true for these inputs
}

}  // namespace

extern "C" mtp_status mtp_fp32_peak(int repeats, double* tflops) {
    if (!tflops || repeats < 1 || repeats > 1000) return MTP_EINVAL;
    int dev = 0, n_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return MTP_ECUDA;
    const int blocks = n_sm * (2048 / kThreads);
    const int iters = 4096;
    float* out = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    mtp_status status = MTP_OK;
    std::vector<double> rates;
    if (cudaMalloc(&out, sizeof(float)) != cudaSuccess) return MTP_ENOMEM;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        status = MTP_ECUDA;
    } else {
        const double flops = 2.0 * kChains * kUnroll * (double)iters * kThreads * blocks;
        for (int r = 0; r < repeats + 2 && status == MTP_OK; ++r) {  // two warm-up launches
            cudaEventRecord(e0, st);
            k_ffma_peak<<<blocks, kThreads, 0, st>>>(out, iters, 1.0f + 1e-3f * (float)r);
            cudaEventRecord(e1, st);
            float ms = 0.f;
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
                status = MTP_ECUDA;
            else if (r >= 2)
                rates.push_back(flops / (ms * 1e-3) / 1e12);
        }
    }
    if (status == MTP_OK) {
        std::sort(rates.begin(), rates.end());
        *tflops = rates[rates.size() / 2];
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    cudaFree(out);
    return status;
}
