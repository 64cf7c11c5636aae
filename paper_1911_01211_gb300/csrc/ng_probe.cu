// FP64 throughput probe (ng_fp64_probe): sustained rate of the FP64 FMA pipe (DFMA) and of the
// FP64 tensor path (DMMA, mma.sync m8n8k4 f64) on the current device, for the roofline of the
// FP64 time-step kernels.  Both kernels are plain register loops with fixed trip counts.
#include <cuda_runtime.h>

#include "../../include/ng.h"

namespace {

constexpr int kChains = 8;       // independent FMA chains per thread
constexpr int kThreads = 256;

// written only if a result matched an impossible value: keeps the loops from being removed
__device__ double g_probe_sink;

__global__ void __launch_bounds__(kThreads) k_probe_dfma(int iters, double seed) {
    double a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = seed + 1e-3 * (threadIdx.x + c);
    const double b = 0.999999, d = 1e-7;
#pragma unroll 4
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], b, d);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    if (s == -1.0) g_probe_sink = s;   // the chains converge to 0.1 each: never true
}

// one warp-wide m8n8k4 FP64 product per instruction: 8 * 8 * 4 = 256 FMA = 512 flop
__global__ void __launch_bounds__(kThreads) k_probe_dmma(int iters, double seed) {
    double acc[4][2];
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[c][0] = acc[c][1] = 0.0;
    const double av = seed + 1e-3 * threadIdx.x, bv = 0.5 - 1e-3 * threadIdx.x;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < 4; ++c)
            asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};\n"
                         : "+d"(acc[c][0]), "+d"(acc[c][1])
                         : "d"(av), "d"(bv));
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < 4; ++c) s += acc[c][0] + acc[c][1];
    if (s == -1.0) g_probe_sink = s;   // sums of positive products: never true
}

}  // namespace

extern "C" ng_status ng_fp64_probe(double* out, void* stream) {
    if (!out) return NG_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return NG_ECUDA;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        if (e0) cudaEventDestroy(e0);
        return NG_ECUDA;
    }
    const int blocks = sms * 8;
    const int it_fma = 20000, it_mma = 20000;
    ng_status st = NG_OK;
    float ms_fma = 0.f, ms_mma = 0.f;
    // about a quarter second of warm-up (the clocks ramp up under load), then the best of
    // three timed launches of each kernel
    for (int w = 0; w < 3; ++w) k_probe_dfma<<<blocks, kThreads, 0, s>>>(it_fma, 1.0);
    auto timed = [&](bool mma, float* best) {
        *best = 1e30f;
        for (int rep = 0; rep < 3 && st == NG_OK; ++rep) {
            float ms = 0.f;
            cudaEventRecord(e0, s);
            if (mma) k_probe_dmma<<<blocks, kThreads, 0, s>>>(it_mma, 1.0);
            else k_probe_dfma<<<blocks, kThreads, 0, s>>>(it_fma, 1.0);
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) st = NG_ECUDA;
            if (ms > 0.f && ms < *best) *best = ms;
        }
    };
    timed(false, &ms_fma);
    timed(true, &ms_mma);
    if (cudaGetLastError() != cudaSuccess) st = NG_ECUDA;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != NG_OK) return st;
    const double threads = (double)blocks * kThreads, warps = threads / 32.0;
    out[0] = 2.0 * kChains * (double)it_fma * threads / (ms_fma * 1e-3) / 1e12;
    out[1] = 512.0 * 4.0 * (double)it_mma * warps / (ms_mma * 1e-3) / 1e12;
    out[2] = (double)sms;
    return NG_OK;
}
