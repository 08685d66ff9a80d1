// probe.cu -- measured FMA issue rates of the current device, the
// denominators of the ALU rooflines the benchmark reports (not part of the
// paper's method).
//
// A register-only kernel: every thread runs kChains independent FMA
// dependency chains for `iters` rounds, so the FMA pipe, not the latency of
// one chain, sets the rate; one block of 256 threads per 1/8 of an SM's
// thread slots, 8 blocks per SM.  The result of every chain is folded into
// one value per thread and stored only when it equals a value no input can
// produce, so the compiler keeps the work and the kernel writes nothing.
#include <cuda_runtime.h>

#include <cstdint>

#include "common.cuh"
#include "solver.h"

namespace pitn {

constexpr int kProbeChains = 8;
constexpr int kProbeBlock = 256;

template <typename T>
__global__ void __launch_bounds__(kProbeBlock) fma_rate_kernel(T seed, T mul, T add, int iters, T* sink) {
    T a[kProbeChains];
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) a[c] = seed + (T)(threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kProbeChains; ++c) a[c] = fma(a[c], mul, add);
    }
    T s = (T)0;
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) s += a[c];
    if (s == (T)-12345.0) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace pitn

extern "C" int pitn_probe_fma_rate(int kind, double* fma_per_s) {
    using namespace pitn;
    using namespace pitn_host;
    if (!fma_per_s || (kind != 0 && kind != 1)) return PITN_EINVAL;
    std::lock_guard<std::recursive_mutex> lk(api_mutex());
    const int sms = props().multiProcessorCount;
    const int grid = sms * 8;
    // FP32 issues ~60x faster than FP64 on GB300: more rounds keep the kernel
    // long enough (several ms) for event timing
    const int iters = kind == 0 ? 2048 : 65536;
    void* sink = workspace((size_t)grid * kProbeBlock * sizeof(double), kSlotAux2);
    if (!sink) return PITN_ENOMEM;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return PITN_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return PITN_ECUDA;
    }
    float best = 0.f;
    int rc = PITN_OK;
    for (int rep = 0; rep < 4 && rc == PITN_OK; ++rep) {   // the first launch warms up
        cudaEventRecord(e0, 0);
        if (kind == 0)
            fma_rate_kernel<double><<<grid, kProbeBlock>>>(1.0, 0.999999, 1e-6, iters, (double*)sink);
        else
            fma_rate_kernel<float><<<grid, kProbeBlock>>>(1.f, 0.9999f, 1e-4f, iters, (float*)sink);
        count_launch(1);
        cudaEventRecord(e1, 0);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
            rc = PITN_ECUDA;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && (best == 0.f || ms < best)) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != PITN_OK) return rc;
    const double fmas = (double)grid * kProbeBlock * (double)iters * kProbeChains;
    *fma_per_s = fmas / (best / 1e3);
    return PITN_OK;
}
