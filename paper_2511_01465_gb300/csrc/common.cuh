// common.cuh -- device helpers shared by the solver's kernels: memory-order
// primitives for inter-CTA signalling, bounded waits, a grid barrier for
// cooperative launches, and the workspace / launch bookkeeping of the host side.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <float.h>

#include "pitn.h"

namespace pitn {

// ---------------------------------------------------------------------------
// Memory-order primitives (gpu scope).
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Every spin-wait in the library gives up after a bounded time (default 2 s,
// passed in by the host, see WaitLimits) and raises PITN_ETIMEOUT instead of
// hanging the device.
constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s

// Error word written by kernels (0 = fine).
__device__ __forceinline__ void raise_error(int* err, int code) { atomicCAS(err, 0, code); }

// Grid-wide barrier for cooperative launches (all CTAs co-resident).
// count/gen live in device memory zeroed before the launch.  Returns false
// (and sets *err) when the wait times out or another CTA already failed.
__device__ __forceinline__ bool grid_barrier(unsigned* count, unsigned* gen, unsigned nblocks,
                                             int* err, uint64_t limit_ns = kWaitLimitNs) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        unsigned g = ld_acquire_u32(gen);
        __threadfence();
        unsigned arrived = atomicAdd(count, 1u);
        if (arrived == nblocks - 1) {
            atomicExch(count, 0u);
            __threadfence();
            st_release_u32(gen, g + 1);
        } else {
            if (limit_ns == 0) limit_ns = kWaitLimitNs;
            uint64_t t0 = globaltimer_ns();
            while (ld_acquire_u32(gen) == g) {
                if (*(volatile int*)err != 0) { ok = 0; break; }
                if (globaltimer_ns() - t0 > limit_ns) {
                    raise_error(err, PITN_ETIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(32);
            }
        }
        if (*(volatile int*)err != 0) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    __threadfence();
    return s_ok != 0;
}

// |x| as its IEEE bit pattern, computed on the integer pipe: the register
// pair is split and the sign bit cleared in the high word by a 32-bit AND.
// (fabs(), or a 64-bit mask on the bit pattern, compiles to an FP64-pipe
// instruction, which on GB300 costs as much as a DFMA.)  Non-negative doubles
// order like their bit patterns; NaN orders above +inf.
__device__ __forceinline__ unsigned long long abs_bits(double x) {
    unsigned lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=r"(lo), "=r"(hi) : "d"(x));
    hi &= 0x7fffffffu;
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "r"(lo), "r"(hi));
    return r;
}
constexpr unsigned long long kInfBitsAbs = 0x7ff0000000000000ull;  // bits of +inf

}  // namespace pitn

// ---------------------------------------------------------------------------
// Host-side helpers (implemented in api.cu).
// ---------------------------------------------------------------------------
namespace pitn_host {

// Scratch memory cache of the current device; returns nullptr on failure.
void* workspace(size_t bytes, int slot = 0);
// Counts kernel launches issued by the library.
void count_launch(int64_t n = 1);
// Device properties of the current device (cached).
const cudaDeviceProp& props();

}  // namespace pitn_host
