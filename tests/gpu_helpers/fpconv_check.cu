// Checks the integer-pipe FP64 <-> FP32 conversions (csrc/fpconv.cuh)
// against the hardware conversions on the GPU: special values, binade
// boundaries and 2^24 random bit patterns.  Prints one line of counts; the
// pytest wrapper (tests/test_gpu_fpconv.py) builds, runs and parses it.
#include <cstdio>
#include <cstdint>
#include <cmath>
#include <cuda_runtime.h>

#include "fpconv.cuh"

__device__ unsigned long long mix64(unsigned long long z) {  // splitmix64 finaliser
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

// counts[0]: d2f mismatches outside exact ties and subnormal results
// counts[1]: d2f results further than half an ulp from the hardware result
// counts[2]: f2d mismatches on normal, infinite or NaN inputs
// counts[3]: f2d results that are not zero for subnormal inputs
// counts[4]: values checked
__global__ void check(const double* special, int nspecial, long long nrand, unsigned long long* counts) {
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long total = nspecial + nrand;
    for (long long i = tid; i < total; i += (long long)gridDim.x * blockDim.x) {
        double x;
        if (i < nspecial) {
            x = special[i];
        } else {
            const unsigned long long r = mix64((unsigned long long)i);
            // bias the exponent towards the float range half of the time
            unsigned long long bits = r;
            if (r & 1ull) {
                const unsigned long long e = 1023ull - 140ull + ((r >> 1) % 280ull);
                bits = (r & 0x800fffffffffffffull) | (e << 52);
            }
            x = __longlong_as_double((long long)bits);
        }
        const float a = pitn::d2f_int(x);
        const float h = __double2float_rn(x);
        const unsigned ab = __float_as_uint(a), hb = __float_as_uint(h);
        const bool hsub = (hb & 0x7f800000u) == 0u && (hb & 0x7fffffu) != 0u;
        const bool hnan = isnan(h), anan = isnan(a);
        bool bad = false;
        if (hnan || anan) {
            bad = hnan != anan;
        } else if (hsub || (hb & 0x7fffffffu) == 0u) {
            // subnormal or zero results: flushed to a zero of the right sign,
            // or (rounding up to the smallest normal) that normal
            bad = (ab & 0x7fffffffu) != 0u && (ab & 0x7fffffffu) != 0x00800000u;
            bad = bad || ((ab ^ hb) & 0x80000000u);
        } else if (ab != hb) {
            // allowed: an exact tie rounded away from zero instead of to even
            const unsigned long long xb = (unsigned long long)__double_as_longlong(x);
            const bool tie = (xb & 0x1fffffffull) == 0x10000000ull;
            bad = !tie;
        }
        if (bad) atomicAdd(&counts[0], 1ull);
        if (!hnan && !isinf(h) && !isinf(a) && !hsub && (hb & 0x7fffffffu) != 0u) {
            const double ulp = (double)nextafterf(fabsf(h), INFINITY) - (double)fabsf(h);
            if (fabs((double)a - x) > 0.5 * ulp * (1.0 + 1e-12)) atomicAdd(&counts[1], 1ull);
        }
        // float -> double on the 32-bit pattern taken from the same draw
        const unsigned fb = (unsigned)__double_as_longlong(x) ^ (unsigned)(__double_as_longlong(x) >> 32);
        const float v = __uint_as_float(fb);
        const double dv = pitn::f2d_int(v), dh = (double)v;
        const bool vsub = (fb & 0x7f800000u) == 0u;
        if (vsub) {
            if (dv != 0.0 || signbit(dv) != signbit(v)) atomicAdd(&counts[3], 1ull);
        } else if (isnan(v)) {
            if (!isnan(dv)) atomicAdd(&counts[2], 1ull);
        } else if (__double_as_longlong(dv) != __double_as_longlong(dh)) {
            atomicAdd(&counts[2], 1ull);
        }
        atomicAdd(&counts[4], 1ull);
    }
}

int main() {
    const double sp[] = {0.0, -0.0, 1.0, -1.0, 0.1, 1.0 / 3.0, 3.4028234663852886e38, 3.4028235677973366e38,
                         3.402823669209385e38, 1e39, -1e39, 1.1754943508222875e-38, 1.1754942e-38, 1e-45,
                         -1e-300, 1e300, INFINITY, -INFINITY, NAN, 16777217.0, 16777219.0, 1.0000000596046448,
                         1.0000001788139343, 2.9802322387695312e-08, 65504.0, 1e-7, -123456.789};
    const int ns = sizeof(sp) / sizeof(sp[0]);
    double* dsp = nullptr;
    unsigned long long* dc = nullptr;
    if (cudaMalloc(&dsp, sizeof(sp)) != cudaSuccess || cudaMalloc(&dc, 5 * sizeof(unsigned long long)) != cudaSuccess)
        return 2;
    cudaMemcpy(dsp, sp, sizeof(sp), cudaMemcpyHostToDevice);
    cudaMemset(dc, 0, 5 * sizeof(unsigned long long));
    check<<<1024, 256>>>(dsp, ns, 1ll << 24, dc);
    unsigned long long c[5] = {};
    cudaError_t e = cudaMemcpy(c, dc, sizeof(c), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        printf("cuda error %s\n", cudaGetErrorString(e));
        return 1;
    }
    printf("d2f_bad %llu d2f_far %llu f2d_bad %llu f2d_sub_bad %llu checked %llu\n", c[0], c[1], c[2], c[3], c[4]);
    cudaFree(dsp);
    cudaFree(dc);
    return 0;
}
