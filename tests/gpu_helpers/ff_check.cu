// Checks the float-float arithmetic of csrc/ffarith.cuh on the GPU against
// FP64 references: the integer-pipe split of a double into hi + lo, and the
// sum and product of two float-float values, on special values and 2^22
// random operands per check.  Prints one line of counts; the pytest wrapper
// (tests/test_gpu_ff.py) builds, runs and parses it.
#include <cstdio>
#include <cstdint>
#include <cmath>
#include <cuda_runtime.h>

#include "ffarith.cuh"

__device__ unsigned long long mix64(unsigned long long z) {  // splitmix64 finaliser
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

// a double with a random significand and sign and an exponent in [-40, 40)
// (products and their low parts stay in the float normal range)
__device__ double rand_double(unsigned long long r) {
    const unsigned long long e = 1023ull - 40ull + ((r >> 53) % 80ull);
    const unsigned long long bits = (r & 0x800fffffffffffffull) | (e << 52);
    return __longlong_as_double((long long)bits);
}

__device__ double ffd(pitn::ff v) { return (double)v.hi + (double)v.lo; }

// counts[0]: splits whose hi is not the double rounded to float (ties aside)
// counts[1]: splits with |x - (hi + lo)| > 2^-47 |x|
// counts[2]: splits with |lo| > ulp(hi) (not normalised)
// counts[3]: sums with |ff_add - (a + b)| > 2^-44 (|a| + |b|)
// counts[4]: products with |ff_mul - a b| > 2^-44 |a b|
// counts[5]: values checked
// counts[6]: special values whose split differs from the expected one
__global__ void check(long long n, unsigned long long* counts) {
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid == 0) {
        const double sp[] = {0.0, -0.0, 1.0, -1.0, 2.0, 0.1, -1e-4, 1e30, 1e-30, 3.0e38,
                             INFINITY, -INFINITY};
        for (double x : sp) {
            const pitn::ff v = pitn::ff_from_double(x);
            const bool ok = (v.hi == __double2float_rn(x) || (isinf(x) && isinf(v.hi))) &&
                            (isinf(x) ? v.lo == 0.f : fabs(x - ffd(v)) <= ldexp(fabs(x), -47));
            if (!ok) atomicAdd(counts + 6, 1ull);
        }
        const pitn::ff nv = pitn::ff_from_double(NAN);
        if (!isnan(nv.hi)) atomicAdd(counts + 6, 1ull);
    }
    for (long long i = tid; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double x = rand_double(mix64(3 * (unsigned long long)i));
        const double y = rand_double(mix64(3 * (unsigned long long)i + 1));
        const pitn::ff a = pitn::ff_from_double(x), b = pitn::ff_from_double(y);
        const float hw = __double2float_rn(x);
        const double rem = x - (double)hw;
        const bool tie = fabs(rem) == ldexp(fabs((double)hw), -24);
        if (a.hi != hw && !tie) atomicAdd(counts + 0, 1ull);
        if (fabs(x - ffd(a)) > ldexp(fabs(x), -47)) atomicAdd(counts + 1, 1ull);
        if (fabsf(a.lo) > ldexpf(fabsf(a.hi), -23)) atomicAdd(counts + 2, 1ull);
        const double ad = ffd(a), bd = ffd(b);
        const pitn::ff s = pitn::ff_add(a, b);
        if (fabs(ffd(s) - (ad + bd)) > ldexp(fabs(ad) + fabs(bd), -44)) atomicAdd(counts + 3, 1ull);
        const pitn::ff p = pitn::ff_mul(a, b);
        if (fabs(ffd(p) - ad * bd) > ldexp(fabs(ad * bd), -44)) atomicAdd(counts + 4, 1ull);
        atomicAdd(counts + 5, 1ull);
    }
}

int main() {
    unsigned long long* d = nullptr;
    if (cudaMalloc(&d, 8 * sizeof(unsigned long long)) != cudaSuccess) return 2;
    cudaMemset(d, 0, 8 * sizeof(unsigned long long));
    check<<<1024, 256>>>(1ll << 22, d);
    unsigned long long h[8] = {};
    if (cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) return 3;
    printf("split_hi_bad %llu split_err %llu split_unnorm %llu add_bad %llu mul_bad %llu checked %llu "
           "special_bad %llu\n", h[0], h[1], h[2], h[3], h[4], h[5], h[6]);
    cudaFree(d);
    return 0;
}
