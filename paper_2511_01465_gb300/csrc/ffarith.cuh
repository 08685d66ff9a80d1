// ffarith.cuh -- double-FP32 ("float-float") arithmetic for the small-state
// scan: a value is an unevaluated sum hi + lo of two floats with
// |lo| <= ulp(hi) / 2, a 48-bit significand carried on the FP32 pipe.
//
// On GB300 the FP32 pipe issues about 60 times faster than the FP64 pipe, so
// a scan in float-float costs less FP64-pipe time than one in FP64 while
// keeping a relative precision of about 2^-47 (against 2^-53 for FP64).  The
// operations follow the published error-free transformations: Knuth's
// TwoSum, Dekker's FastTwoSum (renormalisation) and the FMA-based exact
// product, composed as in Dekker's double-length arithmetic and the
// double-single libraries built on it.  Every operation uses the _rn
// intrinsics, which the compiler never contracts into FMAs or reorders: an
// error-free transformation depends on each rounding step happening as
// written.
//
// Conversions from FP64 run on the integer pipes (as in fpconv.cuh): hi is
// the double rounded to 24 bits, lo the remainder rounded to 24 bits, built
// from the bit pattern, so that a conversion puts no work on the FP64 pipe.
// Remainders far below the float range flush to zero (this arithmetic serves
// only the scan of the Newton step, an inexact linear solve).
#pragma once

#include "fpconv.cuh"

namespace pitn {

struct __align__(8) ff {
    float hi, lo;
};

// s + e = a + b exactly (Knuth's TwoSum, six operations)
__device__ __forceinline__ ff ff_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return ff{s, e};
}

// s + e = a + b exactly when |a| >= |b| or a = 0 (Dekker's FastTwoSum)
__device__ __forceinline__ ff ff_fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return ff{s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ ff ff_add(ff a, ff b) {
    const ff s = ff_two_sum(a.hi, b.hi);
    const float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return ff_fast_two_sum(s.hi, e);
}

__device__ __forceinline__ ff ff_neg(ff a) { return ff{-a.hi, -a.lo}; }

__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }

// a * b: the exact product of the high parts by one FMA, the cross terms
// added to its error, renormalised
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return ff_fast_two_sum(p, e);
}

// a * b + c
__device__ __forceinline__ ff ff_fma(ff a, ff b, ff c) { return ff_add(ff_mul(a, b), c); }

__device__ __forceinline__ ff ff_zero() { return ff{0.f, 0.f}; }
__device__ __forceinline__ ff ff_one() { return ff{1.f, 0.f}; }

__device__ __forceinline__ ff ff_shfl_up(ff v, int off) {
    return ff{__shfl_up_sync(0xffffffffu, v.hi, off), __shfl_up_sync(0xffffffffu, v.lo, off)};
}

// FP64 -> float-float on the integer pipes.  With x = (-1)^s M 2^(E-52),
// M the 53-bit significand, hi = d2f_int(x) keeps the top 24 bits of M
// rounded (ties away), so x - hi = (-1)^s t 2^(E-52) with t the low 29 bits
// of M taken as a signed number (t >= 2^28 rounded up, leaving t - 2^29).
// lo = t converted to float (rounds to nearest even), scaled by 2^(E-52).
__device__ __forceinline__ ff ff_from_double(double x) {
    unsigned w0, w1;
    asm("mov.b64 {%0, %1}, %2;" : "=r"(w0), "=r"(w1) : "d"(x));
    const float hi = d2f_int(x);
    const int t = ((int)(w0 << 3)) >> 3;                   // low 29 bits, sign-extended
    const int eb = (int)((w1 >> 20) & 0x7ffu);             // biased exponent of x
    const int es = eb - 1023 - 52 + 127;                   // biased float exponent of 2^(E-52)
    const bool finite_hi = (__float_as_uint(hi) & 0x7f800000u) != 0x7f800000u;
    float lo = 0.f;
    if (eb != 0 && finite_hi && t != 0) {
        const float tf = __int2float_rn(t);
        if (es >= 1) {            // 2^(E-52) a normal float (es <= 254 whenever hi is finite)
            lo = __fmul_rn(tf, __uint_as_float((unsigned)es << 23));
        } else if (es >= -99) {   // two scalings: the remainder itself may still be normal
            lo = __fmul_rn(__fmul_rn(tf, __uint_as_float((unsigned)(es + 100) << 23)),
                           __uint_as_float(27u << 23));   // 2^-100
        }
        if (w1 & 0x80000000u) lo = -lo;
    }
    return ff{hi, lo};
}

// constants on the host or the device (hardware conversions; used once)
__host__ __device__ inline ff ff_const(double x) {
    const float hi = (float)x;
    return ff{hi, (float)(x - (double)hi)};
}

// x + (hi + lo) in FP64: the float parts widened on the integer pipes,
// two FP64 additions
__device__ __forceinline__ double ff_add_to_double(double x, ff v) {
    return (x + f2d_int(v.hi)) + f2d_int(v.lo);
}

}  // namespace pitn
