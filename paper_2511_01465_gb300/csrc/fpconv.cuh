// fpconv.cuh -- FP64 <-> FP32 conversions on the integer pipes.
//
// On GB300 a hardware F2F conversion to or from FP64 issues on the FP64
// pipe, which runs at 1/62 of the FP32 rate; in the mixed-precision scan it
// would cost as much as the FP64 residual it feeds.  These helpers build the
// other format's bit pattern with 32-bit integer operations instead, from
// the IEEE-754 binary64 / binary32 layouts:
//   binary64: sign 1 | exponent 11 (bias 1023) | fraction 52
//   binary32: sign 1 | exponent  8 (bias  127) | fraction 23
// They are used only where the scan's operands are already inexact (the
// FP32 delta-form scan), so subnormal results are flushed to signed zero.
#pragma once

namespace pitn {

// double -> float, round to nearest (ties away from zero on the 29 dropped
// fraction bits); magnitudes below the smallest normal float give signed
// zero, above the largest finite float +-inf; NaN stays NaN.
__device__ __forceinline__ float d2f_int(double x) {
    unsigned lo, hi;   // the register pair, split without any FP64 instruction
    asm("mov.b64 {%0, %1}, %2;" : "=r"(lo), "=r"(hi) : "d"(x));
    const unsigned s = hi & 0x80000000u;
    const unsigned ea = (hi >> 20) & 0x7ffu;                // biased binary64 exponent
    // add half an ulp of the result at bit 28; a carry out of the fraction
    // moves into the exponent field, which is the correctly rounded result
    const unsigned long long rb = ((unsigned long long)(hi & 0x7fffffffu) << 32 | lo) + (1ull << 28);
    const unsigned rhi = (unsigned)(rb >> 32), rlo = (unsigned)rb;
    const int e = (int)((rhi >> 20) & 0x7ffu) - 1023 + 127;  // rebiased exponent after rounding
    const unsigned frac = ((rhi & 0xfffffu) << 3) | (rlo >> 29);
    unsigned f = s | ((unsigned)e << 23) | frac;
    f = (e <= 0) ? s : f;                                   // underflow: signed zero
    f = (e >= 255) ? (s | 0x7f800000u) : f;                 // overflow: infinity
    const bool nan = ea == 0x7ffu && ((hi & 0xfffffu) | lo) != 0u;
    f = nan ? (s | 0x7fc00000u) : f;                        // NaN stays NaN (inf handled above)
    return __uint_as_float(f);
}

// float -> double, exact for normal numbers; subnormal floats give signed
// zero; infinities and NaN keep their class.
__device__ __forceinline__ double f2d_int(float v) {
    const unsigned f = __float_as_uint(v);
    const unsigned s = f & 0x80000000u;
    const unsigned e = (f >> 23) & 0xffu;
    const unsigned m = f & 0x7fffffu;
    unsigned hi = s | ((e + 896u) << 20) | (m >> 3);        // 896 = 1023 - 127
    unsigned lo = m << 29;
    hi = (e == 0u) ? s : hi;
    lo = (e == 0u) ? 0u : lo;
    hi = (e == 0xffu) ? (s | 0x7ff00000u | (m >> 3)) : hi;
    double r;
    asm("mov.b64 %0, {%1, %2};" : "=d"(r) : "r"(lo), "r"(hi));
    return r;
}

}  // namespace pitn
