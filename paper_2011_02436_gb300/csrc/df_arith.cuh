// Double-float helpers shared by the factorisation and the refinement
// kernels: a value v = h + l held as two floats in eight bytes, integer-only
// conversions from and to FP64, and the error-free transformations of
// Dekker (TwoProduct by FMA, FastTwoSum) and Knuth (TwoSum).  About 2^-44
// relative; everything runs on the FP32 and integer pipes.
#pragma once
#include <stdint.h>

namespace elm {
namespace df {

// Storage of the active matrix in the mixed form: v = h + l, two floats in
// the eight bytes of a double.  The conversions use integer moves only (an
// FP64 instruction costs a 64-cycle issue slot per SM sub-partition).
struct F2 {
    float h, l;
};
// h = v truncated to 24 significant bits, l = the remainder truncated to 24
// bits: |v - h - l| < 2^-47 |v| for |v| >= 2^-70; magnitudes below 2^-126
// (and the part of l below it) are dropped.
__device__ __forceinline__ F2 d2df(double v) {
    const uint64_t b = (uint64_t)__double_as_longlong(v);
    const uint32_t sgn = (uint32_t)(b >> 63) << 31;
    const int e = (int)((b >> 52) & 0x7ff) - 1023;
    F2 r{0.f, 0.f};
    if (e < -126) return r;
    r.h = __uint_as_float(sgn | ((uint32_t)(e + 127) << 23) | (uint32_t)((b >> 29) & 0x7fffff));
    const uint64_t m = b & 0x1fffffffull;   // the low 29 mantissa bits
    if (m == 0) return r;
    const int top = 63 - __clzll((long long)m);
    const int el = e - 52 + top;
    if (el < -126) return r;
    const uint32_t mant = top >= 23 ? (uint32_t)(m >> (top - 23)) & 0x7fffff
                                    : (uint32_t)(m << (23 - top)) & 0x7fffff;
    r.l = __uint_as_float(sgn | ((uint32_t)(el + 127) << 23) | mant);
    return r;
}
// exact value of a normal float (or zero) as a double
__device__ __forceinline__ double f2d(float x) {
    const uint32_t b = __float_as_uint(x);
    const uint32_t ef = (b >> 23) & 0xff;
    if (ef == 0) return 0.0;
    return __longlong_as_double((long long)(((uint64_t)(b >> 31) << 63) |
                                            ((uint64_t)(ef - 127 + 1023) << 52) |
                                            ((uint64_t)(b & 0x7fffff) << 29)));
}

// Double-float arithmetic (Knuth's TwoSum, Dekker's FastTwoSum, TwoProduct
// by FMA): about 2^-44 relative, all on the FP32 pipes.
__device__ __forceinline__ F2 df_renorm(float s, float e) {   // |s| >= |e|
    const float h = s + e;
    return F2{h, e - (h - s)};
}
__device__ __forceinline__ F2 df_add(F2 a, F2 b) {
    const float s = a.h + b.h;
    const float bb = s - a.h;
    const float e = ((a.h - (s - bb)) + (b.h - bb)) + (a.l + b.l);
    return df_renorm(s, e);
}
__device__ __forceinline__ F2 df_neg(F2 a) { return F2{-a.h, -a.l}; }
__device__ __forceinline__ F2 df_mul(F2 a, F2 b) {
    const float p = a.h * b.h;
    float e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, e);
    e = fmaf(a.l, b.h, e);
    return df_renorm(p, e);
}
// (sh, sl) += a b, left unnormalised (renormalise after a run of terms)
__device__ __forceinline__ void df_acc_prod(float &sh, float &sl, F2 a, F2 b) {
    const float p = a.h * b.h;
    float e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, e);
    e = fmaf(a.l, b.h, e);
    const float s = sh + p;
    const float bb = s - sh;
    sl += ((sh - (s - bb)) + (p - bb)) + e;
    sh = s;
}

}  // namespace df
}  // namespace elm
