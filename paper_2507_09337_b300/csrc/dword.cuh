// dword.cuh -- double-word ("float-float") arithmetic for the FF hydro task.
//
// A value is the unevaluated sum hi + lo of two binary32 numbers with
// |lo| <= ulp(hi)/2: about 48 significant bits, computed on the FP32 pipe
// (71 times the FP64 rate on this GPU) instead of the FP64 pipe. The
// building blocks are the error-free transforms 2Sum (Knuth), Fast2Sum
// (Dekker) and the FMA-based 2Prod; the double-word sum and product are the
// classic constructions analysed by Joldes, Muller and Popescu ("Tight and
// rigorous error bounds for basic building blocks of double-word
// arithmetic", ACM TOMS 44, 2017), and the reciprocal and reciprocal square
// root are one Newton correction, carried in double-word, of the hardware
// approximations. With u = 2^-24:
//   x + y  2Sum of the high parts, low parts added, renormalised by
//          Fast2Sum; error at most about 5u^2 (|x| + |y|) (relative to the
//          operands, as an FP64 sum's error is relative to its rounded
//          operands)
//   x * y  2Prod of the high parts plus the cross terms; relative <= 7u^2
//   1 / y, rsqrt(y): relative error of a few u^2
// (measured maxima on 2^26 random operands: 2.8, 4.6, 3.0 and 4.5 u^2).
// Every operation uses the _rn intrinsics, so no step is contracted or
// reordered by the compiler. Checked on the GPU against FP64 references by
// orcha_selftest_dword.
#pragma once

#include <cuda_runtime.h>

namespace orcha {

struct __align__(8) dw {
    float hi, lo;
};

namespace dwx {
// s + t = a + b exactly (any a, b)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& t) {
    s = __fadd_rn(a, b);
    const float ap = __fsub_rn(s, b);
    const float bp = __fsub_rn(s, ap);
    t = __fadd_rn(__fsub_rn(a, ap), __fsub_rn(b, bp));
}
// s + t = a + b exactly when |a| >= |b| (or a = 0)
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& t) {
    s = __fadd_rn(a, b);
    t = __fsub_rn(b, __fsub_rn(s, a));
}
}  // namespace dwx

// Sum: 2Sum of the high parts, the low parts added to its error, and the
// result renormalised by Fast2Sum (11 FP32 additions). When the high parts
// cancel so far that |w| > |sh|, Fast2Sum may be off by about u |w|, within
// the same O(u^2 (|x| + |y|)) as the rounding of the low parts.
__device__ __forceinline__ dw operator+(dw x, dw y) {
    float sh, sl;
    dwx::two_sum(x.hi, y.hi, sh, sl);
    const float w = __fadd_rn(sl, __fadd_rn(x.lo, y.lo));
    dw z;
    dwx::fast_two_sum(sh, w, z.hi, z.lo);
    return z;
}
__device__ __forceinline__ dw operator-(dw x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ dw operator-(dw x, dw y) { return x + (-y); }
// The product is returned as the pair (ch, cl) before the final Fast2Sum:
// the same value (Fast2Sum is exact) with |cl| <= ~2u |ch| instead of
// u |ch|. Every consumer accepts that: sums and products use the low part
// only in rounded terms, the reciprocal and rsqrt fold it into their
// residual, the conversion to binary64 is still exact, and a sign test reads
// the high part, whose sign is the value's. Comparisons (dw_lt) are only
// applied to sums, which are normalised.
__device__ __forceinline__ dw operator*(dw x, dw y) {
    const float ch = __fmul_rn(x.hi, y.hi);
    const float cl1 = __fmaf_rn(x.hi, y.hi, -ch);            // x.hi * y.hi = ch + cl1 exactly
    const float cl2 = __fmaf_rn(x.lo, y.hi, __fmul_rn(x.hi, y.lo));
    return {ch, __fadd_rn(cl1, cl2)};
}

// 1 / y: r1 = the hardware reciprocal of y.hi refined by one FP32 Newton
// step (within about an ulp), e = 1 - y r1 by FMAs, then
// 1/y = r1 (1 + e + e^2 + ...) with the correction carried as the low part.
__device__ __forceinline__ dw dw_rcp(dw y) {
    const float r0 = __fdividef(1.0f, y.hi);
    const float r1 = __fmaf_rn(r0, __fmaf_rn(-y.hi, r0, 1.0f), r0);
    float e = __fmaf_rn(-y.hi, r1, 1.0f);
    e = __fmaf_rn(-y.lo, r1, e);
    dw z;
    dwx::fast_two_sum(r1, __fmul_rn(r1, __fmaf_rn(e, e, e)), z.hi, z.lo);
    return z;
}

// 1 / sqrt(y), y > 0: r1 = the hardware rsqrt of y.hi refined by one FP32
// Newton step, e = 1 - y r1^2 (r1^2 exact by 2Prod), then
// y^(-1/2) = r1 (1 + e/2 + 3e^2/8 + ...).
__device__ __forceinline__ dw dw_rsqrt(dw y) {
    const float r0 = rsqrtf(y.hi);
    const float e0 = __fmaf_rn(-__fmul_rn(y.hi, r0), r0, 1.0f);
    const float r1 = __fmaf_rn(__fmul_rn(0.5f, r0), e0, r0);
    const float qh = __fmul_rn(r1, r1);
    const float ql = __fmaf_rn(r1, r1, -qh);
    float e = __fmaf_rn(-y.hi, qh, 1.0f);
    e = __fmaf_rn(-y.hi, ql, e);
    e = __fmaf_rn(-y.lo, qh, e);
    const float h = __fmul_rn(0.5f, e);
    const float t = __fmaf_rn(__fmul_rn(0.75f, e), h, h);    // e/2 + 3e^2/8
    dw z;
    dwx::fast_two_sum(r1, __fmul_rn(r1, t), z.hi, z.lo);
    return z;
}

// Totally ordered comparison of normalised double-words.
__device__ __forceinline__ bool dw_lt(dw a, dw b) { return (a.hi < b.hi) | ((a.hi == b.hi) & (a.lo < b.lo)); }

}  // namespace orcha
