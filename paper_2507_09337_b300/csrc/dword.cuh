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
__device__ __forceinline__ bool dw_lt(dw a, dw b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }

// ---------------------------------------------------------------- two double-words per instruction
// dw2 carries two independent double-words in the x and y lanes of float2
// pairs. Each operation is the dw operation above applied to both lanes with
// the packed FP32x2 instructions (add / mul / fma .f32x2, round to nearest
// even per lane, never contracted), so every lane gets the same bits as the
// scalar operation while one instruction issue does the work of two.
struct dw2 {
    float2 hi, lo;
};

namespace dwx {
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, neg2(b)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 splat2(float a) { return make_float2(a, a); }
}  // namespace dwx

__device__ __forceinline__ dw2 pack2(dw a, dw b) { return {make_float2(a.hi, b.hi), make_float2(a.lo, b.lo)}; }
__device__ __forceinline__ dw lane_x(dw2 a) { return {a.hi.x, a.lo.x}; }
__device__ __forceinline__ dw lane_y(dw2 a) { return {a.hi.y, a.lo.y}; }

__device__ __forceinline__ dw2 operator+(dw2 x, dw2 y) {
    using namespace dwx;
    const float2 sh = add2(x.hi, y.hi);                   // 2Sum of the high parts
    const float2 ap = sub2(sh, y.hi);
    const float2 bp = sub2(sh, ap);
    const float2 sl = add2(sub2(x.hi, ap), sub2(y.hi, bp));
    const float2 w = add2(sl, add2(x.lo, y.lo));
    const float2 zh = add2(sh, w);                        // Fast2Sum
    return {zh, sub2(w, sub2(zh, sh))};
}
__device__ __forceinline__ dw2 operator-(dw2 x) { return {dwx::neg2(x.hi), dwx::neg2(x.lo)}; }
__device__ __forceinline__ dw2 operator-(dw2 x, dw2 y) { return x + (-y); }
__device__ __forceinline__ dw2 operator*(dw2 x, dw2 y) {
    using namespace dwx;
    const float2 ch = mul2(x.hi, y.hi);
    const float2 cl1 = fma2(x.hi, y.hi, neg2(ch));
    const float2 cl2 = fma2(x.lo, y.hi, mul2(x.hi, y.lo));
    return {ch, add2(cl1, cl2)};
}
__device__ __forceinline__ dw2 dw2_rsqrt(dw2 y) {
    using namespace dwx;
    const float2 r0 = make_float2(rsqrtf(y.hi.x), rsqrtf(y.hi.y));
    const float2 e0 = fma2(neg2(mul2(y.hi, r0)), r0, splat2(1.0f));
    const float2 r1 = fma2(mul2(splat2(0.5f), r0), e0, r0);
    const float2 qh = mul2(r1, r1);
    const float2 ql = fma2(r1, r1, neg2(qh));
    float2 e = fma2(neg2(y.hi), qh, splat2(1.0f));
    e = fma2(neg2(y.hi), ql, e);
    e = fma2(neg2(y.lo), qh, e);
    const float2 h = mul2(splat2(0.5f), e);
    const float2 t = fma2(mul2(splat2(0.75f), e), h, h);
    const float2 p = mul2(r1, t);
    const float2 zh = add2(r1, p);
    return {zh, sub2(p, sub2(zh, r1))};
}
// x * rsqrt(x * rho) per lane, 0 where x <= 0 (the other lane's value is
// kept; a lane with x <= 0 computes a discarded NaN).
__device__ __forceinline__ dw2 dw2_sound(dw2 x, dw2 rho) {
    dw2 c = x * dw2_rsqrt(x * rho);
    if (!(x.hi.x > 0.0f)) { c.hi.x = 0.0f; c.lo.x = 0.0f; }
    if (!(x.hi.y > 0.0f)) { c.hi.y = 0.0f; c.lo.y = 0.0f; }
    return c;
}

}  // namespace orcha
