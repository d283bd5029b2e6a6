// common.cuh -- device-side types shared by the block-hydro kernels.
//
// Arithmetic contract of the FP64 path (type rd). Default build
// (ORCHA_FP64_CONTRACT = 1): a product a * b written directly as an operand
// of a sum or difference is fused into it (one FMA, the product unrounded);
// every other operation is one round-to-nearest operation that the compiler
// may not contract. Where products are fused is thus fixed by the source
// expressions, so every kernel instantiation (tile shape, launch bounds,
// packet or persistent path) gives the same bits. Two more rewrites need
// fewer FP64-pipe slots (the HLL sound speed as x * rsqrt(x * rho), the
// predictor as an FMA chain). The result differs from the unfused definition
// by rounding only (a few ulp per step). Exact build (ORCHA_FP64_CONTRACT =
// 0): every operation is one round-to-nearest operation, none fused or
// reordered, so the kernels evaluate the definition's expression trees and
// reproduce an unfused CPU evaluation of them bit for bit. The FP32 flux path
// uses plain float, where contraction is allowed.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace orcha {

constexpr int kGuard = 2;   // guard layers per side: the scheme's stencil reaches two cells

// ---------------------------------------------------------------- FP64: fused only where written
struct rdp;
struct rd {
    double v;
    __device__ __forceinline__ rd() {}
    __device__ __forceinline__ constexpr rd(double x) : v(x) {}
    __device__ __forceinline__ rd(const rdp& p);
};
#ifndef ORCHA_FP64_CONTRACT
#define ORCHA_FP64_CONTRACT 1
#endif
constexpr bool kContract = ORCHA_FP64_CONTRACT != 0;
// The product a * b not yet rounded (default build): a sum or difference that
// takes it as an operand is one FMA; any other use rounds it first. With two
// products as operands the left one is fused and the right one rounded.
struct rdp {
    double a, b;
};
__device__ __forceinline__ rd::rd(const rdp& p) { v = __dmul_rn(p.a, p.b); }
#if ORCHA_FP64_CONTRACT
__device__ __forceinline__ rd operator+(rd a, rd b) { return rd(__dadd_rn(a.v, b.v)); }
__device__ __forceinline__ rd operator-(rd a, rd b) { return rd(__dsub_rn(a.v, b.v)); }
__device__ __forceinline__ rdp operator*(rd a, rd b) { return rdp{a.v, b.v}; }
__device__ __forceinline__ rd operator+(rdp p, rd c) { return rd(fma(p.a, p.b, c.v)); }
__device__ __forceinline__ rd operator+(rd c, rdp p) { return rd(fma(p.a, p.b, c.v)); }
__device__ __forceinline__ rd operator-(rdp p, rd c) { return rd(fma(p.a, p.b, -c.v)); }
__device__ __forceinline__ rd operator-(rd c, rdp p) { return rd(fma(-p.a, p.b, c.v)); }
__device__ __forceinline__ rd operator+(rdp p, rdp q) { return rd(fma(p.a, p.b, __dmul_rn(q.a, q.b))); }
__device__ __forceinline__ rd operator-(rdp p, rdp q) { return rd(fma(p.a, p.b, -__dmul_rn(q.a, q.b))); }
#else
__device__ __forceinline__ rd operator+(rd a, rd b) { return rd(__dadd_rn(a.v, b.v)); }
__device__ __forceinline__ rd operator-(rd a, rd b) { return rd(__dsub_rn(a.v, b.v)); }
__device__ __forceinline__ rd operator*(rd a, rd b) { return rd(__dmul_rn(a.v, b.v)); }
#endif
__device__ __forceinline__ rd operator-(rd a) { return rd(-a.v); }
__device__ __forceinline__ bool operator<(rd a, rd b) { return a.v < b.v; }
__device__ __forceinline__ bool operator>(rd a, rd b) { return a.v > b.v; }
__device__ __forceinline__ bool operator<=(rd a, rd b) { return a.v <= b.v; }
__device__ __forceinline__ bool operator>=(rd a, rd b) { return a.v >= b.v; }

// Precision traits: storage type, conversions, reciprocal, square root and
// the sign tests the scheme uses. For rd every function is the correctly
// rounded IEEE operation (1/x by __drcp_rn equals the IEEE quotient 1.0/x).
template <class T> struct P;

// FP64 sign tests, selects and exact halvings are done on the IEEE bit
// patterns with integer instructions: on this GPU every FP64 compare,
// min/max and multiply issues on the FP64 pipe, the scarcest unit, while the
// integer forms below give bitwise the same answers (NaN never reaches them
// on a physical state; the non-physical checks run on finite values).
__device__ __forceinline__ long long bits(rd x) { return __double_as_longlong(x.v); }

template <> struct P<rd> {
    using store = double;
    static __device__ __forceinline__ rd in(double x) { return rd(x); }
    static __device__ __forceinline__ double out(rd x) { return x.v; }
    static __device__ __forceinline__ rd rcp(rd x) { return rd(__drcp_rn(x.v)); }
    static __device__ __forceinline__ rd sqrt(rd x) { return rd(__dsqrt_rn(x.v)); }
    // sqrt(x / rho) for x = gamma * p: the definition's sqrt(x * (1/rho)), or in
    // the contracted build x * rsqrt(x * rho) (one reciprocal square root
    // instead of a reciprocal and a square root; rsqrt is within 1 ulp), left
    // as an unrounded product so that each wave speed u -+ c is one FMA.
    static __device__ __forceinline__ auto sound(rd x, rd rho) {
        if constexpr (kContract) return rdp{x.v, ::rsqrt(__dmul_rn(x.v, rho.v))};
        else return rd(__dsqrt_rn(__dmul_rn(x.v, __drcp_rn(rho.v))));
    }
    static __device__ __forceinline__ rd ld(const double* p) { return rd(*p); }
    static __device__ __forceinline__ void st(double* p, rd x) { *p = x.v; }
    // x > 0 (false for +-0 and NaN; true for +inf)
    static __device__ __forceinline__ bool pos(rd x) {
        const long long b = bits(x);
        return b > 0 && b <= 0x7FF0000000000000LL;
    }
    // x < 0 (false for +-0 and NaN; true for -inf)
    static __device__ __forceinline__ bool neg(rd x) {
        const unsigned long long b = (unsigned long long)bits(x);
        return b > 0x8000000000000000ULL && b <= 0xFFF0000000000000ULL;
    }
    // a < b for non-NaN values, except that -0 < +0 here (the bit pattern
    // with the magnitude bits of a negative number flipped is a signed
    // integer key in value order): the HLL wave speeds, its only use, can
    // then differ from those of a value comparison at most in the sign of a
    // zero, which ge0 and le0 do not see, so every flux has the same bits.
    static __device__ __forceinline__ bool lt(rd a, rd b) {
        const long long ba = bits(a), bb = bits(b);
        return (ba ^ (long long)((unsigned long long)(ba >> 63) >> 1)) <
               (bb ^ (long long)((unsigned long long)(bb >> 63) >> 1));
    }
    // a >= 0 and a <= 0 with -0 == +0 (sign clear or -0; sign set or +0),
    // from the high word
    static __device__ __forceinline__ bool ge0(rd a) {
        const unsigned hi = (unsigned)__double2hiint(a.v);
        return (int)hi >= 0 || ((hi & 0x7FFFFFFFu) | (unsigned)__double2loint(a.v)) == 0u;
    }
    static __device__ __forceinline__ bool le0(rd a) {
        const unsigned hi = (unsigned)__double2hiint(a.v);
        return (int)hi < 0 || (hi | (unsigned)__double2loint(a.v)) == 0u;
    }
    // minmod: same strict sign -> the argument of smaller magnitude, else +0
    static __device__ __forceinline__ rd minmod(rd a, rd b) {
        const long long ba = bits(a), bb = bits(b);
        const long long ma = ba & 0x7FFFFFFFFFFFFFFFLL, mb = bb & 0x7FFFFFFFFFFFFFFFLL;
        const bool ok = ((ba ^ bb) >= 0) && ma != 0 && mb != 0 && ma <= 0x7FF0000000000000LL &&
                        mb <= 0x7FF0000000000000LL;
        return ok ? (ma < mb ? a : b) : rd(0.0);
    }
    // 0.5 * x, entirely on the integer pipe (a fallback multiply would be
    // predicated into every call): exponent decrement when the result is
    // normal; infinities and NaN unchanged; otherwise the result is in the
    // subnormal range and is the magnitude bits shifted right by one with the
    // dropped bit rounded to nearest even (the IEEE result bit for bit).
    static __device__ __forceinline__ rd half(rd x) {
        // the common case (a normal result): one decrement of the exponent
        // field in the high word
        const unsigned hi = (unsigned)__double2hiint(x.v);
        if (((hi >> 20) & 0x7FFu) - 2u <= 0x7FCu)
            return rd(__hiloint2double((int)(hi - 0x00100000u), __double2loint(x.v)));
        const unsigned long long b = (unsigned long long)bits(x);
        const unsigned long long sign = b & 0x8000000000000000ull, a = b & 0x7FFFFFFFFFFFFFFFull;
        const unsigned e = (unsigned)(a >> 52);
        unsigned long long r;
        if (e > 1u && e < 0x7FFu) r = a - (1ull << 52);
        else if (e == 0x7FFu) r = a;
        else r = (a >> 1) + ((a & 1ull) & ((a >> 1) & 1ull));
        return rd(__longlong_as_double((long long)(sign | r)));
    }
    static __device__ __forceinline__ rd zero() { return rd(0.0); }
    static __device__ __forceinline__ double to_double(rd x) { return x.v; }
};

// ---------------------------------------------------------------- IEEE-754 format conversions on the integer pipe
// Written from the binary64/binary32 layouts (sign | biased exponent |
// fraction), entirely in integer arithmetic -- including zeros, subnormals,
// overflow, infinities and NaN -- so no conversion instruction issues on the
// FP64 pipe (even a predicated-off one). Bitwise equal to the hardware
// conversions (NaN payloads aside); checked on the GPU by
// orcha_selftest_conversions.

// binary64 -> binary32, round to nearest, ties to even; every case.
__device__ __forceinline__ float d2f_any(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned long long a = b & 0x7FFFFFFFFFFFFFFFull;
    const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
    const int e = (int)(a >> 52);                        // biased binary64 exponent
    const unsigned long long m = a & 0xFFFFFFFFFFFFFull;
    unsigned r;
    if (e >= 897 && e <= 1150) {                         // normal binary32 result (or overflow by rounding)
        r = ((unsigned)(e - 896) << 23) | (unsigned)(m >> 29);
        const unsigned rem = (unsigned)(m & 0x1FFFFFFFull);          // the 29 dropped fraction bits
        r += (rem > 0x10000000u) || (rem == 0x10000000u && (r & 1u));  // a carry may reach the exponent
    } else if (e > 1150) {                               // overflow to infinity, or inf / NaN
        r = 0x7F800000u | ((e == 2047 && m) ? (0x00400000u | (unsigned)(m >> 29)) : 0u);
    } else if (e == 0 && m == 0) {                       // zero
        r = 0u;
    } else {                                             // subnormal binary32 result (units of 2^-149)
        const unsigned long long full = (e ? (1ull << 52) : 0ull) | m;
        const int shift = (e ? 926 - e : 925);           // value = full * 2^(shift_base) -> units of 2^-149
        if (shift >= 64) {
            r = 0u;
        } else {
            r = (unsigned)(full >> shift);
            const unsigned long long rem = full & ((1ull << shift) - 1ull), half = 1ull << (shift - 1);
            r += (rem > half) || (rem == half && (r & 1u));
        }
    }
    return __uint_as_float(sign | r);
}

// binary32 -> binary64 (exact), every case.
__device__ __forceinline__ double f2d_any(float x) {
    const unsigned b = __float_as_uint(x);
    const unsigned a = b & 0x7FFFFFFFu;
    const unsigned long long sign = (unsigned long long)(b & 0x80000000u) << 32;
    unsigned long long r;
    if (a >= 0x00800000u && a < 0x7F800000u) {          // normal: rebias 127 -> 1023
        r = ((unsigned long long)a + (896ull << 23)) << 29;
    } else if (a >= 0x7F800000u) {                      // inf / NaN
        r = 0x7FF0000000000000ull | ((unsigned long long)(a & 0x007FFFFFu) << 29) |
            ((a & 0x007FFFFFu) ? 0x0008000000000000ull : 0ull);
    } else if (a == 0u) {
        r = 0ull;
    } else {                                            // subnormal: a * 2^-149, normalise
        const int p = 31 - __clz((int)a);               // leading bit, 0..22
        r = ((unsigned long long)(p - 149 + 1023) << 52) | (((unsigned long long)a << (52 - p)) & 0xFFFFFFFFFFFFFull);
    }
    return __longlong_as_double((long long)(sign | r));
}

// binary64 -> binary32, round to nearest, ties to even: a normal binary32
// result (or an overflow by rounding) in a few integer instructions -- the
// top 23 fraction bits and the exponent rebiased by 896 (its 9 low bits plus
// 128, mod 512, for biased exponents 897 .. 1150), plus one unit where the 29
// dropped bits exceed half a unit or equal it with an odd result -- zeros
// directly, and the rest (subnormal results, overflow, infinities, NaN) by
// the general form behind a branch.
__device__ __forceinline__ float d2f_rn(double x) {
    const unsigned lo = (unsigned)__double2loint(x), hi = (unsigned)__double2hiint(x);
    const unsigned a = hi & 0x7FFFFFFFu;
    if ((a >> 20) - 897u <= 253u) {
        unsigned r = __funnelshift_l(lo, a, 3) + 0x40000000u;
        const unsigned rem = lo & 0x1FFFFFFFu;
        r += (rem > 0x10000000u || (rem == 0x10000000u && (r & 1u))) ? 1u : 0u;
        return __uint_as_float(r | (hi & 0x80000000u));
    }
    if ((a | lo) == 0u) return __uint_as_float(hi & 0x80000000u);
    return d2f_any(x);
}

// binary32 -> binary64 (exact): normal numbers and zeros in a few integer
// instructions -- the high word is the sign, the exponent rebiased by
// 1023 - 127 = 896 and the top 20 fraction bits, the low word the last 3
// fraction bits -- and the rare subnormals, infinities and NaNs by the
// general form behind a branch.
__device__ __forceinline__ double f2d(float x) {
    const unsigned b = __float_as_uint(x);
    const unsigned a = b & 0x7FFFFFFFu;
    if (a - 0x00800000u < 0x7F000000u || a == 0u) {
        const unsigned hi = (b & 0x80000000u) | (a ? (a >> 3) + (896u << 20) : 0u);
        return __hiloint2double((int)hi, (int)(a << 29));
    }
    return f2d_any(x);
}

// Which conversions the FP32-flux path issues, per direction: the
// integer-pipe forms above (1) or the hardware conversions (0). All are
// exact, so results do not depend on the choice; it balances FP64-pipe
// slots (one per hardware conversion) against integer instructions (about
// 8 per narrowing and 5 per widening on their fast paths). Measured on a
// B300 (C2 set-up): widening on the integer pipe is faster (the FP64 pipe
// carries the configured arithmetic's update), narrowing there is slower
// (FP32 flux 6.61 against 6.72 G, the shortcut 7.6 against 9.1 G).
#ifndef ORCHA_D2F_ON_INT_PIPE
#define ORCHA_D2F_ON_INT_PIPE 0
#endif
#ifndef ORCHA_F2D_ON_INT_PIPE
#define ORCHA_F2D_ON_INT_PIPE 1
#endif

__device__ __forceinline__ float to_f32(double x) {
#if ORCHA_D2F_ON_INT_PIPE
    return d2f_rn(x);
#else
    return __double2float_rn(x);
#endif
}

__device__ __forceinline__ double to_f64(float x) {
#if ORCHA_F2D_ON_INT_PIPE
    return f2d(x);
#else
    return (double)x;
#endif
}

// ---------------------------------------------------------------- FP64 on the integer pipe
// Same values as rd (IEEE round-to-nearest-even, never fused), computed by
// integer instructions (softfp64.cuh): the FP64 task moves a share of its
// adds and multiplies here to balance the FP64 pipe against the idle
// integer pipe.
struct re {
    double v;
    __device__ __forceinline__ re() {}
    __device__ __forceinline__ constexpr re(double x) : v(x) {}
};
}  // namespace orcha
#include "softfp64.cuh"
namespace orcha {
__device__ __forceinline__ re operator+(re a, re b) { return re(em_add(a.v, b.v)); }
__device__ __forceinline__ re operator-(re a, re b) { return re(em_sub(a.v, b.v)); }
__device__ __forceinline__ re operator*(re a, re b) { return re(em_mul(a.v, b.v)); }
__device__ __forceinline__ re operator-(re a) { return re(-a.v); }

template <> struct P<re> {
    using store = double;
    static __device__ __forceinline__ re in(double x) { return re(x); }
    static __device__ __forceinline__ re rcp(re x) { return re(__drcp_rn(x.v)); }
    static __device__ __forceinline__ re sqrt(re x) { return re(__dsqrt_rn(x.v)); }
    static __device__ __forceinline__ re sound(re x, re rho) { return re(__dsqrt_rn(em_mul(x.v, __drcp_rn(rho.v)))); }
    static __device__ __forceinline__ bool pos(re x) { return P<rd>::pos(rd(x.v)); }
    static __device__ __forceinline__ bool neg(re x) { return P<rd>::neg(rd(x.v)); }
    static __device__ __forceinline__ bool lt(re a, re b) { return P<rd>::lt(rd(a.v), rd(b.v)); }
    static __device__ __forceinline__ bool ge0(re a) { return P<rd>::ge0(rd(a.v)); }
    static __device__ __forceinline__ bool le0(re a) { return P<rd>::le0(rd(a.v)); }
    static __device__ __forceinline__ re minmod(re a, re b) { return re(P<rd>::minmod(rd(a.v), rd(b.v)).v); }
    static __device__ __forceinline__ re half(re x) { return re(P<rd>::half(rd(x.v)).v); }
    static __device__ __forceinline__ re zero() { return re(0.0); }
};

// Value-preserving moves between the FP64 arithmetic types (free: both hold a double).
template <class A, class T> __device__ __forceinline__ A as(T x);
template <> __device__ __forceinline__ rd as<rd, rd>(rd x) { return x; }
template <> __device__ __forceinline__ re as<re, rd>(rd x) { return re(x.v); }
template <> __device__ __forceinline__ rd as<rd, re>(re x) { return rd(x.v); }
template <> __device__ __forceinline__ re as<re, re>(re x) { return x; }
template <> __device__ __forceinline__ float as<float, float>(float x) { return x; }

template <> struct P<float> {
    using store = float;
    static __device__ __forceinline__ float in(double x) { return to_f32(x); }
    static __device__ __forceinline__ float out(float x) { return x; }
    // hardware approximations (about 1 ulp): the FP32 flux path states its error against FP64
    static __device__ __forceinline__ float rcp(float x) { return __fdividef(1.0f, x); }
    static __device__ __forceinline__ float sqrt(float x) { return x > 0.0f ? x * rsqrtf(x) : 0.0f; }
    static __device__ __forceinline__ float sound(float x, float rho) { return x > 0.0f ? x * rsqrtf(x * rho) : 0.0f; }
    static __device__ __forceinline__ float ld(const float* p) { return *p; }
    static __device__ __forceinline__ void st(float* p, float x) { *p = x; }
    static __device__ __forceinline__ bool pos(float x) { return x > 0.0f; }
    static __device__ __forceinline__ bool neg(float x) { return x < 0.0f; }
    static __device__ __forceinline__ bool lt(float a, float b) { return a < b; }
    static __device__ __forceinline__ bool ge0(float a) { return a >= 0.0f; }
    static __device__ __forceinline__ bool le0(float a) { return a <= 0.0f; }
    // the median of (0, a, b): the smaller magnitude when a and b have one
    // strict sign, else zero; four min/max operations, no branch. A zero
    // result carries a -0 only when an argument is -0; adding +0 makes it
    // +0, so the bits are those of the sign-test form (checked by
    // orcha_selftest_fp64_emulation). Measured on a B300 against that form:
    // FP32-flux shortcut +3 %.
    static __device__ __forceinline__ float minmod(float a, float b) {
        return __fadd_rn(fmaxf(fminf(a, b), fminf(fmaxf(a, b), 0.0f)), 0.0f);
    }
    static __device__ __forceinline__ float half(float x) { return 0.5f * x; }
    static __device__ __forceinline__ float zero() { return 0.0f; }
    static __device__ __forceinline__ double to_double(float x) { return to_f64(x); }
};

// ---------------------------------------------------------------- double-word (FF task)
// Reconstruction, predictor and HLL fluxes in double-word arithmetic
// (dword.cuh, ~48 bits on the FP32 pipe); the conserved-state update, the
// guard fill and the dt reduction stay FP64.
}  // namespace orcha
#include "dword.cuh"
namespace orcha {
template <> __device__ __forceinline__ dw as<dw, dw>(dw x) { return x; }
template <> struct P<dw> {
    using store = dw;
    // binary64 -> double-word: hi = x rounded to binary32, lo = (x - hi)
    // rounded (x - hi is exact in binary64); |x - (hi + lo)| <= 2^-49 |x|
    static __device__ __forceinline__ dw in(double x) {
        const float h = __double2float_rn(x);
        return {h, __double2float_rn(__dsub_rn(x, to_f64(h)))};
    }
    static __device__ __forceinline__ dw rcp(dw x) { return dw_rcp(x); }
    static __device__ __forceinline__ dw sqrt(dw x) { return x.hi > 0.0f ? x * dw_rsqrt(x) : dw{0.0f, 0.0f}; }
    static __device__ __forceinline__ dw sound(dw x, dw rho) {
        return x.hi > 0.0f ? x * dw_rsqrt(x * rho) : dw{0.0f, 0.0f};
    }
    static __device__ __forceinline__ dw ld(const dw* p) { return *p; }
    static __device__ __forceinline__ void st(dw* p, dw x) { *p = x; }
    // signs and order of a normalised double-word are those of its high part
    static __device__ __forceinline__ bool pos(dw x) { return x.hi > 0.0f; }
    static __device__ __forceinline__ bool neg(dw x) { return x.hi < 0.0f; }
    static __device__ __forceinline__ bool lt(dw a, dw b) { return dw_lt(a, b); }
    static __device__ __forceinline__ bool ge0(dw a) { return a.hi >= 0.0f; }
    static __device__ __forceinline__ bool le0(dw a) { return a.hi <= 0.0f; }
    // without branches: both positive -> the smaller, both negative -> the
    // larger, else 0
    static __device__ __forceinline__ dw minmod(dw a, dw b) {
        const bool pos = (a.hi > 0.0f) & (b.hi > 0.0f), neg = (a.hi < 0.0f) & (b.hi < 0.0f);
        const bool take_a = pos ? dw_lt(a, b) : dw_lt(b, a);
        const dw m = take_a ? a : b;
        return (pos | neg) ? m : dw{0.0f, 0.0f};
    }
    static __device__ __forceinline__ dw half(dw x) { return {__fmul_rn(0.5f, x.hi), __fmul_rn(0.5f, x.lo)}; }
    static __device__ __forceinline__ dw zero() { return dw{0.0f, 0.0f}; }
    static __device__ __forceinline__ double to_double(dw x) { return __dadd_rn(to_f64(x.hi), to_f64(x.lo)); }
};

// ---------------------------------------------------------------- float-float (error-free transformations)
// A value carried as an unevaluated sum hi + lo of two floats (about 46
// significant bits). two_sum (Knuth) and two_prod (with FMA) are exact.
struct ff {
    float hi, lo;
};
__device__ __forceinline__ ff two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
// c * (hi + lo) for a float-float constant c = ch + cl, as an unnormalised pair.
__device__ __forceinline__ ff ff_scale(ff d, float ch, float cl) {
    const float p = d.hi * ch;
    const float pe = fmaf(d.hi, ch, -p);                  // d.hi * ch = p + pe exactly
    return {p, fmaf(d.hi, cl, fmaf(d.lo, ch, pe))};
}
// (a.hi + a.lo) + (b.hi + b.lo) without renormalising: the high parts'
// sum exactly (two_sum) and the low parts added to its error. The pair may
// be an ulp or so off normalised, which its uses do not need: another such
// sum, or ff_to_double, whose one FP64 addition rounds hi + lo, the same
// real number a renormalised pair would hold.
__device__ __forceinline__ ff ff_add(ff a, ff b) {
    const ff s = two_sum(a.hi, b.hi);
    return {s.hi, s.lo + (a.lo + b.lo)};
}
// Exact difference a - b of two floats as a float-float.
__device__ __forceinline__ ff ff_diff(float a, float b) { return two_sum(a, -b); }
__device__ __forceinline__ double ff_to_double(ff a) { return __dadd_rn(to_f64(a.hi), to_f64(a.lo)); }

// ---------------------------------------------------------------- mesh as the kernels see it
struct MeshDev {
    int ndim, nvar;
    int nb[3];          // blocks per axis
    int bs[3];          // interior cells per block per axis
    int pad[3];         // padded extents: bs + 2*kGuard on active axes, 1 otherwise
    int periodic[3];
    long long var_stride;   // pad[0]*pad[1]*pad[2]
    long long blk_stride;   // nvar * var_stride
    double gamma, gm1, igm1, cfl;   // gm1 = gamma - 1, igm1 = 1 / (gamma - 1), formed in FP64 on the host
    double idx[3];          // 1 / dx_d
    const double* dt;       // device: current time step
    unsigned long long* smax;   // device: per-block largest signal speed (bits of a non-negative double)
    int* err;               // device: error word (ORCHA_DEVERR_* bits)
    // device, or null: per-block largest FP32 upper bound of the signal speeds
    // the step skipped (bits of a non-negative double; see SpeedBound in
    // hydro.cuh). Null: every cell's speed is evaluated in FP64.
    unsigned long long* sub = nullptr;
};

// |x| rounded toward zero to binary32, on the integer pipe: f <= |x| <
// f (1 + 2^-23). True when x is 0 or 2^-40 <= |x| < 2^41, the range in which
// the signal-speed bound below keeps every FP32 intermediate normal; false
// otherwise (f is then meaningless). The top 23 fraction bits of the binary64
// pattern are the binary32 fraction; the 9 low exponent bits plus 128 (mod
// 512) are the binary32 biased exponent e - 896 for e in that range.
__device__ __forceinline__ bool mag_f32_rz(double x, float& f) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned hi = (unsigned)(b >> 32) & 0x7FFFFFFFu, lo = (unsigned)b;
    f = __uint_as_float(__funnelshift_l(lo, hi, 3) + 0x40000000u);
    if ((hi | lo) == 0u) f = 0.0f;
    return (hi >> 20) - 983u <= 80u || (hi | lo) == 0u;
}

// Largest of two non-negative doubles given as bit patterns (NaN patterns of
// either sign compare above every finite value, so a NaN is never lost).
__device__ __forceinline__ unsigned long long umax64(unsigned long long a, unsigned long long b) {
    return a > b ? a : b;
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = umax64(x, __shfl_xor_sync(0xffffffffu, x, o));
    return x;
}

// Reduce a per-thread signal speed over the CTA and raise the block's entry.
// `scratch` holds one word per warp. Every thread of the CTA must call it.
__device__ __forceinline__ void cta_raise_smax(double s, unsigned long long* scratch,
                                               unsigned long long* dst) {
    unsigned long long b = warp_max_u64((unsigned long long)__double_as_longlong(s));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) scratch[warp] = b;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long m = 0;
        for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) m = umax64(m, scratch[w]);
        atomicMax(dst, m);
    }
}

// The same for two values at once (one barrier): a into dst, b into dst2.
// Needs at most 16 warps (scratch holds 32 words).
__device__ __forceinline__ void cta_raise_smax2(unsigned long long a, unsigned long long b, unsigned long long* scratch,
                                                unsigned long long* dst, unsigned long long* dst2) {
    a = warp_max_u64(a);
    b = warp_max_u64(b);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) { scratch[warp] = a; scratch[16 + warp] = b; }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long ma = 0, mb = 0;
        for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) { ma = umax64(ma, scratch[w]); mb = umax64(mb, scratch[16 + w]); }
        atomicMax(dst, ma);
        if (mb) atomicMax(dst2, mb);
    }
}

}  // namespace orcha
