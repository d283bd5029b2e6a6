// softfp64.cuh -- binary64 add, subtract and multiply, round to nearest
// even, computed with integer instructions.
//
// On this GPU the FP64 pipe (2 lanes per SM per clock) is the bound of the
// FP64 hydro path while the integer pipe sits nearly idle, so a share of the
// FP64 adds and multiplies is issued as integer code instead. Written from
// the IEEE-754 binary64 definition: the exact result is formed in integer
// arithmetic (106-bit product; 10 guard bits plus a sticky bit for sums) and
// rounded to nearest, ties to even, so the result equals the hardware
// operation bit for bit (checked on the GPU by orcha_selftest_fp64_emulation).
// Operands that are subnormal, infinite or NaN, and results that would be
// subnormal or overflow, branch to the hardware instruction; exact zeros are
// handled inline.
#pragma once

#include <cuda_runtime.h>

namespace orcha {

static __device__ __noinline__ double hw_dmul(double x, double y) { return __dmul_rn(x, y); }
static __device__ __noinline__ double hw_dadd(double x, double y) { return __dadd_rn(x, y); }

constexpr unsigned long long kM52 = 0x000FFFFFFFFFFFFFull;
constexpr unsigned long long kHid = 0x0010000000000000ull;
constexpr unsigned long long kSign = 0x8000000000000000ull;
constexpr unsigned long long kAbs = 0x7FFFFFFFFFFFFFFFull;

__device__ __forceinline__ double em_mul(double x, double y) {
    const unsigned long long a = (unsigned long long)__double_as_longlong(x);
    const unsigned long long b = (unsigned long long)__double_as_longlong(y);
    const unsigned long long sign = (a ^ b) & kSign;
    const int ea = (int)((a >> 52) & 0x7FF), eb = (int)((b >> 52) & 0x7FF);
    if (ea == 0 || eb == 0 || ea == 0x7FF || eb == 0x7FF) {
        if ((((a & kAbs) == 0) || ((b & kAbs) == 0)) && ea != 0x7FF && eb != 0x7FF)
            return __longlong_as_double((long long)sign);          // 0 x finite = signed 0
        return hw_dmul(x, y);
    }
    const unsigned long long ma = (a & kM52) | kHid, mb = (b & kM52) | kHid;
    const unsigned long long lo = ma * mb;                         // product = hi:lo in [2^104, 2^106)
    const unsigned long long hi = __umul64hi(ma, mb);
    const int top = (int)(hi >> 41);                               // product >= 2^105
    int e = ea + eb - 1023 + top;
    const int s = 52 + top;                                        // dropped low bits (all in lo)
    unsigned long long m = (hi << (64 - s)) | (lo >> s);           // 53 significant bits
    const unsigned long long rem = lo & ((1ull << s) - 1ull), half = 1ull << (s - 1);
    m += (rem > half) || (rem == half && (m & 1ull));
    if (m >> 53) {                                                 // rounding carried out of the significand
        m >>= 1;
        ++e;
    }
    if (e <= 0 || e >= 0x7FF) return hw_dmul(x, y);                // subnormal result or overflow
    return __longlong_as_double((long long)(sign | ((unsigned long long)e << 52) | (m & kM52)));
}

__device__ __forceinline__ double em_add(double x, double y) {
    unsigned long long a = (unsigned long long)__double_as_longlong(x);
    unsigned long long b = (unsigned long long)__double_as_longlong(y);
    if ((a & kAbs) < (b & kAbs)) {                                 // |a| >= |b|
        const unsigned long long t = a;
        a = b;
        b = t;
    }
    const int ea = (int)((a >> 52) & 0x7FF), eb = (int)((b >> 52) & 0x7FF);
    if (ea == 0x7FF || eb == 0) {
        if ((b & kAbs) == 0 && ea != 0x7FF) {                      // b = +-0
            if ((a & kAbs) == 0) return __longlong_as_double((long long)(a & b));   // +0 unless both -0
            return __longlong_as_double((long long)a);
        }
        return hw_dadd(x, y);
    }
    const unsigned long long ma = ((a & kM52) | kHid) << 10;       // leading bit at 62, 10 guard bits
    const unsigned long long mb0 = ((b & kM52) | kHid) << 10;
    const int d = ea - eb;
    const unsigned long long mb =
        d >= 63 ? 1ull : ((mb0 >> d) | ((mb0 & ((1ull << d) - 1ull)) != 0ull));   // aligned, sticky in bit 0
    int e = ea;
    unsigned long long m;
    if (((a ^ b) >> 63) == 0) {
        m = ma + mb;
        if (m >> 63) {
            m = (m >> 1) | (m & 1ull);
            ++e;
        }
    } else {
        m = ma - mb;
        if (m == 0) return 0.0;                                    // exact cancellation: +0
        const int lz = __clzll((long long)m) - 1;
        m <<= lz;
        e -= lz;
        if (e <= 0) return hw_dadd(x, y);                          // subnormal result
    }
    unsigned long long r = m >> 10;
    const unsigned rem = (unsigned)(m & 0x3FFull);
    r += (rem > 0x200u) || (rem == 0x200u && (r & 1ull));
    if (r >> 53) {
        r >>= 1;
        ++e;
    }
    if (e >= 0x7FF) return hw_dadd(x, y);                          // overflow
    return __longlong_as_double((long long)((a & kSign) | ((unsigned long long)e << 52) | (r & kM52)));
}

__device__ __forceinline__ double em_sub(double x, double y) {
    return em_add(x, __longlong_as_double(__double_as_longlong(y) ^ (long long)kSign));
}

}  // namespace orcha
