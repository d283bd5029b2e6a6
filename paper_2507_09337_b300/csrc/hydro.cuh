// hydro.cuh -- the fused block-hydro task kernel (one time step of a packet).
//
// Scheme (per cell, per step): primitives W from the conserved state U
// (ideal gamma-law EOS), minmod slopes of W along each axis, a Hancock
// half-step predictor in primitive form summed over all axes, face states
// Wbar -+ dW/2 (a cell whose face states have rho <= 0 or p <= 0 falls back
// to first order), HLL fluxes with Davis wave speeds, and the unsplit
// conservative update U+ = U - sum_d (dt/dx_d)(F_hi - F_lo) summed x, y, z.
// The epilogue raises the block's largest signal speed sum_d (|u_d|+c)/dx_d
// of U+ (the next CFL time step). The paper's solver paragraph (section
// "Experiments") describes the task only as explicit finite volume with
// guard-cell halos refreshed before it runs; the expression trees below are
// the ones of the FP64 definition, operation for operation (the contracted
// FP64 build fuses a product into the sum it is written in, and regroups the
// predictor and rewrites the sound speed and the HLL combination; see
// common.cuh).
//
// GPU mapping. One CTA owns a TX x TY column tile of one block and sweeps it
// along z (2.5D blocking), one owner thread per interior column (the FP64
// Hancock variant adds one thread per tile-ring cell). Per plane:
//   L  primitives of the (TX+4)(TY+4) plane two layers ahead into a ring of
//      three planes in shared memory (the z stencil needs p-1, p, p+1), read
//      as 16-byte pairs of x-neighbours;
//   P  slopes, predictor and face states of plane p: interior cells by their
//      owner thread (z face states stay in its registers), the one-cell ring
//      around the tile by the ring threads, or else by the first 2(TX+TY)
//      owners after their own cell (the one x or y face state a tile reads);
//   F  every x and y face flux of plane p once, into shared memory over the
//      face state it was formed from;
//   U  each owner forms its z face flux from registers, finishes the update
//      of plane p-1 (whose z fluxes are now both known) and writes it.
// Every face flux is evaluated exactly once per CTA and used by both cells,
// so the update telescopes; tiles of one block recompute only their one-cell
// ring of predicted states and their boundary faces.
#pragma once

#include <type_traits>

#include "common.cuh"

namespace orcha {

// ---------------------------------------------------------------- FP64 pipe balance
// Which stages of the FP64 task compute their adds and multiplies on the
// integer pipe (type re) instead of the FP64 pipe (type rd); both give the
// same bits, so the split only moves work between pipes. Bits: 1 primitive
// conversion on load, 2 predictor, 4 HLL left state, 8 HLL right state,
// 16 HLL combination, 32 HLL wave speeds. Measured on a B300: every
// emulated share is slower (an emulated operation costs more integer issue
// than the FP64-pipe time it frees), so the default is 0.
#ifndef ORCHA_EMU
#define ORCHA_EMU 0
#endif
// Whether a variant asks L2 for each plane's source lines two planes ahead of
// its load. Measured on a B300 (128^3 Sedov): FF +7 %, FP64 neutral (-0.4 %
// with ring threads, one CTA per SM), FP32 flux -4 %, so only the FF variant
// does.
template <class T> struct Prefetch { static constexpr bool value = false; };
template <> struct Prefetch<dw> { static constexpr bool value = true; };

template <class T, int BIT>
using Arith = typename std::conditional<std::is_same<T, rd>::value && ((ORCHA_EMU & BIT) != 0), re, T>::type;

// ---------------------------------------------------------------- point functions

// W from U: r = 1/rho, u_d = m_d * r, p = (gamma-1) * (E - 0.5 * sum_d m_d u_d).
template <class T, int NDIM>
__device__ __forceinline__ void prim_from_cons(const T* U, T* W, T& r, T gm1) {
    constexpr int NV = NDIM + 2;
    W[0] = U[0];
    r = P<T>::rcp(U[0]);
    T mu;
#pragma unroll
    for (int d = 0; d < NDIM; ++d) {
        W[1 + d] = U[1 + d] * r;
        mu = (d == 0) ? (U[1] * W[1]) : (mu + (U[1 + d] * W[1 + d]));
    }
    T ke = P<T>::half(mu);
    W[NV - 1] = gm1 * (U[NV - 1] - ke);
}

// The same with the arithmetic done in type A (values in and out in T).
template <class A, class T, int NDIM>
__device__ __forceinline__ void prim_from_cons_as(const T* U, T* W, T& r, T gm1) {
    constexpr int NV = NDIM + 2;
    A u[NV], w[NV], ra;
#pragma unroll
    for (int v = 0; v < NV; ++v) u[v] = as<A>(U[v]);
    prim_from_cons<A, NDIM>(u, w, ra, as<A>(gm1));
#pragma unroll
    for (int v = 0; v < NV; ++v) W[v] = as<T>(w[v]);
    r = as<T>(ra);
}

// minmod: the smaller-magnitude argument when both share a strict sign, else 0.
template <class T>
__device__ __forceinline__ T minmod(T a, T b) {
    return P<T>::minmod(a, b);
}

// Conserved state and physical flux of a primitive state given normal-first:
// W = (rho, u_n, u_t1[, u_t2], p). |u|^2 is summed in coordinate order x, y, z;
// for an x or y normal that is (u_n^2 + u_t1^2) + u_t2^2 (addition commutes),
// for a z normal (u_t1^2 + u_t2^2) + u_n^2.
template <class A, class T, int NDIM, bool ZNORMAL>
__device__ __forceinline__ void cons_flux(const T* Wt, T* Ut, T* Ft, T igm1t) {
    constexpr int NV = NDIM + 2;
    A W[NV], U[NV], F[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) W[v] = as<A>(Wt[v]);
    const A igm1 = as<A>(igm1t);
    const A rho = W[0], un = W[1], p = W[NV - 1];
    U[0] = rho;
#pragma unroll
    for (int k = 1; k <= NDIM; ++k) U[k] = rho * W[k];
    A q2;
    if (NDIM == 2) q2 = (W[1] * W[1]) + (W[2] * W[2]);
    else if (!ZNORMAL) q2 = ((W[1] * W[1]) + (W[2] * W[2])) + (W[3] * W[3]);
    else q2 = ((W[2] * W[2]) + (W[3] * W[3])) + (W[1] * W[1]);
    U[NV - 1] = (p * igm1) + (P<A>::half(rho) * q2);
    F[0] = U[1];
    F[1] = (U[1] * un) + p;
#pragma unroll
    for (int k = 2; k <= NDIM; ++k) F[k] = U[k] * un;
    F[NV - 1] = (U[NV - 1] + p) * un;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        Ut[v] = as<T>(U[v]);
        Ft[v] = as<T>(F[v]);
    }
}

// HLL flux with Davis wave speeds between normal-first states L and R.
template <class T, int NDIM, bool ZNORMAL>
__device__ __forceinline__ void hll(const T* L, const T* R, T* F, T g, T igm1) {
    constexpr int NV = NDIM + 2;
    using AS = Arith<T, 32>;     // wave speeds
    using AC = Arith<T, 16>;     // combination
    const AS gs = as<AS>(g);
    const auto cL = P<AS>::sound(gs * as<AS>(L[NV - 1]), as<AS>(L[0]));
    const auto cR = P<AS>::sound(gs * as<AS>(R[NV - 1]), as<AS>(R[0]));
    AS a = as<AS>(L[1]) - cL, b = as<AS>(R[1]) - cR;
    const AS SL = P<AS>::lt(a, b) ? a : b;
    a = as<AS>(L[1]) + cL;
    b = as<AS>(R[1]) + cR;
    const AS SR = P<AS>::lt(b, a) ? a : b;
    T UL[NV], UR[NV], FL[NV], FR[NV];
    cons_flux<Arith<T, 4>, T, NDIM, ZNORMAL>(L, UL, FL, igm1);
    cons_flux<Arith<T, 8>, T, NDIM, ZNORMAL>(R, UR, FR, igm1);
    if (P<AS>::ge0(SL)) {
#pragma unroll
        for (int v = 0; v < NV; ++v) F[v] = FL[v];
    } else if (P<AS>::le0(SR)) {
#pragma unroll
        for (int v = 0; v < NV; ++v) F[v] = FR[v];
    } else if constexpr (kContract && std::is_same<AC, rd>::value) {
        // the same flux as F_L + k ((F_L - F_R) + S_R (U_R - U_L)), k = S_L / (S_R - S_L):
        // four FP64 operations per variable instead of five
        const rd sl = SL, sr = SR;
        const rd k = sl * P<rd>::rcp(sr - sl);
#pragma unroll
        for (int v = 0; v < NV; ++v)
            F[v] = rd(fma(k.v, fma(sr.v, (UR[v] - UL[v]).v, (FL[v] - FR[v]).v), FL[v].v));
    } else {
        const AC sl = as<AC>(SL), sr = as<AC>(SR);
        const AC slsr = sl * sr;
        const AC inv = P<AC>::rcp(sr - sl);
#pragma unroll
        for (int v = 0; v < NV; ++v)
            F[v] = as<T>((((sr * as<AC>(FL[v])) - (sl * as<AC>(FR[v]))) +
                          (slsr * (as<AC>(UR[v]) - as<AC>(UL[v])))) * inv);
    }
}

// Largest signal speed sum_d (|u_d| + c) / dx_d over the interior cells of
// block `blk` of the padded state U handled by this thread (stride
// blockDim.x), as the bits of a non-negative double; flags non-physical cells.
// (chunk, nchunks): this CTA takes cells chunk * blockDim.x + t, stepping
// nchunks * blockDim.x. CG: load through L2 only (__ldcg), for a state other
// CTAs of the same launch have just written.
template <bool CG = false>
__device__ __forceinline__ unsigned long long block_signal_speed(const MeshDev& m, int blk,
                                                                 const double* __restrict__ U, int chunk = 0,
                                                                 int nchunks = 1) {
    const double* Ub = U + (long long)blk * m.blk_stride;
    const int ncell = m.bs[0] * m.bs[1] * m.bs[2];
    unsigned long long smaxb = 0ull;
    for (int c = chunk * blockDim.x + threadIdx.x; c < ncell; c += nchunks * blockDim.x) {
        const int i = c % m.bs[0], r0 = c / m.bs[0], j = r0 % m.bs[1], k = r0 / m.bs[1];
        const int kk = (m.ndim == 3) ? k + kGuard : 0;
        const int po = (kk * m.pad[1] + (j + kGuard)) * m.pad[0] + (i + kGuard);
        rd Uc[5], W[5], r;
        for (int v = 0; v < m.nvar; ++v) Uc[v] = rd(CG ? __ldcg(&Ub[po + v * m.var_stride]) : Ub[po + v * m.var_stride]);
        if (m.ndim == 3) prim_from_cons<rd, 3>(Uc, W, r, rd(m.gm1));
        else prim_from_cons<rd, 2>(Uc, W, r, rd(m.gm1));
        const int nv = m.nvar;
        if (!(P<rd>::pos(W[0]) && P<rd>::pos(W[nv - 1]))) atomicOr(m.err, 1);
        const rd cs = P<rd>::sqrt((rd(m.gamma) * W[nv - 1]) * r);
        rd s = (rd(fabs(W[1].v)) + cs) * rd(m.idx[0]);
        for (int d = 1; d < m.ndim; ++d) s = s + ((rd(fabs(W[1 + d].v)) + cs) * rd(m.idx[d]));
        smaxb = umax64(smaxb, (unsigned long long)bits(s));   // s >= 0 or NaN
    }
    return smaxb;
}

// Signal speed sum_d (|u_d| + c) / dx_d of one new FP64 state, as the bits of
// a non-negative double; raises the non-physical flag. T = rd: the
// definition's expression tree (FP64 and FP32-flux tasks). T = float (the
// FP32-flux shortcut): evaluated in FP32 from the
// state rounded to nearest and rounded up by a factor 1 + 2^-18 (above the
// few-ulp error of that evaluation), so dt = cfl / max never exceeds the FP64
// value by more than rounding; a cell whose FP32 pressure is not positive is
// re-evaluated in FP64 (cancellation in E - |m|^2/(2 rho)).
template <class T, int NDIM>
__device__ __forceinline__ unsigned long long new_state_speed(const MeshDev& m, const rd* Un) {
    constexpr int NV = NDIM + 2;
    if constexpr (std::is_same<T, float>::value) {
        float U[NV], W[NV], r;
#pragma unroll
        for (int v = 0; v < NV; ++v) U[v] = to_f32(Un[v].v);
        prim_from_cons<float, NDIM>(U, W, r, to_f32(m.gm1));
        if (W[0] > 0.0f && W[NV - 1] > 0.0f) {
            const float c = P<float>::sqrt((to_f32(m.gamma) * W[NV - 1]) * r);
            float s = (fabsf(W[1]) + c) * to_f32(m.idx[0]);
#pragma unroll
            for (int d = 1; d < NDIM; ++d) s = s + (fabsf(W[1 + d]) + c) * to_f32(m.idx[d]);
            s = s * 1.0000038146972656f;                     // 1 + 2^-18
            return (unsigned long long)__double_as_longlong(to_f64(s));
        }
    }
    rd W[NV], r;
    prim_from_cons<rd, NDIM>(Un, W, r, rd(m.gm1));
    if (!(P<rd>::pos(W[0]) && P<rd>::pos(W[NV - 1]))) atomicOr(m.err, 1);
    const rd c = P<rd>::sqrt((rd(m.gamma) * W[NV - 1]) * r);
    rd s = (rd(fabs(W[1].v)) + c) * rd(m.idx[0]);
#pragma unroll
    for (int d = 1; d < NDIM; ++d) s = s + ((rd(fabs(W[1 + d].v)) + c) * rd(m.idx[d]));
    return (unsigned long long)bits(s);   // s >= 0 or NaN
}

// ---------------------------------------------------------------- signal-speed filter
// Only the largest signal speed of a step matters (dt = cfl / max), and on
// most meshes nearly every cell lies far below it. The FP64 evaluation
// (new_state_speed<rd>: a reciprocal, a square root and ~20 more FP64-pipe
// operations) is therefore skipped for a cell whose rigorous FP32 upper
// bound lies below a threshold, a quarter of the previous step's maximum
// (cfl / (4 dt)); the bound is raised into the block's `sub` entry instead.
// The step's reducer accepts max smax as the exact maximum only when no
// skipped bound exceeds it, and otherwise evaluates the cells of the blocks
// whose bound does in FP64 (finish_mesh_step). So dt has the bits of the
// unfiltered evaluation whatever the threshold; the threshold only decides
// how often the FP64 path runs.
//
// The bound: the state's magnitudes rounded toward zero to binary32 (below)
// and up by one ulp bracket the exact ones; every later operation rounds
// towards the side it bounds (__fmul_ru and friends, the IEEE directed
// roundings), so p_hi >= (gamma-1)(E - |m|^2/(2 rho)), c_hi >= sqrt(gamma p /
// rho) and s_hi >= sum_d (|m_d|/rho + c) / dx_d for the real numbers the
// double state and constants define. The FP64 evaluation differs from that
// real value by at most ~2^-23 (1/dx_max / 1/dx_min) of it, even under
// cancellation in E - |m|^2/(2 rho) (its pressure error is ~2^-50 (E + ke),
// whose square root is ~2^-25 (c + |u|)); `margin` covers it 16 times over.
// A cell is skipped only if its FP32 lower bound of p exceeds 2^-40 E, which
// keeps the FP64 pressure positive too (the non-physical check the FP64 path
// makes), and only if its values lie in the range mag_f32_rz accepts.
struct SpeedBound {
    float gm1_lo, gm1_hi, g_hi, idx_hi[3], margin, thr;
};

__device__ __forceinline__ SpeedBound speed_bound_setup(const MeshDev& m, double dt) {
    SpeedBound b;
    b.gm1_lo = __double2float_rd(m.gm1);
    b.gm1_hi = __double2float_ru(m.gm1);
    b.g_hi = __double2float_ru(m.gamma);
    double imin = m.idx[0], imax = m.idx[0];
    for (int d = 0; d < 3; ++d) {
        b.idx_hi[d] = __double2float_ru(m.idx[d]);
        if (d < m.ndim) { imin = fmin(imin, m.idx[d]); imax = fmax(imax, m.idx[d]); }
    }
    b.margin = __fmaf_ru(__double2float_ru(imax / imin), 0x1p-19f, 1.0f);
    const double t = m.cfl / (4.0 * dt);
    b.thr = (m.sub != nullptr && t > 0.0 && t < 1e30) ? __double2float_rd(t) : 0.0f;
    return b;
}

// An FP32 upper bound ub of the FP64 signal speed of the state Un (the value
// new_state_speed<rd> returns), or false if the bound does not apply.
template <int NDIM>
__device__ __forceinline__ bool speed_upper(const SpeedBound& sb, const rd* Un, float& ub) {
    constexpr int NV = NDIM + 2;
    constexpr float kUp = 0x1.000002p0f;                 // 1 + 2^-23: a truncated magnitude times this bounds it
    float rl, el, ml[NDIM];
    bool ok = mag_f32_rz(Un[0].v, rl) && mag_f32_rz(Un[NV - 1].v, el) && __double_as_longlong(Un[0].v) > 0 &&
              __double_as_longlong(Un[NV - 1].v) > 0;
#pragma unroll
    for (int d = 0; d < NDIM; ++d) ok = mag_f32_rz(Un[1 + d].v, ml[d]) && ok;
    if (!ok) return false;
    const float rh = __fmul_ru(rl, kUp), eh = __fmul_ru(el, kUp);
    const float ri_hi = __frcp_ru(rl), ri_lo = __frcp_rd(rh);      // bracket 1/rho
    float kel = 0.0f, keh = 0.0f, ah[NDIM];
#pragma unroll
    for (int d = 0; d < NDIM; ++d) {
        const float mh = __fmul_ru(ml[d], kUp);
        ah[d] = __fmul_ru(mh, ri_hi);                                // >= |m_d| / rho
        kel = __fadd_rd(kel, __fmul_rd(ml[d], __fmul_rd(ml[d], ri_lo)));
        keh = __fadd_ru(keh, __fmul_ru(mh, ah[d]));
    }
    kel = 0.5f * kel;                                                // exact halvings (normal range)
    keh = 0.5f * keh;
    const float pl = __fmul_rd(sb.gm1_lo, __fadd_rd(el, -keh));
    if (!(pl > eh * 0x1p-40f)) return false;
    const float ph = __fmul_ru(sb.gm1_hi, __fadd_ru(eh, -kel));
    const float ch = __fsqrt_ru(__fmul_ru(__fmul_ru(sb.g_hi, ph), ri_hi));
    float s = 0.0f;
#pragma unroll
    for (int d = 0; d < NDIM; ++d) s = __fadd_ru(s, __fmul_ru(__fadd_ru(ah[d], ch), sb.idx_hi[d]));
    ub = __fmul_ru(s, sb.margin);
    return true;
}

// The FP32-flux shortcut's signal speed (new_state_speed<float>: FP32, rounded
// up by 1 + 2^-18, FP64 where the FP32 pressure is not positive) over the
// interior cells of block `blk` handled by this thread; the first time step
// of a shortcut run comes from the same rule as every later one.
__device__ __forceinline__ unsigned long long block_signal_speed_f32(const MeshDev& m, int blk,
                                                                     const double* __restrict__ U, int chunk = 0,
                                                                     int nchunks = 1) {
    const double* Ub = U + (long long)blk * m.blk_stride;
    const int ncell = m.bs[0] * m.bs[1] * m.bs[2];
    unsigned long long smaxb = 0ull;
    for (int c = chunk * blockDim.x + threadIdx.x; c < ncell; c += nchunks * blockDim.x) {
        const int i = c % m.bs[0], r0 = c / m.bs[0], j = r0 % m.bs[1], k = r0 / m.bs[1];
        const int kk = (m.ndim == 3) ? k + kGuard : 0;
        const int po = (kk * m.pad[1] + (j + kGuard)) * m.pad[0] + (i + kGuard);
        rd Uc[5];
        for (int v = 0; v < m.nvar; ++v) Uc[v] = rd(Ub[po + v * m.var_stride]);
        const unsigned long long b =
            (m.ndim == 3) ? new_state_speed<float, 3>(m, Uc) : new_state_speed<float, 2>(m, Uc);
        smaxb = umax64(smaxb, b);
    }
    return smaxb;
}

// ---------------------------------------------------------------- the kernel

template <int NDIM, int TX, int TY>
struct Tile {
    static constexpr int NV = NDIM + 2;
    static constexpr int NW = NV + 1;                 // primitives + 1/rho
    static constexpr int NT = TX * TY;                // owner threads = interior columns
    static constexpr int R2X = TX + 4, R2Y = TY + 4, R2N = R2X * R2Y;
    static constexpr int R1X = TX + 2, R1Y = TY + 2, R1N = R1X * R1Y;
    static constexpr int NRING = 2 * (TX + TY);       // predicted ring cells (corners unused)
    // Threads per CTA. The FP64 Hancock variant adds one thread per ring cell
    // (in whole warps), so the ring is predicted alongside the interior
    // instead of after it by the first NRING owners: measured on a B300, 16x16
    // tiles +5 %. The FP32-flux, double-word and Runge-Kutta variants lose with
    // it (less predictor work per cell, or fewer CTAs per SM) and keep one
    // thread per interior column.
    template <class T, bool RK>
    static constexpr int nb() {
        return std::is_same<T, rd>::value && !RK ? (NT + NRING + 31) / 32 * 32 : NT;
    }
    static constexpr int NXF = (TX + 1) * TY, NYF = TX * (TY + 1);
    static constexpr int NSLOT = (NDIM == 3) ? 3 : 1;
    template <class S>
    static constexpr size_t smem_bytes() {
        return sizeof(S) * ((size_t)NSLOT * NW * R2N + 4 * NV * R1N);
    }
};

// Where a hydro_tile sweep reads its planes and where its new state goes.
// GlobalIO is the one-step task: planes gathered from the state buffer Uin,
// new values written into the interiors of Uout, signal speeds raised. The
// two passes of a fused sweep (fused.cuh) keep the intermediate state of an
// extended tile in a per-CTA scratch instead:
//   pass A (ScratchOutIO): the tile grown by 2 cells on each side in x and
//     y, and by 2 planes in z (x0, y0, z0 lowered by 2, z1 raised by 2);
//     planes from Uin, base values gathered from Uin as well (owner columns
//     can lie in neighbouring blocks), new values into
//     scratch[plane - z0][var][column of the grown tile];
//   pass B (ScratchInIO): the tile itself; planes and base values from the
//     scratch (positions beyond an outflow edge of the domain read the
//     nearest in-domain cell, the boundary rule), new values into Uout; a
//     Heun second stage averages with the step's initial state in Uin.
// kThreads: the CTA size of a fused launch (pass A's thread count); a pass
// with fewer threads idles the rest outside its barriers.
struct GlobalIO {
    static constexpr bool kFilter = false;  // skip FP64 signal speeds below the threshold (SpeedBound)
    static constexpr bool kIn = false;      // planes and base values from the scratch
    static constexpr bool kOut = false;     // new values into the scratch
    static constexpr int kRaise = 1;        // 0: none; 1: m.smax (RK: stage 2); 2: the inner cells into io.smax2
    static constexpr int kThreads = 0;      // 0: the variant's own thread count
    static constexpr bool kReg = false;     // record the fluxes through the block's faces (FluxRegIO)
    double* scratch = nullptr;
    unsigned long long* smax2 = nullptr;    // kRaise 2: per-block maxima of the intermediate state
    double* reg = nullptr;
    int fsz = 0;
};
template <int NTH, int RAISE>
struct ScratchOutIO {
    static constexpr bool kIn = false, kOut = true, kReg = false, kFilter = false;
    static constexpr int kRaise = RAISE, kThreads = NTH;
    double* scratch;
    unsigned long long* smax2;
    double* reg;
    int fsz;
};
template <int NTH>
struct ScratchInIO {
    static constexpr bool kIn = true, kOut = false, kReg = false, kFilter = false;
    static constexpr int kRaise = 1, kThreads = NTH;
    double* scratch;
    unsigned long long* smax2;
    double* reg;
    int fsz;
};
// The one-step task that also records, per block, the flux through every
// cell of its six faces (the flux registers of a two-level mesh's flux
// correction): reg[((blk * 6 + 2 d + side) * nvar + v) * fsz + face cell],
// face cell = the two other axes' indices, lower axis fastest; packet path
// (whole blocks) only.
struct FluxRegIO : GlobalIO {
    static constexpr bool kReg = true;
};
// The one-step task of the persistent path, whose reducer (finish_mesh_step)
// handles the skipped speeds' bounds: GlobalIO with the signal-speed filter.
struct FilterIO : GlobalIO {
    static constexpr bool kFilter = true;
};

// One column tile of one block: the z sweep over interior planes [z0, z1)
// (default: the whole block; a sub-range recomputes its own z halo, so a
// block may be advanced as several z slabs with the same result bits). With
// GATHER the range may run on through the blocks above blk in the same
// column (plane q lies in block blk + (q / bz) nb_x nb_y), so one sweep
// covers several blocks with one z halo. Each block's largest signal speed
// of the new state is raised (atomicMax into m.smax, using the CTA scratch
// red) when the sweep leaves that block or the range ends.
// GATHER = false: guard cells are read from the padded block (filled by the
// guard-fill task). GATHER = true: guard cells are read straight from the
// source cell (a neighbour's interior, or the boundary rule's cell), so no
// guard-fill pass and no guard storage traffic are needed; the values are
// the same copies the guard fill would make.
//
// RK = true: one stage of Heun's two-stage Runge-Kutta method with the plain
// MUSCL operator L (face states from the stage's own primitives, no half
// step). stage 1: Uout = Uin + dt L(Uin); stage 2: Uout = 0.5 * (Uout +
// (Uin + dt L(Uin))), the old Uout (the step's initial state) read at the
// cell just before it is overwritten. Stage 1 raises no signal speed.
//
// FX (T = float only): the FP32-flux variant's shortcut update. By default
// (FX = false) the FP32 face fluxes are promoted to FP64 before the
// difference and the difference, its dt/dx scaling, the x+y+z sum, the
// update and the new state's signal speed are FP64, as for T = rd. With FX
// the differences are formed exactly in float-float, summed to ~46 bits, and
// the signal speed is evaluated in FP32 (rounded up by 1 + 2^-18).
template <int NDIM, int TX, int TY, class T, bool GATHER, bool RK = false, bool FX = false, class IO = GlobalIO>
__device__ __forceinline__ void hydro_tile(const MeshDev& m, const int blk, const int x0, const int y0,
                                           const double* __restrict__ Uin, double* __restrict__ Uout,
                                           unsigned char* smem_raw, unsigned long long* red, int z0 = 0,
                                           int z1 = -1, int stage = 0, IO io = IO{}) {
    using Tl = Tile<NDIM, TX, TY>;
    using S = typename P<T>::store;
    constexpr int NV = Tl::NV, NW = Tl::NW, NT = Tl::NT;
    constexpr int R2X = Tl::R2X, R2N = Tl::R2N, R1X = Tl::R1X, R1N = Tl::R1N;

    S* sW = reinterpret_cast<S*>(smem_raw);                 // [slot][NW][R2N]
    S* sFS = sW + Tl::NSLOT * NW * R2N;                    // [face 0..3 = x-,x+,y-,y+][NV][R1N]
    // Face fluxes overwrite the x+ / y+ face states they were formed from: the
    // left state of each x (y) face is read by that face's thread alone, before
    // it stores the flux. The flux of the x face on the high side of R1 cell i
    // is at sGx[v * R1N + i], that of the y face likewise in sGy.
    S* sGx = sFS + 1 * NV * R1N;
    S* sGy = sFS + 3 * NV * R1N;

    const int tid = threadIdx.x;
    const int px = m.pad[0], py = m.pad[1];
    const long long vs = m.var_stride;
    const double* Ub = Uin + (long long)blk * m.blk_stride;
    double* Ob = Uout + (long long)blk * m.blk_stride;
    const int bz = (NDIM == 3) ? m.bs[2] : 1;
    const int lgbz = 31 - __clz(bz);     // block sizes are 8, 16 or 32 (1 in 2D): bz = 2^lgbz
    if (NDIM != 3 || z1 < 0) { z0 = 0; z1 = bz; }
    const int bc[3] = {blk % m.nb[0], (blk / m.nb[0]) % m.nb[1], blk / (m.nb[0] * m.nb[1])};

    const T g = P<T>::in(m.gamma), gm1 = P<T>::in(m.gm1), igm1 = P<T>::in(m.igm1);
    const double dt = *m.dt;
    double cd[3];
    T hd[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        cd[d] = __dmul_rn(dt, m.idx[d]);              // dt / dx_d
        hd[d] = P<T>::in(__dmul_rn(0.5, cd[d]));      // (dt/2) / dx_d
    }

    // Threads 0 .. NT-1 own an interior column (its z state stays in their
    // registers); the ring cells are predicted by threads NT .. NT+NRING-1
    // when the variant has them (kSplit), else by owners 0 .. NRING-1 after
    // their own cell; every thread loads planes and forms face fluxes.
    constexpr int NB = Tl::template nb<T, RK>();
    constexpr bool kSplit = NB > NT;
    static_assert(IO::kThreads == 0 || IO::kThreads >= NB, "a fused launch has at least each pass's threads");
    constexpr bool kPartial = IO::kThreads > NB;     // threads NB.. only take part in the barriers
    const bool member = !kPartial || tid < NB;
    const bool owner = kPartial ? tid < NT : (!kSplit || tid < NT);
    const int ti = tid % TX, tj = tid / TX;         // owner column
    const int o2 = (tj + 2) * R2X + (ti + 2);       // in the R2 plane
    const int o1 = (tj + 1) * R1X + (ti + 1);       // in the R1 plane
    // ring cell of this thread: bottom row, top row, left column, right column
    const int rt = kSplit ? tid - NT : tid;
    const bool ringer = rt >= 0 && rt < Tl::NRING;
    int rc1 = 0, rc2 = 0, rface = 0;
    if (ringer) {
        int ci, cj;
        if (rt < TX) { ci = rt + 1; cj = 0; rface = 3; }                        // row -1: needs y+
        else if (rt < 2 * TX) { ci = rt - TX + 1; cj = TY + 1; rface = 2; }     // row TY: needs y-
        else if (rt < 2 * TX + TY) { ci = 0; cj = rt - 2 * TX + 1; rface = 1; }         // col -1: x+
        else { ci = TX + 1; cj = rt - 2 * TX - TY + 1; rface = 0; }             // col TX: x-
        rc1 = cj * R1X + ci;
        rc2 = (cj + 1) * R2X + (ci + 1);
    }

    // L: primitives of plane pz (interior z index, -2 .. bz+1) into its ring slot
    // Source of each R2 cell this thread loads. The x/y part of the halo
    // mapping is the same on every plane, so it is resolved once: the source
    // block's (x, y) index times the block stride plus the in-block offset of
    // the source column. Per plane only the z part is added (uniform over the
    // CTA). GATHER = false reads the padded block itself.
    // Cells are loaded in x pairs (2q, 2q + 1); R2X is even, so a pair never
    // straddles rows. When the two sources are consecutive (everywhere but a
    // clamped outflow edge) the pair is one 16-byte load per variable: the
    // first cell's padded x index is even (x0, the block size and the padded
    // row length are even), so with 16-byte aligned state buffers the address
    // is 16-byte aligned.
    constexpr int R2P = R2N / 2;
    constexpr int KMAX = (R2P + NB - 1) / NB;
    int bxy[KMAX][2], oxy[KMAX][2];       // per cell of pair k: source block's (x, y) index; in-block column offset
    unsigned interior_mask = 0;           // bit 2k + e: cell e of pair k is an interior column of the tile
    unsigned contig_mask = 0;             // bit k: the sources of pair k are consecutive
#pragma unroll
    for (int k = 0; k < KMAX; ++k) {
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int c = 2 * (tid + k * NB) + e;
            const int ci = c % R2X, cj = c / R2X;
            int sbx = bc[0], sby = bc[1], sx = x0 + ci, sy = y0 + cj;
            if (GATHER) {
                const int l[2] = {x0 + ci - kGuard, y0 + cj - kGuard};
                int sb[2], sl[2];
#pragma unroll
                for (int d = 0; d < 2; ++d) {
                    const int n = m.nb[d] * m.bs[d];
                    int gi = bc[d] * m.bs[d] + l[d];
                    if (l[d] < 0 || l[d] >= m.bs[d]) {
                        if (m.periodic[d]) { gi %= n; gi = gi < 0 ? gi + n : gi; }
                        else gi = gi < 0 ? 0 : (gi > n - 1 ? n - 1 : gi);
                    }
                    sb[d] = gi / m.bs[d];
                    sl[d] = gi % m.bs[d] + kGuard;
                }
                sbx = sb[0]; sby = sb[1]; sx = sl[0]; sy = sl[1];
            }
            bxy[k][e] = sbx + m.nb[0] * sby;
            oxy[k][e] = sy * px + sx;
            if constexpr (IO::kIn) {
                // the scratch holds this tile's R2 cells; beyond an outflow
                // edge of the domain the boundary rule's cell is read instead
                int cc[2] = {ci, cj};
#pragma unroll
                for (int d = 0; d < 2; ++d) {
                    const int n = m.nb[d] * m.bs[d];
                    const int gi = bc[d] * m.bs[d] + (d == 0 ? x0 : y0) + cc[d] - kGuard;
                    if (!m.periodic[d]) cc[d] -= gi < 0 ? gi : (gi > n - 1 ? gi - (n - 1) : 0);
                }
                bxy[k][e] = 0;
                oxy[k][e] = cc[1] * R2X + cc[0];
            }
            if (ci >= 2 && ci < TX + 2 && cj >= 2 && cj < TY + 2) interior_mask |= 1u << (2 * k + e);
        }
        if (bxy[k][1] == bxy[k][0] && oxy[k][1] == oxy[k][0] + 1) contig_mask |= 1u << k;
    }
    const int nbxy = m.nb[0] * m.nb[1];
    const int plane = py * px;
    // pass A of a fused sweep: the source of the owner's own column (for its
    // base values), gathered like the loads (it may lie in a neighbour block)
    int own_b = 0, own_o = 0;
    if constexpr (IO::kOut) {
        const int l[2] = {x0 + ti, y0 + tj};
        int sb[2], sl[2];
#pragma unroll
        for (int d = 0; d < 2; ++d) {
            const int n = m.nb[d] * m.bs[d];
            int gi = bc[d] * m.bs[d] + l[d];
            if (m.periodic[d]) { gi %= n; gi = gi < 0 ? gi + n : gi; }
            else gi = gi < 0 ? 0 : (gi > n - 1 ? n - 1 : gi);
            sb[d] = gi / m.bs[d];
            sl[d] = gi % m.bs[d] + kGuard;
        }
        own_b = sb[0] + m.nb[0] * sb[1];
        own_o = sl[1] * px + sl[0];
    }
    // plane pzi's slot in the scratch of a fused sweep (pass A writes planes
    // z0 .. z1-1 of its grown range, pass B reads z0-2 .. z1+1 of its own)
    auto scratch_slot = [&](int pzi) -> int {
        if (NDIM != 3) return 0;
        if constexpr (IO::kIn) {
            if (!m.periodic[2]) {        // beyond an outflow edge: the boundary plane
                const int n = m.nb[2] * m.bs[2], gz = bc[2] * m.bs[2] + pzi;
                pzi -= gz < 0 ? gz : (gz > n - 1 ? gz - (n - 1) : 0);
            }
            return pzi - (z0 - 2);
        }
        return pzi - z0;
    };
    const long long lvs = IO::kIn ? (long long)R2N : vs;   // variable stride of the plane source
    // slot of plane pzi in the three-plane ring; planes run from -2 (from -4
    // in pass A of a fused sweep), and % of a negative number is negative
    auto ring_slot = [](int pzi) -> int { return (pzi + 6) % 3; };
    int slot_m = 0, slot_c = 0, slot_p = 0;     // ring slots of planes p - 1, p, p + 1 (3D), rotated per plane

    // z part of the source of plane pzi (interior z index, -2 .. bz+1; 2D: 0):
    // the block-index offset (zb) and the in-block cell offset (zc)
    auto plane_z = [&](int pzi, int& zb, int& zc) {
        zb = 0;
        zc = 0;
        if (NDIM != 3) return;
        if constexpr (IO::kIn) {
            zc = scratch_slot(pzi) * NV * R2N;
            return;
        }
        int sbz = bc[2], sz = pzi + kGuard;
        if (GATHER && (pzi < 0 || pzi >= bz)) {
            // a sweep's planes reach at most four past the ends of its column
            // (pass A of a fused sweep), so one wrap suffices
            const int n = m.nb[2] * bz;
            int gi = bc[2] * bz + pzi;
            if (m.periodic[2]) gi = gi < 0 ? gi + n : (gi >= n ? gi - n : gi);
            else gi = gi < 0 ? 0 : (gi > n - 1 ? n - 1 : gi);
            sbz = gi >> lgbz;
            sz = (gi & (bz - 1)) + kGuard;
        }
        zb = sbz * nbxy;
        zc = sz * plane;
    };
    // source of cell e of pair k of this thread in the plane with z part (zb, zc)
    auto src_of = [&](int k, int e, int zb, int zc) -> const double* {
        if constexpr (IO::kIn) return io.scratch + (oxy[k][e] + zc);
        return Uin + (long long)(bxy[k][e] + zb) * m.blk_stride + (oxy[k][e] + zc);
    };
    // Ask L2 for the source lines of plane pzi ahead of its load (no registers held).
    auto prefetch_plane = [&](int pzi) {
        int zb, zc;
        plane_z(pzi, zb, zc);
#pragma unroll
        for (int k = 0; k < KMAX; ++k) {
            if (tid + k * NB >= R2P || !member) break;
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                if (e == 1 && ((contig_mask >> k) & 1u)) break;     // same 16 bytes as cell 0
                const double* src = src_of(k, e, zb, zc);
#pragma unroll
                for (int v = 0; v < NV; ++v) asm volatile("prefetch.global.L2 [%0];" ::"l"(src + v * lvs));
            }
        }
    };
    // L: primitives of plane pzi into ring slot `slot`
    auto load_plane = [&](int pzi, int slot) {
        S* w = sW + slot * NW * R2N;
        int zb, zc;
        plane_z(pzi, zb, zc);
        const bool zin = pzi >= z0 && pzi < z1;        // planes this item owns: each cell checked once
#pragma unroll
        for (int k = 0; k < KMAX; ++k) {
            const int q = tid + k * NB;
            if (q >= R2P || !member) break;
            double u[2][NV];
            const double* s0 = src_of(k, 0, zb, zc);
            if (((contig_mask >> k) & 1u) && ((reinterpret_cast<uintptr_t>(s0) & 15u) == 0)) {
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    const double2 d = *reinterpret_cast<const double2*>(s0 + v * lvs);
                    u[0][v] = d.x;
                    u[1][v] = d.y;
                }
            } else {
                const double* s1 = src_of(k, 1, zb, zc);
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    u[0][v] = s0[v * lvs];
                    u[1][v] = s1[v * lvs];
                }
            }
            if constexpr (std::is_same<T, float>::value) {
                // FP32: both cells' primitives and 1/rho, then one 8-byte store per array
                // (the pair's slots are adjacent and 2-element aligned). Measured on a B300:
                // FP32 flux +2.6 %; the FP64 and FF variants keep the per-cell stores
                // (FF -1 % with the pair held in registers).
                float W[2][NW];
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    float U[NV];
#pragma unroll
                    for (int v = 0; v < NV; ++v) U[v] = P<T>::in(u[e][v]);
                    prim_from_cons_as<Arith<T, 1>, T, NDIM>(U, W[e], W[e][NV], gm1);
                    if (zin && ((interior_mask >> (2 * k + e)) & 1u) && !(W[e][0] > 0.0f && W[e][NV - 1] > 0.0f))
                        atomicOr(m.err, 1);
                }
#pragma unroll
                for (int v = 0; v < NW; ++v)
                    *reinterpret_cast<float2*>(&w[v * R2N + 2 * q]) = make_float2(W[0][v], W[1][v]);
            } else {
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int c = 2 * q + e;
                    T U[NV], W[NV], r;
#pragma unroll
                    for (int v = 0; v < NV; ++v) U[v] = P<T>::in(u[e][v]);
                    prim_from_cons_as<Arith<T, 1>, T, NDIM>(U, W, r, gm1);
#pragma unroll
                    for (int v = 0; v < NV; ++v) P<T>::st(&w[v * R2N + c], W[v]);
                    P<T>::st(&w[NV * R2N + c], r);
                    if (zin && ((interior_mask >> (2 * k + e)) & 1u) && !(P<T>::pos(W[0]) && P<T>::pos(W[NV - 1])))
                        atomicOr(m.err, 1);
                }
            }
        }
    };

    // P: slopes, predictor and face states of the cell at R2 index c2 of plane
    // pzi; writes flo/fhi (face states on the low/high side along each axis).
    // P: slopes and predictor of the cell at R2 index c2 of plane pzi: its
    // primitives Wc, limited slopes dW and half-step state Wb.
    using A2 = Arith<T, 2>;      // arithmetic type of the predictor
    auto predict_core = [&](int pzi, int c2, A2 (&Wc)[NV], A2 (&dW)[3][NV], A2 (&Wb)[NV]) {
        using A = A2;
        const S* w = sW + slot_c * NW * R2N;
#pragma unroll
        for (int v = 0; v < NV; ++v) Wc[v] = as<A>(P<T>::ld(&w[v * R2N + c2]));
        const A rc = as<A>(P<T>::ld(&w[NV * R2N + c2]));
#pragma unroll
        for (int d = 0; d < NDIM; ++d) {
            const S* wm;
            const S* wp;
            int cm = c2, cp = c2;
            if (d == 0) { cm = c2 - 1; cp = c2 + 1; wm = w; wp = w; }
            else if (d == 1) { cm = c2 - R2X; cp = c2 + R2X; wm = w; wp = w; }
            else {
                wm = sW + slot_m * NW * R2N;
                wp = sW + slot_p * NW * R2N;
            }
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                const A dl = Wc[v] - as<A>(P<T>::ld(&wm[v * R2N + cm]));
                const A dr = as<A>(P<T>::ld(&wp[v * R2N + cp])) - Wc[v];
                dW[d][v] = minmod(dl, dr);
            }
        }
        if constexpr (RK) {                      // plain MUSCL: face states about Wc itself
#pragma unroll
            for (int v = 0; v < NV; ++v) Wb[v] = Wc[v];
            return;
        }
        const A gp = as<A>(g) * Wc[NV - 1];
        // The exact FP64 build (and the software-FP64 type) evaluates the
        // definition's expression tree; every other arithmetic the regrouped form.
        constexpr bool kRegroup = std::is_same<A, rd>::value ? kContract : !std::is_same<A, re>::value;
        if constexpr (kRegroup) {
            // Wc - sum_d hd_d A_d dW_d regrouped: every row has the advective
            // term sum_d (hd_d u_d) dW_d[v]; the density and pressure rows share
            // the divergence D = sum_d hd_d du_d (times rho, gamma p); velocity
            // row d adds hd_d dp_d / rho. 30 operations per 3D cell instead of
            // the definition's 40; the same value up to rounding.
            A t[NDIM];
            A D = as<A>(hd[0]) * dW[0][1];
#pragma unroll
            for (int d = 0; d < NDIM; ++d) {
                t[d] = as<A>(hd[d]) * Wc[1 + d];
                if (d > 0) D = D + as<A>(hd[d]) * dW[d][1 + d];
            }
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                Wb[v] = Wc[v];
#pragma unroll
                for (int d = 0; d < NDIM; ++d) Wb[v] = Wb[v] - t[d] * dW[d][v];
            }
            Wb[0] = Wb[0] - Wc[0] * D;
            Wb[NV - 1] = Wb[NV - 1] - gp * D;
#pragma unroll
            for (int d = 0; d < NDIM; ++d) Wb[1 + d] = Wb[1 + d] - rc * A(as<A>(hd[d]) * dW[d][NV - 1]);
        } else {
            A a[3][NV];
#pragma unroll
            for (int d = 0; d < NDIM; ++d) {
                const A un = Wc[1 + d], dun = dW[d][1 + d], dp = dW[d][NV - 1];
                a[d][0] = (un * dW[d][0]) + (Wc[0] * dun);
#pragma unroll
                for (int t = 0; t < NDIM; ++t)
                    a[d][1 + t] = (t == d) ? ((un * dun) + (dp * rc)) : (un * dW[d][1 + t]);
                a[d][NV - 1] = (gp * dun) + (un * dp);
            }
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                A s = as<A>(hd[0]) * a[0][v];
#pragma unroll
                for (int d = 1; d < NDIM; ++d) s = s + (as<A>(hd[d]) * a[d][v]);
                Wb[v] = Wc[v] - s;
            }
        }
    };
    // First-order fallback test: every face state's density and pressure positive.
    auto faces_ok = [&](const A2 (&dW)[3][NV], const A2 (&Wb)[NV]) {
        bool ok = true;
#pragma unroll
        for (int d = 0; d < NDIM; ++d) {
            const A2 h0 = P<A2>::half(dW[d][0]), hp = P<A2>::half(dW[d][NV - 1]);
            ok = ok && P<T>::pos(as<T>(Wb[0] - h0)) && P<T>::pos(as<T>(Wb[NV - 1] - hp)) &&
                 P<T>::pos(as<T>(Wb[0] + h0)) && P<T>::pos(as<T>(Wb[NV - 1] + hp));
        }
        return ok;
    };
    // Owner cells: every face state Wb -+ dW/2, or Wc on fallback. The x and
    // y face states of an inner plane go to shared memory as soon as they
    // are formed, beside the positivity test, and a cell that falls back
    // (rare) overwrites them with Wc: the same values end up in the same
    // places as with the test first, without the stores waiting for it.
    // The z face states stay in registers (zlo, zhi).
    auto predict_owner = [&](int pzi, bool inner, T (&zlo)[NV], T (&zhi)[NV]) {
        A2 Wc[NV], dW[3][NV], Wb[NV];
        predict_core(pzi, o2, Wc, dW, Wb);
        bool ok = true;
#pragma unroll
        for (int d = 0; d < NDIM; ++d) {
            T lo[NV], hi[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                const A2 hs = P<A2>::half(dW[d][v]);
                lo[v] = as<T>(Wb[v] - hs);
                hi[v] = as<T>(Wb[v] + hs);
            }
            ok = ok && P<T>::pos(lo[0]) && P<T>::pos(lo[NV - 1]) && P<T>::pos(hi[0]) && P<T>::pos(hi[NV - 1]);
            if (d < 2) {
                if (inner) {
#pragma unroll
                    for (int v = 0; v < NV; ++v) {
                        P<T>::st(&sFS[((2 * d) * NV + v) * R1N + o1], lo[v]);
                        P<T>::st(&sFS[((2 * d + 1) * NV + v) * R1N + o1], hi[v]);
                    }
                }
            } else {
#pragma unroll
                for (int v = 0; v < NV; ++v) { zlo[v] = lo[v]; zhi[v] = hi[v]; }
            }
        }
        if (!ok) {
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                const T w = as<T>(Wc[v]);
                if (inner) {
#pragma unroll
                    for (int f = 0; f < 4; ++f) P<T>::st(&sFS[(f * NV + v) * R1N + o1], w);
                }
                zlo[v] = w;
                zhi[v] = w;
            }
        }
    };
    // Ring cells: only the one x or y face state the tile needs (face 0..3 =
    // x-, x+, y-, y+), the same values the owner of that cell would form.
    auto predict_face = [&](int pzi, int c2, int face, T (&out)[NV]) {
        A2 Wc[NV], dW[3][NV], Wb[NV];
        predict_core(pzi, c2, Wc, dW, Wb);
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            const A2 hs = P<A2>::half(face < 2 ? dW[0][v] : dW[1][v]);
            out[v] = as<T>(Wb[v] + ((face & 1) ? hs : -hs));     // Wb + hs or Wb - hs, same bits
        }
        if (!faces_ok(dW, Wb)) {
#pragma unroll
            for (int v = 0; v < NV; ++v) out[v] = as<T>(Wc[v]);
        }
    };

    // z state carried by the owner: high-z face state of the previous plane,
    // its low-z face flux, and its x+y flux-difference sum. FP64 and FP32-flux
    // paths: the sum in FP64 from the face fluxes promoted to FP64, as the
    // definition writes it. FP32-flux shortcut (FX): each difference
    // c_d (F_hi - F_lo) of FP32 face fluxes is
    // formed exactly (two_sum) and scaled by c_d held as a float pair, and the
    // x, y, z terms are summed as float-float (about 46 bits); only the final
    // U+ = U - (sum) is FP64 arithmetic. The same face value enters both cells,
    // so the sum still telescopes to ~1e-14 of each term.
    // FF path: the differences and their c_d scaling and sum are double-word,
    // the final U+ = U - (sum) FP64.
    static_assert(!FX || std::is_same<T, float>::value, "the shortcut update exists for FP32 fluxes only");
    constexpr bool F32 = std::is_same<T, float>::value && FX;     // float-float flux sums
    using SpeedT = typename std::conditional<F32, float, rd>::type;   // signal-speed rule of the new state
    constexpr bool DW = std::is_same<T, dw>::value;
    // the signal-speed filter (SpeedBound): FP64 speeds, one-step task only
    unsigned long long smaxb = 0ull;   // bits of the largest signal speed
    constexpr bool kFilter = std::is_same<SpeedT, rd>::value && IO::kFilter;
    const SpeedBound sbf = kFilter ? speed_bound_setup(m, dt) : SpeedBound{};
    unsigned long long subb = 0ull;    // bits of the largest bound of a skipped cell
    auto raise_speed = [&](const rd (&Un)[NV]) {
        if constexpr (kFilter) {
            float ub;
            if (sbf.thr > 0.0f && speed_upper<NDIM>(sbf, Un, ub) && ub < sbf.thr) {
                subb = umax64(subb, (unsigned long long)__double_as_longlong(to_f64(ub)));
                return;
            }
        }
        smaxb = umax64(smaxb, new_state_speed<SpeedT, NDIM>(m, Un));
    };
    T zp_prev[NV], Fz_prev[NV];
    double acc_prev[NV];
    ff acc_ff[NV];
    dw acc_dw[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        zp_prev[v] = P<T>::zero();
        Fz_prev[v] = P<T>::zero();
        acc_prev[v] = 0.0;
        acc_ff[v] = {0.0f, 0.0f};
        acc_dw[v] = {0.0f, 0.0f};
    }
    dw cdw[3];                           // c_d as double-words (FF path)
#pragma unroll
    for (int d = 0; d < 3; ++d) cdw[d] = DW ? P<dw>::in(cd[d]) : dw{0.0f, 0.0f};
    float ch[3], cl[3];                  // c_d = dt/dx_d as float pairs (FP32-flux shortcut)
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        ch[d] = d2f_rn(cd[d]);
        cl[d] = F32 ? d2f_rn(__dsub_rn(cd[d], to_f64(ch[d]))) : 0.0f;
    }

    // base value of the owner's cell of plane q (gi: its offset in the block
    // column, GlobalIO), where its new value goes, and whether its signal
    // speed counts (see the IO policies)
    auto cell_base = [&](int q, long long gi) -> const double* {
        if constexpr (IO::kIn) return io.scratch + (long long)scratch_slot(q) * NV * R2N + o2;
        if constexpr (IO::kOut) {
            int zb, zc;
            plane_z(q, zb, zc);
            return Uin + (long long)(own_b + zb) * m.blk_stride + (own_o + zc);
        }
        return Ub + gi;
    };
    auto store_new = [&](int q, long long gi, int v, double x) {
        if constexpr (IO::kOut) io.scratch[((long long)scratch_slot(q) * NV + v) * NT + tid] = x;
        else Ob[gi + v * vs] = x;
    };
    auto raise_here = [&](int q) -> bool {
        if constexpr (IO::kRaise == 1) return !RK || stage == 2;
        if constexpr (IO::kRaise == 2)        // the fused item's own cells, not its halo
            return ti >= 2 && ti < TX - 2 && tj >= 2 && tj < TY - 2 && (NDIM != 3 || (q >= z0 + 2 && q < z1 - 2));
        return false;
    };

    const int pbeg = (NDIM == 3) ? z0 - 1 : 0, pend = (NDIM == 3) ? z1 : 0;
    if (NDIM == 3) {
        if (Prefetch<T>::value) { prefetch_plane(z0 - 1); prefetch_plane(z0); }
        slot_m = ring_slot(z0 - 2);
        slot_c = ring_slot(z0 - 1);
        slot_p = ring_slot(z0);
        load_plane(z0 - 2, slot_m);
        load_plane(z0 - 1, slot_c);
    }

    for (int p = pbeg; p <= pend; ++p) {
        if (NDIM == 3) {
            slot_m = ring_slot(p - 1);
            slot_c = ring_slot(p);
            slot_p = ring_slot(p + 1);
        }
        const bool inner = p >= z0 && p < z1;      // plane p is updated here: it has x/y faces to flux
        if (NDIM == 3) {
            if (Prefetch<T>::value && p < pend) prefetch_plane(p + 2);   // planes up to pend + 1 are loaded
            load_plane(p + 1, slot_p);
        }
        else load_plane(0, 0);
        __syncthreads();

        // ---- P: predict
        T zlo[NV], zhi[NV];
        if (owner) predict_owner(p, inner, zlo, zhi);
        // ring cells: the one face state the tile reads, the same bits as the
        // owner of that cell forms (the FP64 operations and their fusion are
        // fixed by the source, so both evaluations agree)
        if (inner && ringer) {
            T fs[NV];
            predict_face(p, rc2, rface, fs);
#pragma unroll
            for (int v = 0; v < NV; ++v) P<T>::st(&sFS[(rface * NV + v) * R1N + rc1], fs[v]);
        }
        __syncthreads();

        // ---- F: x and y face fluxes of plane p
        if (inner) {
            for (int f = member ? tid : Tl::NXF + Tl::NYF; f < Tl::NXF + Tl::NYF; f += NB) {
                // the face's left state (face array x+ or y+, where its flux
                // goes too) and right state (x- or y-), and the slots of the
                // normal and first tangential velocity: (rho, u_n, u_t..., p)
                const bool ynrm = f >= Tl::NXF;
                S* pl;
                const S* pr;
                int on, ot;
                if (!ynrm) {
                    const int fi = f % (TX + 1), fj = f / (TX + 1);
                    pl = sGx + (fj + 1) * R1X + fi;
                    pr = pl - (NV * R1N - 1);
                    on = R1N; ot = 2 * R1N;
                } else {
                    const int f2 = f - Tl::NXF;
                    const int fi = f2 % TX, fj = f2 / TX;
                    pl = sGy + fj * R1X + fi + 1;
                    pr = pl - (NV * R1N - R1X);
                    on = 2 * R1N; ot = R1N;
                }
                T L[NV], R[NV], F[NV];
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    const int o = v == 1 ? on : (v == 2 ? ot : v * R1N);
                    L[v] = P<T>::ld(pl + o);
                    R[v] = P<T>::ld(pr + o);
                }
                hll<T, NDIM, false>(L, R, F, g, igm1);
#pragma unroll
                for (int v = 0; v < NV; ++v) P<T>::st(pl + (v == 1 ? on : (v == 2 ? ot : v * R1N)), F[v]);
            }
        }
        __syncthreads();

        // ---- U: z flux, update of the finished plane, x+y sums of this plane
        if (NDIM == 3) {
            T Fz[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) Fz[v] = P<T>::zero();
            if (owner && p >= z0) {
                T L[NV], R[NV];
                L[0] = zp_prev[0]; L[1] = zp_prev[3]; L[2] = zp_prev[1]; L[3] = zp_prev[2]; L[4] = zp_prev[4];
                R[0] = zlo[0]; R[1] = zlo[3]; R[2] = zlo[1]; R[3] = zlo[2]; R[4] = zlo[4];
                T F[NV];
                hll<T, NDIM, true>(L, R, F, g, igm1);
                Fz[0] = F[0]; Fz[3] = F[1]; Fz[1] = F[2]; Fz[2] = F[3]; Fz[4] = F[4];
                if constexpr (IO::kReg) {      // the block's low (p = 0) and high (p = bz) z faces
                    if (p == 0 || p == bz) {
                        double* r = io.reg + ((long long)blk * 6 + (p == 0 ? 4 : 5)) * NV * io.fsz +
                                    ((y0 + tj) * m.bs[0] + (x0 + ti));
#pragma unroll
                        for (int v = 0; v < NV; ++v) r[(long long)v * io.fsz] = P<T>::to_double(Fz[v]);
                    }
                }
            }
            if (p >= z0 + 1) {
                // plane q of the column: block qb above blk, in-block plane ql
                const int q = p - 1, qb = q >> lgbz, ql = q & (bz - 1);
                if (owner) {
                    const long long gi = (long long)qb * nbxy * m.blk_stride +
                                         ((long long)(ql + kGuard) * py + (y0 + tj + kGuard)) * px + (x0 + ti + kGuard);
                    const double* ub = cell_base(q, gi);
                    const long long bvs = IO::kIn ? (long long)R2N : vs;
                    rd Un[NV];
#pragma unroll
                    for (int v = 0; v < NV; ++v) {
                        if constexpr (F32) {
                            const ff tz = ff_scale(ff_diff(Fz[v], Fz_prev[v]), ch[2], cl[2]);
                            Un[v] = rd(ub[v * bvs]) - rd(ff_to_double(ff_add(acc_ff[v], tz)));
                        } else if constexpr (DW) {
                            const dw tz = cdw[2] * (Fz[v] - Fz_prev[v]);
                            Un[v] = rd(ub[v * bvs]) - rd(P<dw>::to_double(acc_dw[v] + tz));
                        } else {
                            const rd acc = rd(acc_prev[v]) +
                                           rd(cd[2]) * (rd(P<T>::to_double(Fz[v])) - rd(P<T>::to_double(Fz_prev[v])));
                            Un[v] = rd(ub[v * bvs]) - acc;
                        }
                        // Heun stage 2: the average with the step's initial state, in FP64
                        if (RK && stage == 2) Un[v] = P<rd>::half(rd((IO::kIn ? Ub : Ob)[gi + v * vs]) + Un[v]);
                        store_new(q, gi, v, Un[v].v);
                    }
                    if (raise_here(q)) raise_speed(Un);
                }
                // leaving a block (or the item's range): raise its signal speed
                // (CTA-uniform: every thread takes part, non-owners with 0)
                if (IO::kRaise == 1 && (!RK || stage == 2) && (q == z1 - 1 || ql == bz - 1)) {
                    if (kFilter && m.sub) {
                        cta_raise_smax2(smaxb, subb, red, &m.smax[blk + qb * nbxy], &m.sub[blk + qb * nbxy]);
                        subb = 0ull;
                    } else {
                        cta_raise_smax(__longlong_as_double((long long)smaxb), red, &m.smax[blk + qb * nbxy]);
                    }
                    smaxb = 0ull;
                }
            }
            if (owner) {
#pragma unroll
                for (int v = 0; v < NV; ++v) { zp_prev[v] = zhi[v]; Fz_prev[v] = Fz[v]; }
            }
        }
        if constexpr (IO::kReg) {             // the block's x and y faces in plane p
            if (inner && owner) {
                const int i = x0 + ti, j = y0 + tj, k = (NDIM == 3) ? p : 0;
                const long long rb = (long long)blk * 6 * NV * io.fsz;
                auto put = [&](int face, const S* src, int t) {
                    double* r = io.reg + rb + (long long)face * NV * io.fsz + t;
#pragma unroll
                    for (int v = 0; v < NV; ++v) r[(long long)v * io.fsz] = P<T>::to_double(P<T>::ld(&src[v * R1N]));
                };
                if (i == 0) put(0, sGx + o1 - 1, k * m.bs[1] + j);
                if (i == m.bs[0] - 1) put(1, sGx + o1, k * m.bs[1] + j);
                if (j == 0) put(2, sGy + o1 - R1X, k * m.bs[0] + i);
                if (j == m.bs[1] - 1) put(3, sGy + o1, k * m.bs[0] + i);
            }
        }
        if (inner && owner) {
            // x then y flux differences of plane p
            // high x face of the cell at o1, low x face at o1 - 1; high y face at o1, low at o1 - R1X
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                if constexpr (F32) {
                    const ff tx = ff_scale(ff_diff(sGx[v * R1N + o1], sGx[v * R1N + o1 - 1]), ch[0], cl[0]);
                    const ff ty = ff_scale(ff_diff(sGy[v * R1N + o1], sGy[v * R1N + o1 - R1X]), ch[1], cl[1]);
                    acc_ff[v] = ff_add(tx, ty);
                } else if constexpr (DW) {
                    const dw tx = cdw[0] * (P<T>::ld(&sGx[v * R1N + o1]) - P<T>::ld(&sGx[v * R1N + o1 - 1]));
                    const dw ty = cdw[1] * (P<T>::ld(&sGy[v * R1N + o1]) - P<T>::ld(&sGy[v * R1N + o1 - R1X]));
                    acc_dw[v] = tx + ty;
                } else {
                    acc_prev[v] = (rd(cd[0]) * (rd(P<T>::to_double(P<T>::ld(&sGx[v * R1N + o1]))) -
                                                rd(P<T>::to_double(P<T>::ld(&sGx[v * R1N + o1 - 1])))) +
                                   rd(cd[1]) * (rd(P<T>::to_double(P<T>::ld(&sGy[v * R1N + o1]))) -
                                                rd(P<T>::to_double(P<T>::ld(&sGy[v * R1N + o1 - R1X])))))
                                      .v;
                }
            }
            if (NDIM == 2) {
                const long long gi = ((long long)(y0 + tj + kGuard)) * px + (x0 + ti + kGuard);
                const double* ub = cell_base(0, gi);
                const long long bvs = IO::kIn ? (long long)R2N : vs;
                rd Un[NV];
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    if constexpr (F32) Un[v] = rd(ub[v * bvs]) - rd(ff_to_double(acc_ff[v]));
                    else if constexpr (DW) Un[v] = rd(ub[v * bvs]) - rd(P<dw>::to_double(acc_dw[v]));
                    else Un[v] = rd(ub[v * bvs]) - rd(acc_prev[v]);
                    if (RK && stage == 2) Un[v] = P<rd>::half(rd((IO::kIn ? Ub : Ob)[gi + v * vs]) + Un[v]);
                    store_new(0, gi, v, Un[v].v);
                }
                if (raise_here(0)) raise_speed(Un);
            }
        }
    }
    if constexpr (NDIM == 2) {
        if (IO::kRaise == 1 && (!RK || stage == 2)) {
            if (kFilter && m.sub) cta_raise_smax2(smaxb, subb, red, &m.smax[blk], &m.sub[blk]);
            else cta_raise_smax(__longlong_as_double((long long)smaxb), red, &m.smax[blk]);
        }
    }
    if constexpr (IO::kRaise == 2) cta_raise_smax(__longlong_as_double((long long)smaxb), red, &io.smax2[blk]);
}

// Packet path: one CTA per (packet block, column tile); guards come from the
// padded block.
template <int NDIM, int TX, int TY, class T, bool RK = false, bool FX = false, class IO = GlobalIO>
__global__ void __launch_bounds__(Tile<NDIM, TX, TY>::template nb<T, RK>())
hydro_kernel(const MeshDev m, const int* __restrict__ blk_ids, int tiles_x, int tiles_y,
             const double* __restrict__ Uin, double* __restrict__ Uout, int stage, IO io) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ unsigned long long red[32];
    const int ntile = tiles_x * tiles_y;
    const int blk = blk_ids[blockIdx.x / ntile];
    const int tile = blockIdx.x % ntile;
    hydro_tile<NDIM, TX, TY, T, false, RK, FX, IO>(m, blk, (tile % tiles_x) * TX, (tile / tiles_x) * TY, Uin, Uout,
                                               smem_raw, red, 0, -1, stage, io);
}

}  // namespace orcha
