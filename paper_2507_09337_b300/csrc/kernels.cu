// kernels.cu -- guard fill, pack/unpack, signal speed and dt reduction, and
// the launch table of the hydro kernel variants.
#include <cstdio>

#include "common.cuh"
#include "hydro.cuh"
#include "launch.h"
#include "persistent.cuh"
#include "softfp64.cuh"

namespace orcha {

// ---------------------------------------------------------------- guard fill
// Guard cells of block b (padded index outside the interior box) take the
// value of the global cell at the same position, with the boundary rule on
// the domain edge: outflow clamps the index to [0, N-1] on each axis
// (zero-gradient; faces, edges and corners alike), periodic wraps it. The
// source is always an interior cell of some block in the same buffer, so
// guard writes never race with the reads.
__device__ __forceinline__ int map_axis(int gi, int n, int periodic) {
    if (periodic) { gi %= n; return gi < 0 ? gi + n : gi; }
    return gi < 0 ? 0 : (gi > n - 1 ? n - 1 : gi);
}

__global__ void guard_fill_kernel(const MeshDev m, const int* __restrict__ blk_ids, double* __restrict__ U) {
    const int npad = (int)m.var_stride;                  // a padded block has at most 36^3 cells
    const int pb = blockIdx.y;
    const int blk = blk_ids[pb];
    const int b[3] = {blk % m.nb[0], (blk / m.nb[0]) % m.nb[1], blk / (m.nb[0] * m.nb[1])};
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < npad; c += gridDim.x * blockDim.x) {
        const int r = c / m.pad[0];
        int loc[3] = {c % m.pad[0], r % m.pad[1], r / m.pad[1]};
        bool guard = false;
        int src_blk[3], src_loc[3];
        for (int d = 0; d < 3; ++d) {
            if (d >= m.ndim) { src_blk[d] = 0; src_loc[d] = 0; continue; }
            const int li = loc[d] - kGuard;                 // interior-relative index
            if (li < 0 || li >= m.bs[d]) guard = true;
            const int n = m.nb[d] * m.bs[d];
            const int gi = map_axis(b[d] * m.bs[d] + li, n, m.periodic[d]);
            src_blk[d] = gi / m.bs[d];
            src_loc[d] = gi % m.bs[d] + kGuard;
        }
        if (!guard) continue;
        const long long sb = src_blk[0] + (long long)m.nb[0] * (src_blk[1] + (long long)m.nb[1] * src_blk[2]);
        const int sz = (m.ndim == 3) ? src_loc[2] : 0;
        const long long so = sb * m.blk_stride + ((long long)sz * m.pad[1] + src_loc[1]) * m.pad[0] + src_loc[0];
        const long long dof = (long long)blk * m.blk_stride + c;
        for (int v = 0; v < m.nvar; ++v) U[dof + v * npad] = U[so + v * npad];
    }
}

// ---------------------------------------------------------------- pack / unpack
// Interior array [block][var][k][j][i] <-> padded state interior. One CTA per
// (block, var) plane; in-block cell indices are 32-bit (a block has at most
// 32^3 cells). Block sizes are 8, 16 or 32 (1 on an inactive axis; the mesh
// descriptor is rejected otherwise), so the cell index splits by masks and
// shifts instead of integer divisions.
__device__ __forceinline__ void cell_ijk(const MeshDev& m, int c, int& i, int& j, int& k) {
    const int r = c >> (__ffs(m.bs[0]) - 1);
    i = c & (m.bs[0] - 1);
    j = r & (m.bs[1] - 1);
    k = r >> (__ffs(m.bs[1]) - 1);
}
__device__ __forceinline__ int cell_offset(const MeshDev& m, int c) {
    int i, j, k;
    cell_ijk(m, c, i, j, k);
    const int kk = (m.ndim == 3) ? k + kGuard : 0;
    return (kk * m.pad[1] + (j + kGuard)) * m.pad[0] + (i + kGuard);
}

// plane p = block * nvar + var of the packed array; dst block `blk`
__global__ void pack_kernel(const MeshDev m, const double* __restrict__ interior, double* __restrict__ U) {
    const int ncell = m.bs[0] * m.bs[1] * m.bs[2];
    const long long p = blockIdx.x;
    const double* src = interior + p * ncell;
    double* dst = U + p * m.var_stride;
    for (int c = threadIdx.x; c < ncell; c += blockDim.x) dst[cell_offset(m, c)] = src[c];
}

__global__ void unpack_kernel(const MeshDev m, const double* __restrict__ U, double* __restrict__ interior) {
    const int ncell = m.bs[0] * m.bs[1] * m.bs[2];
    const long long p = blockIdx.x;
    const double* src = U + p * m.var_stride;
    double* dst = interior + p * ncell;
    for (int c = threadIdx.x; c < ncell; c += blockDim.x) dst[c] = src[cell_offset(m, c)];
}

// The same for the blocks of one packet: `interior` holds them in packet
// order, [packet position][var][k][j][i]; plane p = position * nvar + var.
__global__ void pack_ids_kernel(const MeshDev m, const int* __restrict__ ids, int n,
                                const double* __restrict__ interior, double* __restrict__ U) {
    const int ncell = m.bs[0] * m.bs[1] * m.bs[2];
    const long long p = blockIdx.x;
    const long long pos = p / m.nvar, v = p % m.nvar;
    const double* src = interior + p * ncell;
    double* dst = U + (long long)ids[pos] * m.blk_stride + v * m.var_stride;
    for (int c = threadIdx.x; c < ncell; c += blockDim.x) dst[cell_offset(m, c)] = src[c];
}

__global__ void unpack_ids_kernel(const MeshDev m, const int* __restrict__ ids, int n, const double* __restrict__ U,
                                  double* __restrict__ interior) {
    const int ncell = m.bs[0] * m.bs[1] * m.bs[2];
    const long long p = blockIdx.x;
    const long long pos = p / m.nvar, v = p % m.nvar;
    const double* src = U + (long long)ids[pos] * m.blk_stride + v * m.var_stride;
    double* dst = interior + p * ncell;
    for (int c = threadIdx.x; c < ncell; c += blockDim.x) dst[c] = src[cell_offset(m, c)];
}

// ---------------------------------------------------------------- signal speed of the current state
__global__ void signal_speed_kernel(const MeshDev m, const int* __restrict__ blk_ids, const double* __restrict__ U) {
    __shared__ unsigned long long red[32];
    const int blk = blk_ids[blockIdx.x];
    const unsigned long long b = block_signal_speed(m, blk, U);
    cta_raise_smax(__longlong_as_double((long long)b), red, &m.smax[blk]);
}

// Every block of the mesh, one CTA per block (no block-id list); F32: the
// FP32-flux variant's signal-speed rule.
template <bool F32>
__global__ void signal_speed_all_kernel(const MeshDev m, const double* __restrict__ U) {
    __shared__ unsigned long long red[32];
    const int blk = blockIdx.x;
    const unsigned long long b = F32 ? block_signal_speed_f32(m, blk, U, blockIdx.y, gridDim.y)
                                     : block_signal_speed(m, blk, U, blockIdx.y, gridDim.y);
    cta_raise_smax(__longlong_as_double((long long)b), red, &m.smax[blk]);     // max: any chunk order
}

// ---------------------------------------------------------------- first CFL time step, filtered
// The first dt of a state needs the largest FP64 signal speed over all its
// cells and has no previous maximum to filter against (hydro.cuh, signal-
// speed filter). Pass 1 takes every cell's rigorous FP32 bounds lb <= s <= ub
// of its FP64 speed s (speed_bounds, below), or s itself where they do not apply,
// and raises the block's largest ub (m.sub), the exactly evaluated speeds
// (m.smax) and the state's largest lb or exact speed (*lbmax). That is at
// most the largest speed, so a cell with ub < *lbmax cannot hold it: pass 2
// evaluates in FP64 only the cells with ub >= *lbmax, in the blocks whose
// m.sub reaches it. The maximum over m.smax is then the maximum over every
// cell, bit for bit, and the non-physical flag is raised as by the full
// evaluation (a cell whose bounds apply has a positive FP64 pressure).
// The lower-side constants of the bounds: gamma and 1/dx_d rounded down.
struct SpeedBoundLo {
    float g_lo, idx_lo[3];
};
__device__ __forceinline__ SpeedBoundLo speed_bound_lo_setup(const MeshDev& m) {
    SpeedBoundLo b;
    b.g_lo = __double2float_rd(m.gamma);
    for (int d = 0; d < 3; ++d) b.idx_lo[d] = __double2float_rd(m.idx[d]);
    return b;
}

// The upper bound ub of speed_upper (hydro.cuh; the same operations, so the
// same bits) and a lower bound lb <= the FP64 signal speed of Un: the mirror
// of the upper bound's steps, every operation rounded down (|m_d| / rho from
// the truncated |m_d| times 1/rho rounded down, the pressure's lower bound
// pl, sqrt(gamma pl / rho) rounded down, the sum times 1/dx_d rounded down),
// divided by `margin`, which covers the FP64 evaluation's own rounding on
// this side as on the other. False where the bounds do not apply (the
// conditions of speed_upper).
template <int NDIM>
__device__ __forceinline__ bool speed_bounds(const SpeedBound& sb, const SpeedBoundLo& sl, const rd* Un, float& lb,
                                             float& ub) {
    constexpr int NV = NDIM + 2;
    constexpr float kUp = 0x1.000002p0f;
    float rl, el, ml[NDIM];
    bool ok = mag_f32_rz(Un[0].v, rl) && mag_f32_rz(Un[NV - 1].v, el) && __double_as_longlong(Un[0].v) > 0 &&
              __double_as_longlong(Un[NV - 1].v) > 0;
#pragma unroll
    for (int d = 0; d < NDIM; ++d) ok = mag_f32_rz(Un[1 + d].v, ml[d]) && ok;
    if (!ok) return false;
    const float rh = __fmul_ru(rl, kUp), eh = __fmul_ru(el, kUp);
    const float ri_hi = __frcp_ru(rl), ri_lo = __frcp_rd(rh);
    float kel = 0.0f, keh = 0.0f, ah[NDIM], al[NDIM];
#pragma unroll
    for (int d = 0; d < NDIM; ++d) {
        const float mh = __fmul_ru(ml[d], kUp);
        ah[d] = __fmul_ru(mh, ri_hi);
        al[d] = __fmul_rd(ml[d], ri_lo);                             // <= |m_d| / rho
        kel = __fadd_rd(kel, __fmul_rd(ml[d], __fmul_rd(ml[d], ri_lo)));
        keh = __fadd_ru(keh, __fmul_ru(mh, ah[d]));
    }
    kel = 0.5f * kel;
    keh = 0.5f * keh;
    const float pl = __fmul_rd(sb.gm1_lo, __fadd_rd(el, -keh));
    if (!(pl > eh * 0x1p-40f)) return false;
    const float ph = __fmul_ru(sb.gm1_hi, __fadd_ru(eh, -kel));
    const float ch = __fsqrt_ru(__fmul_ru(__fmul_ru(sb.g_hi, ph), ri_hi));
    const float cl = __fsqrt_rd(__fmul_rd(__fmul_rd(sl.g_lo, pl), ri_lo));   // <= sqrt(gamma p / rho)
    float s = 0.0f, t = 0.0f;
#pragma unroll
    for (int d = 0; d < NDIM; ++d) {
        s = __fadd_ru(s, __fmul_ru(__fadd_ru(ah[d], ch), sb.idx_hi[d]));
        t = __fadd_rd(t, __fmul_rd(__fadd_rd(al[d], cl), sl.idx_lo[d]));
    }
    ub = __fmul_ru(s, sb.margin);
    lb = __fdiv_rd(t, sb.margin);
    return true;
}

template <int NDIM>
__device__ __forceinline__ void cell_state(const MeshDev& m, const double* __restrict__ Ub, int c, rd (&Un)[NDIM + 2]) {
    int i, j, k;
    cell_ijk(m, c, i, j, k);
    const int kk = (NDIM == 3) ? k + kGuard : 0;
    const int po = (kk * m.pad[1] + (j + kGuard)) * m.pad[0] + (i + kGuard);
#pragma unroll
    for (int v = 0; v < NDIM + 2; ++v) Un[v] = rd(Ub[po + v * m.var_stride]);
}

template <int NDIM>
__global__ void first_dt_bounds_kernel(const MeshDev m, const double* __restrict__ U,
                                       unsigned long long* __restrict__ lbmax) {
    __shared__ unsigned long long red[32];
    const int blk = blockIdx.x;
    const double* Ub = U + (long long)blk * m.blk_stride;
    const int ncell = m.bs[0] * m.bs[1] * m.bs[2];
    const SpeedBound sb = speed_bound_setup(m, 1.0);
    const SpeedBoundLo sl = speed_bound_lo_setup(m);
    float ubm = 0.0f, lbm = 0.0f;
    unsigned long long em = 0ull;        // bits of the largest exactly evaluated speed
    for (int c = blockIdx.y * blockDim.x + threadIdx.x; c < ncell; c += gridDim.y * blockDim.x) {
        rd Un[NDIM + 2];
        cell_state<NDIM>(m, Ub, c, Un);
        float lb, ub;
        if (speed_bounds<NDIM>(sb, sl, Un, lb, ub)) {
            ubm = fmaxf(ubm, ub);
            lbm = fmaxf(lbm, lb);
        } else {
            em = umax64(em, new_state_speed<rd, NDIM>(m, Un));
        }
    }
    const unsigned long long ubb = (unsigned long long)__double_as_longlong((double)ubm);
    const unsigned long long lbb = umax64((unsigned long long)__double_as_longlong((double)lbm), em);
    cta_raise_smax2(ubb, em, red, &m.sub[blk], &m.smax[blk]);
    __syncthreads();
    cta_raise_smax(__longlong_as_double((long long)lbb), red, lbmax);
}

template <int NDIM>
__global__ void first_dt_eval_kernel(const MeshDev m, const double* __restrict__ U,
                                     const unsigned long long* __restrict__ lbmax) {
    __shared__ unsigned long long red[32];
    const int blk = blockIdx.x;
    const unsigned long long L = *lbmax;
    if (m.sub[blk] < L) return;          // the whole CTA: no cell of this block reaches L
    const double* Ub = U + (long long)blk * m.blk_stride;
    const int ncell = m.bs[0] * m.bs[1] * m.bs[2];
    const SpeedBound sb = speed_bound_setup(m, 1.0);
    unsigned long long em = 0ull;
    for (int c = blockIdx.y * blockDim.x + threadIdx.x; c < ncell; c += gridDim.y * blockDim.x) {
        rd Un[NDIM + 2];
        cell_state<NDIM>(m, Ub, c, Un);
        float ub;      // cells without bounds were evaluated by pass 1
        if (speed_upper<NDIM>(sb, Un, ub) && (unsigned long long)__double_as_longlong((double)ub) >= L)
            em = umax64(em, new_state_speed<rd, NDIM>(m, Un));
    }
    cta_raise_smax(__longlong_as_double((long long)em), red, &m.smax[blk]);
}

// ---------------------------------------------------------------- dt reduction
// dt = cfl / max over blocks; then clear the per-block maxima for the next step.
__global__ void dt_reduce_kernel(const MeshDev m, int nblk, double* __restrict__ dt) {
    __shared__ unsigned long long red[32];
    unsigned long long b = 0;
    for (int i = threadIdx.x; i < nblk; i += blockDim.x) b = umax64(b, m.smax[i]);
    b = warp_max_u64(b);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = b;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = umax64(t, red[w]);
        const double s = __longlong_as_double((long long)t);
        if (s > 0.0 && s <= 1.7976931348623157e308) *dt = m.cfl / s;
        else atomicOr(m.err, 2);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nblk; i += blockDim.x) m.smax[i] = 0ull;
}

// ---------------------------------------------------------------- synthetic state (autotuning)
// A smooth, everywhere-physical state computed from the cell position alone:
// rho = 1 + 0.2 sin(2 pi (x + 2y + 3z)), u_d = 0.3 cos(2 pi (d + 1) x_d), p = 1 + 0.1 cos(...).
__global__ void synthetic_state_kernel(const MeshDev m, double* __restrict__ U) {
    const long long ncell = (long long)m.bs[0] * m.bs[1] * m.bs[2];
    const long long total = (long long)m.nb[0] * m.nb[1] * m.nb[2] * ncell;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long blk = e / ncell, c = e % ncell;
        const int l[3] = {(int)(c % m.bs[0]), (int)((c / m.bs[0]) % m.bs[1]), (int)(c / ((long long)m.bs[0] * m.bs[1]))};
        const int b[3] = {(int)(blk % m.nb[0]), (int)((blk / m.nb[0]) % m.nb[1]), (int)(blk / ((long long)m.nb[0] * m.nb[1]))};
        double x[3];
        for (int d = 0; d < 3; ++d) x[d] = (b[d] * m.bs[d] + l[d] + 0.5) / (double)(m.nb[d] * m.bs[d]);
        const double ph = 6.283185307179586 * (x[0] + 2.0 * x[1] + (m.ndim == 3 ? 3.0 * x[2] : 0.0));
        const double rho = 1.0 + 0.2 * sin(ph), p = 1.0 + 0.1 * cos(ph);
        double ke = 0.0, mom[3];
        for (int d = 0; d < m.ndim; ++d) {
            const double u = 0.3 * cos(6.283185307179586 * (d + 1) * x[d]);
            mom[d] = rho * u;
            ke += 0.5 * rho * u * u;
        }
        const int kk = (m.ndim == 3) ? l[2] + kGuard : 0;
        const long long po = blk * m.blk_stride + ((long long)kk * m.pad[1] + (l[1] + kGuard)) * m.pad[0] + (l[0] + kGuard);
        U[po] = rho;
        for (int d = 0; d < m.ndim; ++d) U[po + (1 + d) * m.var_stride] = mom[d];
        U[po + (m.nvar - 1) * m.var_stride] = p * m.igm1 + ke;
    }
}

cudaError_t launch_synthetic_state(const MeshDev& m, double* U, cudaStream_t st) {
    synthetic_state_kernel<<<148 * 8, 256, 0, st>>>(m, U);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- two-region initial state (serving recipes)
// Cell (gi, gj, gk) is "inside" when, in half-cell units (centre of cell g at
// 2g + 1), sum_d (2 g_d + 1 - c2_d)^2 <= r2 (kind 1, sphere), or when g_axis <
// split (kind 2, half-space). Inside cells take u_in, others u_out: the
// region test is integer arithmetic and the states are given, so the values
// are exact and match any other implementation of the same rule.
__global__ void region_init_kernel(const MeshDev m, double* __restrict__ U, int kind, int4 reg, RegionStates rs) {
    const int ncell = m.bs[0] * m.bs[1] * m.bs[2];
    const int blk = blockIdx.x;
    const int b[3] = {blk % m.nb[0], (blk / m.nb[0]) % m.nb[1], blk / (m.nb[0] * m.nb[1])};
    double* Ub = U + (long long)blk * m.blk_stride;
    for (int c = blockIdx.y * blockDim.x + threadIdx.x; c < ncell; c += gridDim.y * blockDim.x) {
        int l[3];
        cell_ijk(m, c, l[0], l[1], l[2]);
        long long g[3];
        for (int d = 0; d < 3; ++d) g[d] = (long long)b[d] * m.bs[d] + l[d];
        bool in;
        if (kind == 1) {
            const long long c2[3] = {reg.x, reg.y, reg.z};
            long long d2 = 0;
            for (int d = 0; d < m.ndim; ++d) {
                const long long t = 2 * g[d] + 1 - c2[d];
                d2 += t * t;
            }
            in = d2 <= (long long)reg.w;
        } else {
            in = g[reg.x] < reg.y;
        }
        const int po = cell_offset(m, c);
        for (int v = 0; v < m.nvar; ++v) Ub[po + v * m.var_stride] = in ? rs.in[v] : rs.out[v];
    }
}

// Totals of each conserved variable over the interior cells in a fixed
// order, so the result depends only on the state: pass 1 sums each block
// (one CTA per block: per-thread strided sums, then a fixed tree) into
// partial[blk][v]; pass 2 (one CTA) sums the partials in block order.
__global__ void block_totals_kernel(const MeshDev m, const double* __restrict__ U, double* __restrict__ partial) {
    __shared__ double red[256];
    const int blk = blockIdx.x;
    const int ncell = m.bs[0] * m.bs[1] * m.bs[2];
    {
        const int v = blockIdx.y;                    // one CTA per (block, variable)
        // four independent partial sums per thread (cells c, c + 256, c + 512,
        // c + 768 of each stride of 1024), added in a fixed order: the loads
        // of a thread are in flight together instead of one after another
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
        const double* Uv = U + (long long)blk * m.blk_stride + v * m.var_stride;
        const int nb = blockDim.x;
        int c = threadIdx.x;
        for (; c + 3 * nb < ncell; c += 4 * nb) {
            a0 += Uv[cell_offset(m, c)];
            a1 += Uv[cell_offset(m, c + nb)];
            a2 += Uv[cell_offset(m, c + 2 * nb)];
            a3 += Uv[cell_offset(m, c + 3 * nb)];
        }
        for (; c < ncell; c += nb) a0 += Uv[cell_offset(m, c)];
        red[threadIdx.x] = (a0 + a1) + (a2 + a3);
        __syncthreads();
        for (int o = 128; o > 0; o >>= 1) {
            if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) partial[(long long)blk * 5 + v] = red[0];
        __syncthreads();
    }
}

__global__ void sum_partials_kernel(const MeshDev m, int nblk, const double* __restrict__ partial,
                                    double* __restrict__ out) {
    __shared__ double red[256];
    for (int v = 0; v < m.nvar; ++v) {
        double acc = 0.0;
        for (int b = threadIdx.x; b < nblk; b += blockDim.x) acc += partial[(long long)b * 5 + v];
        red[threadIdx.x] = acc;
        __syncthreads();
        for (int o = 128; o > 0; o >>= 1) {
            if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[v] = red[0];
        __syncthreads();
    }
}

// CTAs per block for the per-cell utility kernels: one per 4096 cells.
static unsigned cell_chunks(const MeshDev& m) {
    const int ncell = m.bs[0] * m.bs[1] * m.bs[2];
    return (unsigned)((ncell + 4095) / 4096);
}

cudaError_t launch_region_init(const MeshDev& m, double* U, int kind, int4 reg, const RegionStates& rs, cudaStream_t st) {
    region_init_kernel<<<dim3((unsigned)(m.nb[0] * m.nb[1] * m.nb[2]), cell_chunks(m)), 256, 0, st>>>(m, U, kind, reg,
                                                                                                      rs);
    return cudaGetLastError();
}

// Full-block work items of the meshes slots[0..nslots): slot s owns items
// item0 .. item0 + nitems - 1 in block-major, tile-minor order (one CTA per
// slot), the order a host-built list of the same meshes has.
__global__ void expand_items_kernel(const SlotDev* __restrict__ slots, Item* __restrict__ items) {
    const SlotDev& sd = slots[blockIdx.x];
    const int nt = sd.tiles_x * sd.tiles_y, n = sd.nitems, base = sd.item0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) items[base + i] = Item{(int)blockIdx.x, i / nt, i % nt, 0};
}

cudaError_t launch_expand_items(const SlotDev* slots, int nslots, Item* items, cudaStream_t st) {
    if (nslots <= 0) return cudaSuccess;
    expand_items_kernel<<<nslots, 256, 0, st>>>(slots, items);
    return cudaGetLastError();
}

cudaError_t launch_totals(const MeshDev& m, int nblk, const double* U, double* partial, double* out, cudaStream_t st) {
    block_totals_kernel<<<dim3((unsigned)nblk, (unsigned)m.nvar), 256, 0, st>>>(m, U, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    sum_partials_kernel<<<1, 256, 0, st>>>(m, nblk, partial, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- self-test of the integer-pipe conversions
// f2d on every binary32 pattern in [lo, lo + n) and d2f_rn on patterns from a
// 64-bit mixing function (splitmix64) plus exponents near the binary32 range
// edges; counts results whose bits differ from the hardware conversion.
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void selftest_kernel(unsigned long long lo, unsigned long long n, unsigned long long seed,
                                unsigned long long* bad) {
    unsigned long long cnt = 0;
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned fb = (unsigned)(lo + i);
        const float f = __uint_as_float(fb);
        const double a = f2d(f), b = (double)f;
        if (__double_as_longlong(a) != __double_as_longlong(b) && !(a != a && b != b)) ++cnt;
        unsigned long long db = mix64(seed + i);
        if (i & 1) {   // steer half of the samples to exponents around the binary32 normal range
            const unsigned long long e = 880 + (mix64(db) % 290);
            db = (db & 0x800FFFFFFFFFFFFFull) | (e << 52);
        }
        const double d = __longlong_as_double((long long)db);
        const float x = d2f_rn(d), y = __double2float_rn(d);
        if (__float_as_uint(x) != __float_as_uint(y) && !(x != x && y != y)) ++cnt;
    }
    if (cnt) atomicAdd(bad, cnt);
}

// em_add / em_sub / em_mul against the hardware on pseudo-random operand
// pairs: half unrelated (any exponent, mantissas near all-ones or near zero,
// exact zeros), half related (the second is the first with a flipped sign,
// low mantissa bits perturbed and the exponent moved by a few), which
// exercises carries, ties and cancellation. The same pairs check the FP64
// task's integer forms of the sign tests, the wave-speed order, minmod and
// the halving against FP64 comparisons and 0.5 * x, and the FP32 tasks'
// minmod against FP32 comparisons.
__device__ __forceinline__ unsigned long long rand_double_bits(unsigned long long z) {
    const unsigned long long r = mix64(z), r2 = mix64(z ^ 0x5DEECE66Dull);
    const unsigned k = (unsigned)(r2 % 6);
    const unsigned long long sign = (r2 >> 8) & 1ull;
    if (k == 0) return r;
    if (k == 5) return sign << 63;                                   // +-0
    const unsigned long long e = (k == 1) ? 1 + (r2 >> 16) % 2046 : 1000 + (r2 >> 16) % 50;
    unsigned long long m = r & kM52;
    if (k == 3) m = kM52 - ((r2 >> 32) & 15);
    if (k == 4) m = (r2 >> 32) & 15;
    return (sign << 63) | (e << 52) | m;
}

__global__ void selftest_fp64_kernel(unsigned long long n, unsigned long long seed, unsigned long long* bad) {
    unsigned long long cnt = 0;
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long a = rand_double_bits(seed + 2 * i);
        unsigned long long b;
        const unsigned long long r = mix64(seed ^ (i * 0x9E3779B97F4A7C15ull));
        if (r & 1) {
            b = a ^ ((r >> 1) & 1ull) << 63;
            b ^= (r >> 2) & ((1ull << (1 + (r >> 58) % 52)) - 1ull);
            const long long e = (long long)((b >> 52) & 0x7FF) + (long long)((r >> 40) % 7) - 3;
            if (e > 0 && e < 0x7FF) b = (b & ~(0x7FFull << 52)) | ((unsigned long long)e << 52);
        } else {
            b = rand_double_bits(seed + 2 * i + 1);
        }
        const double x = __longlong_as_double((long long)a), y = __longlong_as_double((long long)b);
        const double m1 = em_mul(x, y), m2 = __dmul_rn(x, y);
        const double a1 = em_add(x, y), a2 = __dadd_rn(x, y);
        const double s1 = em_sub(x, y), s2 = __dsub_rn(x, y);
        cnt += (__double_as_longlong(m1) != __double_as_longlong(m2)) && !(m2 != m2);
        cnt += (__double_as_longlong(a1) != __double_as_longlong(a2)) && !(a2 != a2);
        cnt += (__double_as_longlong(s1) != __double_as_longlong(s2)) && !(s2 != s2);
        // the FP64 task's integer-pipe sign tests, selects and halving against
        // FP64 comparisons and multiplication (NaN operands excepted)
        if (!(x != x) && !(y != y)) {
            const rd X(x), Y(y);
            const bool zz = x == 0.0 && y == 0.0 && signbit(x) && !signbit(y);   // -0 < +0 in lt only
            cnt += P<rd>::lt(X, Y) != ((x < y) || zz);
            cnt += P<rd>::ge0(X) != (x >= 0.0);
            cnt += P<rd>::le0(X) != (x <= 0.0);
            cnt += P<rd>::pos(X) != (x > 0.0);
            cnt += P<rd>::neg(X) != (x < 0.0);
            const double mm = (x > 0.0 && y > 0.0) ? (x < y ? x : y) : ((x < 0.0 && y < 0.0) ? (x > y ? x : y) : 0.0);
            cnt += __double_as_longlong(P<rd>::minmod(X, Y).v) != __double_as_longlong(mm);
            cnt += __double_as_longlong(P<rd>::half(X).v) != __double_as_longlong(__dmul_rn(0.5, x));
        }
        // the FP32 minmod (FP32-flux tasks) against its sign-test definition,
        // both argument orders, on binary32 pairs taken from the high and the
        // low words of the operands (zeros of both signs, ties, subnormals,
        // infinities; NaN excepted)
#pragma unroll
        for (int w = 0; w < 2; ++w) {
            const float fx = __uint_as_float((unsigned)(w ? a : a >> 32)), fy = __uint_as_float((unsigned)(w ? b : b >> 32));
            if (!(fx != fx) && !(fy != fy)) {
                const float fm = (fx > 0.0f && fy > 0.0f) ? (fx < fy ? fx : fy)
                                                          : ((fx < 0.0f && fy < 0.0f) ? (fx > fy ? fx : fy) : 0.0f);
                cnt += __float_as_uint(P<float>::minmod(fx, fy)) != __float_as_uint(fm);
                cnt += __float_as_uint(P<float>::minmod(fy, fx)) != __float_as_uint(fm);
            }
        }
    }
    if (cnt) atomicAdd(bad, cnt);
}

// Double-word arithmetic (dword.cuh) against FP64 references on pseudo-random
// operands (magnitudes 2^-30 .. 2^30, both signs; half of the sum operand
// pairs nearly cancel). Every double-word here is exactly a binary64 value
// (hi + lo spans at most 49 bits), so the references A op B are FP64
// operations on the exact operands, themselves within 2^-53 of the true
// result. Raises err[k] to the largest error of: 0 binary64 -> double-word,
// 1 sum (relative to |A| + |B|), 2 product, 3 reciprocal, 4 reciprocal
// square root, 5 sound speed sqrt(X / R) as X rsqrt(X R) (relative).
__device__ __forceinline__ double st_double(unsigned long long r) {
    const unsigned long long e = 1023 - 30 + (r >> 52) % 61;
    return __longlong_as_double((long long)(((r >> 63) << 63) | (e << 52) | (r & kM52)));
}
__device__ __forceinline__ void st_raise(unsigned long long* slot, double v) {
    atomicMax(slot, (unsigned long long)__double_as_longlong(fabs(v)));
}

__global__ void selftest_dword_kernel(unsigned long long n, unsigned long long seed, unsigned long long* err) {
    double mx[6] = {0, 0, 0, 0, 0, 0};
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long r1 = mix64(seed + 2 * i), r2 = mix64(seed + 2 * i + 1);
        const double x = st_double(r1);
        double y = st_double(r2);
        if (r2 & 1) {   // nearly cancelling partner: -x with its low mantissa bits perturbed
            const unsigned long long b = (unsigned long long)__double_as_longlong(x) ^ (1ull << 63);
            y = __longlong_as_double((long long)(b ^ ((r2 >> 8) & ((1ull << (1 + (r2 >> 58) % 40)) - 1ull))));
        }
        const dw a = P<dw>::in(x), b = P<dw>::in(y);
        const double A = P<dw>::to_double(a), B = P<dw>::to_double(b);
        mx[0] = fmax(mx[0], fabs(__dsub_rn(A, x)) / fabs(x));
        mx[1] = fmax(mx[1], fabs(__dsub_rn(P<dw>::to_double(a + b), __dadd_rn(A, B))) / (fabs(A) + fabs(B)));
        const double AB = __dmul_rn(A, B);
        mx[2] = fmax(mx[2], fabs(__dsub_rn(P<dw>::to_double(a * b), AB)) / fabs(AB));
        const double iA = __drcp_rn(A);
        mx[3] = fmax(mx[3], fabs(__dsub_rn(P<dw>::to_double(dw_rcp(a)), iA)) / fabs(iA));
        const dw aa = {fabsf(a.hi), a.hi < 0.0f ? -a.lo : a.lo}, bb = {fabsf(b.hi), b.hi < 0.0f ? -b.lo : b.lo};
        const double rs = __drcp_rn(__dsqrt_rn(fabs(A)));
        mx[4] = fmax(mx[4], fabs(__dsub_rn(P<dw>::to_double(dw_rsqrt(aa)), rs)) / rs);
        const double c = __dsqrt_rn(__ddiv_rn(fabs(A), fabs(B)));
        mx[5] = fmax(mx[5], fabs(__dsub_rn(P<dw>::to_double(P<dw>::sound(aa, bb)), c)) / c);
    }
    for (int k = 0; k < 6; ++k) st_raise(err + k, mx[k]);
}

// The signal-speed filter's bound (hydro.cuh, speed_upper) against the FP64
// signal speed it stands for, on pseudo-random 3D states: density 2^-20 ..
// 2^20, velocities up to 10^6 in any direction, pressures from 10^-14 of the
// kinetic energy density (heavy cancellation in E - |m|^2/(2 rho)) to 10^6 of
// it, gamma 1.4 or 5/3, cell widths with aspect ratios up to 4. res[0]:
// states where the bound applied but lies below the FP64 speed (must be 0);
// res[1]: states where it applied; res[2]: states where it applied although
// the FP64 path finds the state non-physical (must be 0); res[3]: the
// largest bound / speed ratio, as double bits; res[4]: a scratch word for the
// FP64 path's error flag.
__global__ void selftest_speed_bound_kernel(unsigned long long n, unsigned long long seed, unsigned long long* res,
                                            int* err_sink) {
    unsigned long long bad = 0, applied = 0, nonphys = 0;
    double worst = 0.0;
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long r1 = mix64(seed + 4 * i), r2 = mix64(seed + 4 * i + 1), r3 = mix64(seed + 4 * i + 2),
                                 r4 = mix64(seed + 4 * i + 3);
        auto unit = [](unsigned long long r, int k) { return (double)((r >> (16 * k)) & 0xFFFF) / 65536.0; };
        MeshDev m{};
        m.ndim = 3;
        m.nvar = 5;
        m.gamma = (r4 & 1) ? 1.4 : 5.0 / 3.0;
        m.gm1 = m.gamma - 1.0;
        m.cfl = 0.8;
        for (int d = 0; d < 3; ++d) m.idx[d] = 64.0 * exp2(2.0 * unit(r4, d) - 1.0) * (1 + (int)((r4 >> 60) & 3));
        const double rho = exp2(40.0 * unit(r1, 0) - 20.0);
        double u[3], ke = 0.0;
        for (int d = 0; d < 3; ++d) {
            const double mag = (((r2 >> (8 * d)) & 7) == 0) ? 0.0 : pow(10.0, 12.0 * unit(r1, d + 1) - 6.0);
            u[d] = ((r3 >> d) & 1) ? -mag : mag;
            ke += 0.5 * rho * u[d] * u[d];
        }
        const double pr = (ke > 0.0) ? ke * pow(10.0, 20.0 * unit(r3, 1) - 14.0) : rho * exp2(20.0 * unit(r3, 2) - 10.0);
        rd Un[5];
        Un[0] = rd(rho);
        for (int d = 0; d < 3; ++d) Un[1 + d] = rd(rho * u[d]);
        Un[4] = rd(pr / m.gm1 + ke);
        SpeedBound sb = speed_bound_setup(m, 1.0);
        float ub, lb, ub2;
        const bool two = speed_bounds<3>(sb, speed_bound_lo_setup(m), Un, lb, ub2);   // the first dt's pair
        if (!speed_upper<3>(sb, Un, ub)) {
            bad += two;                                         // both apply under the same conditions
            continue;
        }
        ++applied;
        if (!two || __float_as_uint(ub2) != __float_as_uint(ub)) { ++bad; continue; }
        rd W[5], r;
        prim_from_cons<rd, 3>(Un, W, r, rd(m.gm1));
        if (!(P<rd>::pos(W[0]) && P<rd>::pos(W[4]))) { ++nonphys; continue; }
        m.err = err_sink;
        const double s = __longlong_as_double((long long)new_state_speed<rd, 3>(m, Un));
        const double b = (double)ub;
        if (!(b >= s) || !((double)lb <= s)) ++bad;
        worst = fmax(worst, b / s);
    }
    if (bad) atomicAdd(&res[0], bad);
    if (applied) atomicAdd(&res[1], applied);
    if (nonphys) atomicAdd(&res[2], nonphys);
    atomicMax(&res[3], (unsigned long long)__double_as_longlong(worst));
}

cudaError_t launch_selftest_speed_bound(unsigned long long n, unsigned long long seed, unsigned long long* res,
                                        cudaStream_t st) {
    selftest_speed_bound_kernel<<<148 * 8, 256, 0, st>>>(n, seed, res, reinterpret_cast<int*>(res + 4));
    return cudaGetLastError();
}

cudaError_t launch_selftest_dword(unsigned long long n, unsigned long long seed, unsigned long long* err,
                                  cudaStream_t st) {
    selftest_dword_kernel<<<148 * 8, 256, 0, st>>>(n, seed, err);
    return cudaGetLastError();
}

cudaError_t launch_selftest_fp64(unsigned long long n, unsigned long long seed, unsigned long long* bad,
                                 cudaStream_t st) {
    selftest_fp64_kernel<<<148 * 16, 256, 0, st>>>(n, seed, bad);
    return cudaGetLastError();
}

cudaError_t launch_selftest(unsigned long long lo, unsigned long long n, unsigned long long seed,
                            unsigned long long* bad, cudaStream_t st) {
    selftest_kernel<<<148 * 16, 256, 0, st>>>(lo, n, seed, bad);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- hydro launch table
// Variant of a precision code: arithmetic type and whether the kernel runs
// Runge-Kutta stages (plain MUSCL; kRK2 FP64, kRK2F32 FP32 flux, kRK2FF
// double-word); kF32X is the FP32-flux shortcut update (FX).
template <int NDIM, int TX, int TY, class T, bool RK, bool FX = false>
static cudaError_t launch_hydro_t(const MeshDev& m, const int* ids, int n, const double* Uin, double* Uout,
                                  int stage, cudaStream_t st) {
    using Tl = Tile<NDIM, TX, TY>;
    const size_t smem = Tl::template smem_bytes<typename P<T>::store>();
    auto kern = hydro_kernel<NDIM, TX, TY, T, RK, FX>;
    const int tx = m.bs[0] / TX, ty = m.bs[1] / TY;
    kern<<<dim3((unsigned)(n * tx * ty)), dim3(Tl::template nb<T, RK>()), smem, st>>>(m, ids, tx, ty, Uin, Uout, stage,
                                                                                    GlobalIO{});
    return cudaGetLastError();
}

template <int NDIM, int TX, int TY, class T, bool RK, bool FX = false>
static cudaError_t configure_t() {
    using Tl = Tile<NDIM, TX, TY>;
    const size_t smem = Tl::template smem_bytes<typename P<T>::store>();
    cudaError_t e = cudaFuncSetAttribute(hydro_kernel<NDIM, TX, TY, T, RK, FX>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(persistent_kernel<NDIM, TX, TY, T, RK, FX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem);
}

template <int NDIM, int TX, int TY, class T, bool RK, bool FX = false>
static cudaError_t launch_persistent_t(const SlotDev* slots, const Item* items, int nitems, unsigned* queue, int grid,
                                       int stage, cudaStream_t st) {
    using Tl = Tile<NDIM, TX, TY>;
    const size_t smem = Tl::template smem_bytes<typename P<T>::store>();
    persistent_kernel<NDIM, TX, TY, T, RK, FX><<<grid, Tl::template nb<T, RK>(), smem, st>>>(slots, items, nitems, queue, stage);
    return cudaGetLastError();
}

template <int NDIM, int TX, int TY, class T, bool RK, bool FX = false>
static cudaError_t occupancy_t(int* per_sm) {
    using Tl = Tile<NDIM, TX, TY>;
    const size_t smem = Tl::template smem_bytes<typename P<T>::store>();
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, persistent_kernel<NDIM, TX, TY, T, RK, FX>, Tl::template nb<T, RK>(),
                                                         smem);
}

#define ORCHA_PERS_CASE(ND, X, Y)                                                                         \
    if (ndim == ND && tx == X && ty == Y)                                                                 \
        return prec == kF32   ? launch_persistent_t<ND, X, Y, float, false>(slots, items, nitems, queue, grid, 0, st) \
               : prec == kF32X ? launch_persistent_t<ND, X, Y, float, false, true>(slots, items, nitems, queue, grid, 0, st) \
               : prec == kFF  ? launch_persistent_t<ND, X, Y, dw, false>(slots, items, nitems, queue, grid, 0, st)    \
               : prec == kRK2 ? launch_persistent_t<ND, X, Y, rd, true>(slots, items, nitems, queue, grid, stage, st) \
               : prec == kRK2F32 ? launch_persistent_t<ND, X, Y, float, true>(slots, items, nitems, queue, grid, stage, st) \
               : prec == kRK2FF ? launch_persistent_t<ND, X, Y, dw, true>(slots, items, nitems, queue, grid, stage, st) \
                              : launch_persistent_t<ND, X, Y, rd, false>(slots, items, nitems, queue, grid, 0, st);

cudaError_t launch_persistent(int ndim, int tx, int ty, int prec, const SlotDev* slots, const Item* items,
                              int nitems, unsigned* queue, int grid, int stage, cudaStream_t st) {
    ORCHA_PERS_CASE(2, 8, 8)
    ORCHA_PERS_CASE(2, 16, 8)
    ORCHA_PERS_CASE(2, 16, 16)
    ORCHA_PERS_CASE(3, 8, 8)
    ORCHA_PERS_CASE(3, 16, 8)
    ORCHA_PERS_CASE(3, 16, 16)
    return cudaErrorInvalidConfiguration;
}

#define ORCHA_OCC_CASE(ND, X, Y)                                                                       \
    if (ndim == ND && tx == X && ty == Y)                                                              \
        return prec == kF32   ? occupancy_t<ND, X, Y, float, false>(per_sm)                            \
               : prec == kF32X ? occupancy_t<ND, X, Y, float, false, true>(per_sm)                     \
               : prec == kFF  ? occupancy_t<ND, X, Y, dw, false>(per_sm)                               \
               : prec == kRK2 ? occupancy_t<ND, X, Y, rd, true>(per_sm)                                \
               : prec == kRK2F32 ? occupancy_t<ND, X, Y, float, true>(per_sm)                          \
               : prec == kRK2FF ? occupancy_t<ND, X, Y, dw, true>(per_sm)                              \
                              : occupancy_t<ND, X, Y, rd, false>(per_sm);

cudaError_t persistent_occupancy(int ndim, int tx, int ty, int prec, int* per_sm) {
    ORCHA_OCC_CASE(2, 8, 8)
    ORCHA_OCC_CASE(2, 16, 8)
    ORCHA_OCC_CASE(2, 16, 16)
    ORCHA_OCC_CASE(3, 8, 8)
    ORCHA_OCC_CASE(3, 16, 8)
    ORCHA_OCC_CASE(3, 16, 16)
    return cudaErrorInvalidConfiguration;
}

#define ORCHA_TILE_CASE(ND, X, Y)                                                                      \
    if (ndim == ND && tx == X && ty == Y)                                                              \
        return prec == kF32   ? launch_hydro_t<ND, X, Y, float, false>(m, ids, n, Uin, Uout, 0, st)    \
               : prec == kF32X ? launch_hydro_t<ND, X, Y, float, false, true>(m, ids, n, Uin, Uout, 0, st) \
               : prec == kFF  ? launch_hydro_t<ND, X, Y, dw, false>(m, ids, n, Uin, Uout, 0, st)       \
               : prec == kRK2 ? launch_hydro_t<ND, X, Y, rd, true>(m, ids, n, Uin, Uout, stage, st)    \
               : prec == kRK2F32 ? launch_hydro_t<ND, X, Y, float, true>(m, ids, n, Uin, Uout, stage, st) \
               : prec == kRK2FF ? launch_hydro_t<ND, X, Y, dw, true>(m, ids, n, Uin, Uout, stage, st)  \
                              : launch_hydro_t<ND, X, Y, rd, false>(m, ids, n, Uin, Uout, 0, st);

cudaError_t launch_hydro(const MeshDev& m, int tx, int ty, int prec, const int* ids, int n, const double* Uin,
                         double* Uout, int stage, cudaStream_t st) {
    const int ndim = m.ndim;
    ORCHA_TILE_CASE(2, 8, 8)
    ORCHA_TILE_CASE(2, 16, 8)
    ORCHA_TILE_CASE(2, 16, 16)
    ORCHA_TILE_CASE(3, 8, 8)
    ORCHA_TILE_CASE(3, 16, 8)
    ORCHA_TILE_CASE(3, 16, 16)
    return cudaErrorInvalidConfiguration;
}

#define ORCHA_CONF_CASE(ND, X, Y)                                                                      \
    if (ndim == ND && tx == X && ty == Y) {                                                            \
        cudaError_t e = configure_t<ND, X, Y, float, false>();                                         \
        if (e == cudaSuccess) e = configure_t<ND, X, Y, float, false, true>();                         \
        if (e == cudaSuccess) e = configure_t<ND, X, Y, dw, false>();                                  \
        if (e == cudaSuccess) e = configure_t<ND, X, Y, rd, true>();                                   \
        if (e == cudaSuccess) e = configure_t<ND, X, Y, float, true>();                                \
        if (e == cudaSuccess) e = configure_t<ND, X, Y, dw, true>();                                   \
        return e != cudaSuccess ? e : configure_t<ND, X, Y, rd, false>();                              \
    }

cudaError_t configure_hydro(int ndim, int tx, int ty) {
    ORCHA_CONF_CASE(2, 8, 8)
    ORCHA_CONF_CASE(2, 16, 8)
    ORCHA_CONF_CASE(2, 16, 16)
    ORCHA_CONF_CASE(3, 8, 8)
    ORCHA_CONF_CASE(3, 16, 8)
    ORCHA_CONF_CASE(3, 16, 16)
    return cudaErrorInvalidConfiguration;
}

bool hydro_tile_supported(int ndim, int tx, int ty) {
    const int t[3][2] = {{8, 8}, {16, 8}, {16, 16}};
    for (auto& p : t)
        if (p[0] == tx && p[1] == ty) return ndim == 2 || ndim == 3;
    return false;
}

// One grid row per packet block; a packet of more blocks than a grid has
// rows (65,535) is filled by consecutive launches over slices of its ids.
cudaError_t launch_guard_fill(const MeshDev& m, const int* ids, int n, double* U, cudaStream_t st) {
    const int threads = 256, max_rows = 65535;
    const long long npad = m.var_stride;
    const unsigned gx = (unsigned)((npad + threads - 1) / threads);
    for (int off = 0; off < n; off += max_rows) {
        const int rows = n - off < max_rows ? n - off : max_rows;
        guard_fill_kernel<<<dim3(gx, (unsigned)rows), threads, 0, st>>>(m, ids + off, U);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_pack(const MeshDev& m, const double* interior, double* U, cudaStream_t st) {
    const long long planes = (long long)m.nb[0] * m.nb[1] * m.nb[2] * m.nvar;
    pack_kernel<<<(unsigned)planes, 256, 0, st>>>(m, interior, U);
    return cudaGetLastError();
}

cudaError_t launch_unpack(const MeshDev& m, const double* U, double* interior, cudaStream_t st) {
    const long long planes = (long long)m.nb[0] * m.nb[1] * m.nb[2] * m.nvar;
    unpack_kernel<<<(unsigned)planes, 256, 0, st>>>(m, U, interior);
    return cudaGetLastError();
}

cudaError_t launch_pack_ids(const MeshDev& m, const int* ids, int n, const double* interior, double* U,
                            cudaStream_t st) {
    pack_ids_kernel<<<(unsigned)((long long)n * m.nvar), 256, 0, st>>>(m, ids, n, interior, U);
    return cudaGetLastError();
}

cudaError_t launch_unpack_ids(const MeshDev& m, const int* ids, int n, const double* U, double* interior,
                              cudaStream_t st) {
    unpack_ids_kernel<<<(unsigned)((long long)n * m.nvar), 256, 0, st>>>(m, ids, n, U, interior);
    return cudaGetLastError();
}

cudaError_t launch_signal_speed(const MeshDev& m, const int* ids, int n, const double* U, cudaStream_t st) {
    signal_speed_kernel<<<(unsigned)n, 256, 0, st>>>(m, ids, U);
    return cudaGetLastError();
}

cudaError_t launch_signal_speed_all(const MeshDev& m, int nblk, const double* U, cudaStream_t st, bool f32) {
    const dim3 grid((unsigned)nblk, cell_chunks(m));
    if (f32) signal_speed_all_kernel<true><<<grid, 256, 0, st>>>(m, U);
    else signal_speed_all_kernel<false><<<grid, 256, 0, st>>>(m, U);
    return cudaGetLastError();
}

cudaError_t launch_dt_reduce(const MeshDev& m, int nblk, double* dt, cudaStream_t st) {
    dt_reduce_kernel<<<1, 1024, 0, st>>>(m, nblk, dt);
    return cudaGetLastError();
}

cudaError_t launch_first_dt(const MeshDev& m, int nblk, const double* U, double* dt, unsigned long long* lbmax,
                            cudaStream_t st) {
    if (!m.sub || !lbmax || (m.ndim != 2 && m.ndim != 3)) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(lbmax, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    const dim3 grid((unsigned)nblk, cell_chunks(m));
    if (m.ndim == 3) {
        first_dt_bounds_kernel<3><<<grid, 256, 0, st>>>(m, U, lbmax);
        first_dt_eval_kernel<3><<<grid, 256, 0, st>>>(m, U, lbmax);
    } else {
        first_dt_bounds_kernel<2><<<grid, 256, 0, st>>>(m, U, lbmax);
        first_dt_eval_kernel<2><<<grid, 256, 0, st>>>(m, U, lbmax);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    dt_reduce_kernel<<<1, 1024, 0, st>>>(m, nblk, dt);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return cudaMemsetAsync(m.sub, 0, sizeof(unsigned long long) * (size_t)nblk, st);
}

}  // namespace orcha
