// persistent.cuh -- one launch per time step for many packets (of one or many
// meshes): a persistent grid drains a device work queue of (mesh, block,
// column tile) items.
//
// The paper's runtime keeps several data packets in flight on GPU streams so
// that the device has enough parallelism (sections "Sedov Blast Wave
// Results" and "Milhoja"); here the packets of a step become items of one
// queue instead, which one resident grid (CTAs per SM x SMs) drains, so
// packets of any size -- down to one block -- fill the GPU and no per-packet
// launch is paid.
//
// Per item the CTA reads its tile's halo straight from the neighbouring
// blocks (no separate guard-fill pass), advances it one step and raises the
// block's signal speed. The per-mesh step state lives on the device: the
// index of the current state buffer and dt. The CTA that completes a mesh's
// last item of the step (counted with a fenced atomic) reduces that mesh's
// signal speeds to the next dt, clears them, and flips the mesh's current
// buffer -- so a captured sequence of launches replays correctly.
#pragma once

#include "common.cuh"
#include "hydro.cuh"

namespace orcha {

struct SlotDev {
    MeshDev m;
    double* state[2];
    double* dt;             // writable alias of m.dt
    int* cur;               // device: index of the current state buffer
    unsigned int* done;     // device: items of this mesh finished in the current launch
    int nitems;             // items of this mesh per launch
    int nblk;
    int tiles_x, tiles_y;
    int item0;              // position of this mesh's first item (full-block items built on the device)
    unsigned long long* smax2;  // two-step launches: per-block signal speed of the intermediate state (else null)
};

// One unit of work: a column tile of block blk over its interior planes, or,
// when zr = z0 | z1 << 16 is non-zero, over the planes [z0, z1) of the
// column of blocks above blk (plane q lies in block blk + (q / bz) nb_x nb_y).
struct Item {
    int slot, blk, tile, zr;
};

// Finish a mesh's step: dt = cfl / max signal speed (unless update_dt is
// false: the first stage of a Runge-Kutta step keeps dt), clear the maxima
// and the item counter, flip the current buffer. Called by all threads of
// one CTA.
// Largest of a per-block maximum array over the CTA (all threads call it;
// thread 0 gets the result).
__device__ __forceinline__ unsigned long long cta_max_of(const unsigned long long* a, int n, unsigned long long* red) {
    unsigned long long b = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) b = umax64(b, __ldcg(&a[i]));
    b = warp_max_u64(b);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = b;
    __syncthreads();
    unsigned long long t = 0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) t = umax64(t, red[w]);
    __syncthreads();
    return t;
}

// Finish a mesh's step: dt = cfl / max signal speed (unless update_dt is
// false: the first stage of a Runge-Kutta step keeps dt), clear the maxima
// and the item counter, flip the current buffer. A two-step launch (smax2
// set) also checks that its shared dt kept the second step stable:
// dt * s(intermediate state) <= 1, the limit of the summed-direction rule,
// else ORCHA_DEVERR_CFL. Called by all threads of one CTA.
// With the signal-speed filter (sd.m.sub set; hydro.cuh, SpeedBound) the
// maximum over the exactly evaluated cells is the step's maximum only if no
// skipped cell's bound exceeds it; otherwise this CTA evaluates the cells of
// every block whose bound does in FP64 (rare: the maximum fell below a
// quarter of the previous one) and the result has the unfiltered bits.
__device__ __forceinline__ void finish_mesh_step(const SlotDev& sd, unsigned long long* red, bool update_dt) {
    unsigned long long t = cta_max_of(sd.m.smax, sd.nblk, red);     // valid in thread 0
    if (sd.m.sub && update_dt) {
        const unsigned long long u = cta_max_of(sd.m.sub, sd.nblk, red);
        __shared__ unsigned long long s_tu[2];
        if (threadIdx.x == 0) { s_tu[0] = t; s_tu[1] = u; }
        __syncthreads();
        const unsigned long long tt = s_tu[0];
        if (s_tu[1] > tt) {                         // CTA-uniform: a skipped bound exceeds the maximum
            const double* Un = sd.state[__ldcg(sd.cur) ^ 1];
            unsigned long long b = 0ull;
            for (int i = 0; i < sd.nblk; ++i)       // every thread reads the same entry: uniform branch
                if (__ldcg(&sd.m.sub[i]) > tt) b = umax64(b, block_signal_speed<true>(sd.m, i, Un));
            b = warp_max_u64(b);
            if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = b;
            __syncthreads();
            if (threadIdx.x == 0)
                for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) t = umax64(t, red[w]);
        }
        __syncthreads();
    }
    const unsigned long long t2 = sd.smax2 ? cta_max_of(sd.smax2, sd.nblk, red) : 0ull;
    if (threadIdx.x == 0) {
        const double s = __longlong_as_double((long long)t);
        if (sd.smax2) {
            const double s1 = __longlong_as_double((long long)t2);
            if (!(s1 >= 0.0 && *sd.dt * s1 <= 1.0)) atomicOr(sd.m.err, 8);
        }
        if (update_dt) {
            if (s > 0.0 && s <= 1.7976931348623157e308) *sd.dt = sd.m.cfl / s;
            else atomicOr(sd.m.err, 2);
        }
        *sd.done = 0u;
        *sd.cur ^= 1;
    }
    for (int i = threadIdx.x; i < sd.nblk; i += blockDim.x) sd.m.smax[i] = 0ull;
    if (sd.m.sub)
        for (int i = threadIdx.x; i < sd.nblk; i += blockDim.x) sd.m.sub[i] = 0ull;
    if (sd.smax2)
        for (int i = threadIdx.x; i < sd.nblk; i += blockDim.x) sd.smax2[i] = 0ull;
}

// Resident CTAs per SM requested from the register allocator (A/B-measured
// on a B300): the FP64 variant, bound by the FP64 pipe, gains from 384
// threads per SM (a small spill; +2 %); the FP32-flux variant runs best at
// 768 threads per SM for 16x8 and 16x16 tiles (80 registers, a 20-byte
// spill: +4.8 % and +19 % over 640; seven 16x8 CTAs would fit the shared
// memory but at 72 registers spill and lose 10 %) and at 640 for 8x8 tiles
// (768 loses 12 %). The double-word
// variant has the FP64 variant's register and shared-memory footprint
// (8-byte values) and takes its bound. With one thread per interior column
// both run 16x16 tiles at two 256-thread CTAs per SM (128 registers, a
// ~100-byte spill; two 109 KB tiles fill the SM's shared memory): FP64 +8 %
// and FF +27 % over one CTA, which made 16x16 their fastest tile (FP64
// +2.2 %, FF +9 % over 16x8); the double-word and the FP64 Runge-Kutta
// variants still run so. The FP64 Hancock variant adds ring threads (320
// per 16x16 CTA): one CTA per SM at up to 168 registers (three of its ten
// warps share one of the SM's four 16 K-register files), 5 % faster than
// two 256-thread CTAs.
template <class T, int NB> struct MinBlocks { static constexpr int value = NB <= 64 ? 640 / NB : 768 / NB; };
template <int NB> struct MinBlocks<rd, NB> {
    static constexpr int value = NB == 256 ? 2 : (384 / NB > 1 ? 384 / NB : 1);
};
template <int NB> struct MinBlocks<dw, NB> {
    static constexpr int value = NB == 256 ? 2 : (384 / NB > 1 ? 384 / NB : 1);
};

// RK = true: the launch is Runge-Kutta stage `stage` (1 or 2) of every mesh
// (hydro_tile); the first stage leaves dt as it is. FX: the FP32-flux
// variant's shortcut update (hydro_tile).
template <int NDIM, int TX, int TY, class T, bool RK = false, bool FX = false>
__global__ void __launch_bounds__(Tile<NDIM, TX, TY>::template nb<T, RK>(),
                                  (MinBlocks<T, Tile<NDIM, TX, TY>::template nb<T, RK>()>::value))
persistent_kernel(const SlotDev* __restrict__ slots, const Item* __restrict__ items, int nitems,
                  unsigned int* __restrict__ queue, int stage) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ unsigned long long red[32];
    __shared__ int s_item, s_last;
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(queue, 1u);
        __syncthreads();
        const int it = s_item;
        if (it >= nitems) break;
        const Item w = items[it];
        const SlotDev& sd = slots[w.slot];
        const int cur = __ldcg(sd.cur);
        const int z0 = w.zr ? (w.zr & 0xFFFF) : 0, z1 = w.zr ? (w.zr >> 16) : -1;
        hydro_tile<NDIM, TX, TY, T, true, RK, FX, FilterIO>(sd.m, w.blk, (w.tile % sd.tiles_x) * TX,
                                                        (w.tile / sd.tiles_x) * TY, sd.state[cur], sd.state[cur ^ 1],
                                                        smem_raw, red, z0, z1, stage);
        if (threadIdx.x == 0) {
            __threadfence();
            const unsigned d = atomicAdd(sd.done, 1u);
            s_last = (d == (unsigned)sd.nitems - 1u);
        }
        __syncthreads();
        if (s_last) {
            __threadfence();
            finish_mesh_step(sd, red, !RK || stage == 2);
        }
        __syncthreads();
    }
}

}  // namespace orcha
