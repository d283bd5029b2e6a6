// fused.cuh -- two applications of the hydro operator per launch: one read
// of the state and one write per two operator applications.
//
// The paper's Spark solver avoids a guard-cell exchange between the two
// Runge-Kutta stages by making the halo twice as thick and computing the
// first stage redundantly on the inner halo (section "Experiments", Spark
// paragraph). Here the same idea removes the state's round trip through HBM
// between two operator applications, for
//   Heun's method (RK = true):   U* = U + dt L(U),  U+ = 0.5 (U + (U* + dt L(U*)))
//   two Hancock steps (RK = false, temporal blocking):  U1 = H(U, dt),  U2 = H(U1, dt)
// with the same dt for both steps of a pair (formed from the state at the
// start of the pair; the launch checks that it also keeps the second step
// within the stability limit).
//
// One CTA takes one block's column tile (TX x TY columns, all planes of the
// block) and runs two sweeps of hydro_tile (hydro.cuh):
//   pass A advances the tile grown by 2 cells in x and y and by 2 planes in
//     z (the first stage's halo, i.e. a 4-cell halo of the input) from the
//     state buffer into a per-CTA scratch of (TX+4)(TY+4) columns x nvar x
//     (bz+4) planes of FP64 (L2-resident: a few hundred KB per CTA);
//   pass B advances the tile itself from the scratch into the other state
//     buffer, reading the boundary rule's cell where its halo leaves an
//     outflow domain edge (on periodic edges pass A computed the wrapped
//     cells directly).
// Both passes are the one-step sweep's code, so each gives exactly the bits
// of that step run on its own.
#pragma once

#include "hydro.cuh"
#include "persistent.cuh"

namespace orcha {

template <int NDIM, int TX, int TY, class T, bool RK>
struct Fused {
    using TA = Tile<NDIM, TX + 4, TY + 4>;      // pass A: the grown tile
    using TB = Tile<NDIM, TX, TY>;              // pass B: the tile
    static constexpr int NBA = TA::template nb<T, RK>(), NBB = TB::template nb<T, RK>();
    static constexpr int kThreads = NBA > NBB ? NBA : NBB;
    static constexpr size_t smem_bytes() {
        using S = typename P<T>::store;
        return TA::template smem_bytes<S>() > TB::template smem_bytes<S>() ? TA::template smem_bytes<S>()
                                                                          : TB::template smem_bytes<S>();
    }
    // scratch doubles of one CTA for blocks of bz planes (1 in 2D)
    static __host__ __device__ long long scratch_doubles(int bz) {
        return (long long)(TX + 4) * (TY + 4) * (NDIM + 2) * (NDIM == 3 ? bz + 4 : 1);
    }
};

// One launch advancing every mesh of `slots` by two operator applications.
// Items are whole-block column tiles (Item::zr = 0). scratch: scratch_per_cta
// doubles per resident CTA (indexed by blockIdx.x).
template <int NDIM, int TX, int TY, class T, bool RK>
__global__ void __launch_bounds__(Fused<NDIM, TX, TY, T, RK>::kThreads, 1)
fused_kernel(const SlotDev* __restrict__ slots, const Item* __restrict__ items, int nitems,
             unsigned int* __restrict__ queue, double* __restrict__ scratch, long long scratch_per_cta) {
    using F = Fused<NDIM, TX, TY, T, RK>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ unsigned long long red[32];
    __shared__ int s_item, s_last;
    double* my = scratch + (long long)blockIdx.x * scratch_per_cta;
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(queue, 1u);
        __syncthreads();
        const int it = s_item;
        if (it >= nitems) break;
        const Item w = items[it];
        const SlotDev& sd = slots[w.slot];
        const int cur = __ldcg(sd.cur);
        const int x0 = (w.tile % sd.tiles_x) * TX, y0 = (w.tile / sd.tiles_x) * TY;
        const int bz = NDIM == 3 ? sd.m.bs[2] : 1;
        // pass A: stage 1 (Heun) or the first step, into the scratch; a
        // Hancock pair raises its intermediate state's speeds into smax2
        hydro_tile<NDIM, TX + 4, TY + 4, T, true, RK, false, ScratchOutIO<F::kThreads, RK ? 0 : 2>>(
            sd.m, w.blk, x0 - 2, y0 - 2, sd.state[cur], nullptr, smem_raw, red, -2, bz + 2, 1,
            ScratchOutIO<F::kThreads, RK ? 0 : 2>{my, sd.smax2});
        __syncthreads();
        // pass B: stage 2 (averaged with the step's initial state) or the second step
        hydro_tile<NDIM, TX, TY, T, true, RK, false, ScratchInIO<F::kThreads>>(
            sd.m, w.blk, x0, y0, sd.state[cur], sd.state[cur ^ 1], smem_raw, red, 0, bz, 2,
            ScratchInIO<F::kThreads>{my, nullptr});
        if (threadIdx.x == 0) {
            __threadfence();
            const unsigned d = atomicAdd(sd.done, 1u);
            s_last = (d == (unsigned)sd.nitems - 1u);
        }
        __syncthreads();
        if (s_last) {
            __threadfence();
            finish_mesh_step(sd, red, true);
        }
        __syncthreads();
    }
}

}  // namespace orcha
