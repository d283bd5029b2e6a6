// launch.h -- host-side entry points of the kernels (internal to the library).
#pragma once

#include <cuda_runtime.h>

#include "../../include/orcha.h"
#include "common.cuh"
#include "persistent.cuh"

namespace orcha {

// Variants of the hydro kernels: MUSCL-Hancock steps in FP64, with FP32
// reconstruction/flux or with double-word reconstruction/flux (all with the
// FP64 update), and Heun Runge-Kutta stages (plain MUSCL) in the same three
// arithmetics.
// kF32X: the FP32-flux shortcut (float-float flux sums, FP32 signal speed).
// kTB2, kTB2F32: two Hancock steps per launch (FP64, FP32 flux); kFRK2,
// kFRK2F32: both Heun stages in one launch (fused.cuh).
enum Prec : int {
    kF64 = 0, kF32 = 1, kFF = 2, kRK2 = 3, kRK2F32 = 4, kRK2FF = 5, kF32X = 6,
    kTB2 = 7, kTB2F32 = 8, kFRK2 = 9, kFRK2F32 = 10
};
constexpr int kNumPrec = 11;
inline bool prec_is_rk(int p) { return p == kRK2 || p == kRK2F32 || p == kRK2FF; }
inline bool prec_is_fused(int p) { return p >= kTB2; }
inline bool prec_is_tb2(int p) { return p == kTB2 || p == kTB2F32; }
// variants whose first dt uses the FP32 signal-speed rule (the shortcut's)
inline bool prec_f32_dt(int p) { return p == kF32X; }
// variants with FP32 reconstruction and fluxes
inline bool prec_is_f32(int p) { return p == kF32 || p == kF32X || p == kRK2F32 || p == kTB2F32 || p == kFRK2F32; }
inline bool prec_is_dw(int p) { return p == kFF || p == kRK2FF; }
// Variant of a hydro task, or -1 for any other task.
inline int prec_of(orcha_task t) {
    switch (t) {
        case ORCHA_TASK_HYDRO_FP64: return kF64;
        case ORCHA_TASK_HYDRO_F32FLUX: return kF32;
        case ORCHA_TASK_HYDRO_F32FLUX_FFSUM: return kF32X;
        case ORCHA_TASK_HYDRO_TB2: return kTB2;
        case ORCHA_TASK_HYDRO_F32FLUX_TB2: return kTB2F32;
        case ORCHA_TASK_HYDRO_RK2_FUSED: return kFRK2;
        case ORCHA_TASK_HYDRO_RK2_F32FLUX_FUSED: return kFRK2F32;
        case ORCHA_TASK_HYDRO_FF: return kFF;
        case ORCHA_TASK_HYDRO_RK2:
        case ORCHA_TASK_RK2_STAGE1:
        case ORCHA_TASK_RK2_STAGE2: return kRK2;
        case ORCHA_TASK_HYDRO_RK2_F32FLUX:
        case ORCHA_TASK_RK2_F32FLUX_STAGE1:
        case ORCHA_TASK_RK2_F32FLUX_STAGE2: return kRK2F32;
        case ORCHA_TASK_HYDRO_RK2_FF:
        case ORCHA_TASK_RK2_FF_STAGE1:
        case ORCHA_TASK_RK2_FF_STAGE2: return kRK2FF;
        default: return -1;
    }
}
// Runge-Kutta stage of a packet task (1 or 2), 0 for a whole-step task.
inline int stage_of(orcha_task t) {
    switch (t) {
        case ORCHA_TASK_RK2_STAGE1:
        case ORCHA_TASK_RK2_F32FLUX_STAGE1:
        case ORCHA_TASK_RK2_FF_STAGE1: return 1;
        case ORCHA_TASK_RK2_STAGE2:
        case ORCHA_TASK_RK2_F32FLUX_STAGE2:
        case ORCHA_TASK_RK2_FF_STAGE2: return 2;
        default: return 0;
    }
}
// Whole Heun-step tasks (two launches per step).
inline bool is_rk_step_task(orcha_task t) {
    return t == ORCHA_TASK_HYDRO_RK2 || t == ORCHA_TASK_HYDRO_RK2_F32FLUX || t == ORCHA_TASK_HYDRO_RK2_FF;
}
// Packet task of stage k (1 or 2) of a whole Heun-step task.
inline orcha_task rk_stage_task(orcha_task step, int k) {
    if (step == ORCHA_TASK_HYDRO_RK2_F32FLUX) return k == 1 ? ORCHA_TASK_RK2_F32FLUX_STAGE1 : ORCHA_TASK_RK2_F32FLUX_STAGE2;
    if (step == ORCHA_TASK_HYDRO_RK2_FF) return k == 1 ? ORCHA_TASK_RK2_FF_STAGE1 : ORCHA_TASK_RK2_FF_STAGE2;
    return k == 1 ? ORCHA_TASK_RK2_STAGE1 : ORCHA_TASK_RK2_STAGE2;
}
// Tasks that advance whole steps (mesh_advance, batch_advance, autotune).
inline bool is_step_task(orcha_task t) {
    return t == ORCHA_TASK_HYDRO_FP64 || t == ORCHA_TASK_HYDRO_F32FLUX || t == ORCHA_TASK_HYDRO_FF ||
           t == ORCHA_TASK_HYDRO_F32FLUX_FFSUM || prec_is_fused(prec_of(t)) ||
           is_rk_step_task(t);
}

// Error reporting of the C ABI (sets the calling thread's orcha_last_error).
orcha_status set_error(orcha_status code, const char* msg);
orcha_status cuda_error(cudaError_t e, const char* what);
// Validate a descriptor and build the kernels' view of it (scratch pointers
// left null). Host-only.
orcha_status mesh_dev_from_desc(const orcha_mesh_desc* d, MeshDev* out, long long* nblk_out);

// One hydro launch over the packet blocks ids[0..n); stage: Runge-Kutta stage
// (1 or 2) for the Runge-Kutta variants, else 0.
cudaError_t launch_hydro(const MeshDev& m, int tx, int ty, int prec, const int* ids, int n, const double* Uin,
                         double* Uout, int stage, cudaStream_t st);
bool hydro_tile_supported(int ndim, int tx, int ty);
// Set the dynamic shared-memory limit of every precision of a tile variant on
// the current device (call once per device before launching or capturing).
cudaError_t configure_hydro(int ndim, int tx, int ty);
cudaError_t launch_guard_fill(const MeshDev& m, const int* ids, int n, double* U, cudaStream_t st);
cudaError_t launch_pack(const MeshDev& m, const double* interior, double* U, cudaStream_t st);
cudaError_t launch_unpack(const MeshDev& m, const double* U, double* interior, cudaStream_t st);
// Interiors of the blocks ids[0..n) in packet order <-> the padded state.
cudaError_t launch_pack_ids(const MeshDev& m, const int* ids, int n, const double* interior, double* U,
                            cudaStream_t st);
cudaError_t launch_unpack_ids(const MeshDev& m, const int* ids, int n, const double* U, double* interior,
                              cudaStream_t st);
cudaError_t launch_signal_speed(const MeshDev& m, const int* ids, int n, const double* U, cudaStream_t st);
cudaError_t launch_dt_reduce(const MeshDev& m, int nblk, double* dt, cudaStream_t st);
// The first CFL time step of U with the signal-speed filter (kernels.cu): the
// same dt bits as launch_signal_speed_all (FP64 rule) + launch_dt_reduce, with
// FP64 speeds only where a cell can hold the maximum. Needs m.sub (nblk
// entries) and m.smax zero on entry (left zero) and one scratch word lbmax.
cudaError_t launch_first_dt(const MeshDev& m, int nblk, const double* U, double* dt, unsigned long long* lbmax,
                            cudaStream_t st);
// Signal speed of every block 0..nblk-1 (one CTA per block, no id list).
// f32: the FP32-flux variant's signal-speed rule (its first dt), else FP64.
cudaError_t launch_signal_speed_all(const MeshDev& m, int nblk, const double* U, cudaStream_t st,
                                   bool f32 = false);
// Two conserved states of a two-region initial state (serving recipes).
struct RegionStates {
    double in[5], out[5];
};
cudaError_t launch_region_init(const MeshDev& m, double* U, int kind, int4 reg, const RegionStates& rs, cudaStream_t st);
// out[v] = sum over interior cells of conserved variable v (fixed order);
// partial is scratch of nblk x 5 doubles.
cudaError_t launch_totals(const MeshDev& m, int nblk, const double* U, double* partial, double* out, cudaStream_t st);
// Fill the interiors of a padded state with a smooth physical state (autotuning input).
cudaError_t launch_synthetic_state(const MeshDev& m, double* U, cudaStream_t st);
// Self-test of the integer-pipe format conversions (counts mismatches into *bad).
cudaError_t launch_selftest(unsigned long long lo, unsigned long long n, unsigned long long seed,
                            unsigned long long* bad, cudaStream_t st);
// Self-test of the integer-pipe binary64 add/sub/mul (counts mismatches into *bad).
cudaError_t launch_selftest_fp64(unsigned long long n, unsigned long long seed, unsigned long long* bad,
                                 cudaStream_t st);
// Self-test of the double-word arithmetic: raises err[0..5] (bits of
// non-negative doubles) to the largest errors against FP64 references.
cudaError_t launch_selftest_speed_bound(unsigned long long n, unsigned long long seed, unsigned long long* res,
                                        cudaStream_t st);
cudaError_t launch_selftest_dword(unsigned long long n, unsigned long long seed, unsigned long long* err,
                                  cudaStream_t st);
// Built column-tile variants, widest first.
constexpr int kTiles[3][2] = {{16, 16}, {16, 8}, {8, 8}};
// One persistent launch (one time step of every mesh in `slots`).
cudaError_t launch_persistent(int ndim, int tx, int ty, int prec, const SlotDev* slots, const Item* items,
                              int nitems, unsigned* queue, int grid, int stage, cudaStream_t st);
// Full-block items of slots[0..nslots) written at items[slot.item0 ...]
// (block-major, tile-minor), so a caller uploads only the slots.
cudaError_t launch_expand_items(const SlotDev* slots, int nslots, Item* items, cudaStream_t st);
// Fused two-application launches (prec kTB2 .. kFRK2F32, fused.cuh): one
// launch advances every mesh of `slots` by two Hancock steps or one whole
// Heun step; scratch holds per_cta doubles per resident CTA (grid CTAs).
cudaError_t launch_fused(int ndim, int tx, int ty, int prec, const SlotDev* slots, const Item* items, int nitems,
                         unsigned* queue, double* scratch, long long per_cta, int grid, cudaStream_t st);
cudaError_t fused_occupancy(int ndim, int tx, int ty, int prec, int* per_sm);
cudaError_t configure_fused(int ndim, int tx, int ty, int prec);
// Scratch doubles of one fused CTA for blocks of bz planes.
long long fused_scratch_doubles(int ndim, int tx, int ty, int bz);
// Resident CTAs per SM of a persistent variant.
cudaError_t persistent_occupancy(int ndim, int tx, int ty, int prec, int* per_sm);

}  // namespace orcha
