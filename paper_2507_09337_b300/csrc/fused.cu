// fused.cu -- launch table of the fused two-application kernels (fused.cuh).
#include "../../include/orcha.h"
#include "fused.cuh"
#include "launch.h"

namespace orcha {

namespace {

template <int NDIM, int TX, int TY, class T, bool RK>
cudaError_t launch_fused_t(const SlotDev* slots, const Item* items, int nitems, unsigned* queue, double* scratch,
                           long long per_cta, int grid, cudaStream_t st) {
    using F = Fused<NDIM, TX, TY, T, RK>;
    fused_kernel<NDIM, TX, TY, T, RK><<<grid, F::kThreads, F::smem_bytes(), st>>>(slots, items, nitems, queue,
                                                                                     scratch, per_cta);
    return cudaGetLastError();
}

template <int NDIM, int TX, int TY, class T, bool RK>
cudaError_t configure_fused_t() {
    using F = Fused<NDIM, TX, TY, T, RK>;
    return cudaFuncSetAttribute(fused_kernel<NDIM, TX, TY, T, RK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)F::smem_bytes());
}

template <int NDIM, int TX, int TY, class T, bool RK>
cudaError_t occupancy_fused_t(int* per_sm) {
    using F = Fused<NDIM, TX, TY, T, RK>;
    cudaError_t e = configure_fused_t<NDIM, TX, TY, T, RK>();
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, fused_kernel<NDIM, TX, TY, T, RK>, F::kThreads,
                                                         F::smem_bytes());
}

}  // namespace

#define ORCHA_FUSED_DISPATCH(CALL)                                                                     \
    if (ndim == 3 && tx == 16 && ty == 16) return CALL(3, 16, 16);                                    \
    if (ndim == 3 && tx == 16 && ty == 8) return CALL(3, 16, 8);                                      \
    if (ndim == 3 && tx == 8 && ty == 8) return CALL(3, 8, 8);                                        \
    if (ndim == 2 && tx == 16 && ty == 16) return CALL(2, 16, 16);                                    \
    if (ndim == 2 && tx == 16 && ty == 8) return CALL(2, 16, 8);                                      \
    if (ndim == 2 && tx == 8 && ty == 8) return CALL(2, 8, 8);                                        \
    return cudaErrorInvalidConfiguration;

#define ORCHA_FUSED_PREC(FN, ND, X, Y, ...)                                                            \
    (prec == kTB2F32    ? FN<ND, X, Y, float, false>(__VA_ARGS__)                                      \
     : prec == kFRK2    ? FN<ND, X, Y, rd, true>(__VA_ARGS__)                                          \
     : prec == kFRK2F32 ? FN<ND, X, Y, float, true>(__VA_ARGS__)                                       \
                        : FN<ND, X, Y, rd, false>(__VA_ARGS__))

cudaError_t launch_fused(int ndim, int tx, int ty, int prec, const SlotDev* slots, const Item* items, int nitems,
                         unsigned* queue, double* scratch, long long per_cta, int grid, cudaStream_t st) {
#define ORCHA_L(ND, X, Y) ORCHA_FUSED_PREC(launch_fused_t, ND, X, Y, slots, items, nitems, queue, scratch, per_cta, grid, st)
    ORCHA_FUSED_DISPATCH(ORCHA_L)
#undef ORCHA_L
}

cudaError_t fused_occupancy(int ndim, int tx, int ty, int prec, int* per_sm) {
#define ORCHA_O(ND, X, Y) ORCHA_FUSED_PREC(occupancy_fused_t, ND, X, Y, per_sm)
    ORCHA_FUSED_DISPATCH(ORCHA_O)
#undef ORCHA_O
}

cudaError_t configure_fused(int ndim, int tx, int ty, int prec) {
#define ORCHA_C(ND, X, Y) ORCHA_FUSED_PREC(configure_fused_t, ND, X, Y)
    ORCHA_FUSED_DISPATCH(ORCHA_C)
#undef ORCHA_C
}

long long fused_scratch_doubles(int ndim, int tx, int ty, int bz) {
    return (long long)(tx + 4) * (ty + 4) * (ndim + 2) * (ndim == 3 ? bz + 4 : 1);
}

}  // namespace orcha
