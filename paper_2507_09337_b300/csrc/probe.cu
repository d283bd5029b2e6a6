// probe.cu -- throughput probe of the FP64 pipe (the roofline denominator of
// the FP64 hydro task, which the FP64 pipe bounds on this GPU).
//
// Every SM runs the maximum number of resident warps; each thread advances
// eight independent chains of one FP64 operation, so neither latency nor
// issue slots of other units limit the rate. The result counts lane
// operations per second (one FMA, add or multiply = one operation), the
// same unit in which the hydro task's algorithmic operations are counted.
#include <algorithm>
#include <cstdio>

#include "../../include/orcha.h"
#include "launch.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

// OP 0 FMA, 1 add, 2 multiply; 3 an add issued as an FMA (a * one + b, one =
// 1.0 passed at run time so no compiler can fold it), 4 a multiply issued as
// an FMA (a * b + mzero, mzero = -0.0 at run time): both give the add's and
// the multiply's bits exactly.
template <int OP>
__global__ void __launch_bounds__(kThreads) fp64_rate_kernel(double* sink, int iters, double b, double c, double one,
                                                             double mzero) {
    double a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = 1.0 + 1e-6 * (double)(threadIdx.x + 7 * k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) {
            if (OP == 0) a[k] = fma(a[k], b, c);
            else if (OP == 1) a[k] = __dadd_rn(a[k], b);
            else if (OP == 2) a[k] = __dmul_rn(a[k], b);
            else if (OP == 3) a[k] = fma(a[k], one, b);
            else a[k] = fma(a[k], b, mzero);
        }
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == -1.0) sink[0] = s;     // never true for these operands; keeps the chains live
}

}  // namespace

extern "C" orcha_status orcha_measure_fp64_rate(int32_t op, double* lane_ops_per_s) {
    if (!lane_ops_per_s || op < 0 || op > 4)
        return orcha::set_error(ORCHA_ERR_INVALID, "measure_fp64_rate: op must be 0 .. 4 and the output non-null");
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    auto kern = op == 0   ? fp64_rate_kernel<0>
                : op == 1 ? fp64_rate_kernel<1>
                : op == 2 ? fp64_rate_kernel<2>
                : op == 3 ? fp64_rate_kernel<3>
                          : fp64_rate_kernel<4>;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, 0);
    if (e != cudaSuccess) return orcha::cuda_error(e, "measure_fp64_rate: device query");
    double* sink = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaMalloc(&sink, sizeof(double));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const int grid = sms * std::max(1, per_sm), iters = 16384;
    // b slightly below 1 and c small keep every chain finite and normal
    const double b = (op == 1 || op == 3) ? 1e-9 : 0.999999999, c = 1e-9;
    double best_ms = 1e300;
    for (int rep = 0; rep < 6 && e == cudaSuccess; ++rep) {    // rep 0 warms up
        e = cudaEventRecord(e0, st);
        if (e == cudaSuccess) {
            kern<<<grid, kThreads, 0, st>>>(sink, iters, b, c, 1.0, -0.0);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && rep > 0) best_ms = std::min(best_ms, (double)ms);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    cudaFree(sink);
    if (e != cudaSuccess) return orcha::cuda_error(e, "measure_fp64_rate");
    const double ops = (double)grid * kThreads * kChains * (double)iters;
    *lane_ops_per_s = ops / (best_ms * 1e-3);
    return ORCHA_OK;
}
