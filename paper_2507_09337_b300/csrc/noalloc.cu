// noalloc.cu -- the CFL time step of a state buffer, computed without any
// device allocation.
//
// The mesh objects of this library allocate a small per-block array for the
// signal-speed maxima. Some callers cannot let a library allocate: host
// codes that hand every byte of HBM to their own allocator up front, or that
// must not allocate inside their time loop. For them this entry point keeps
// that per-block array in a file-scope device array of fixed size instead.
#include <cstdio>
#include <mutex>

#include "../../include/orcha.h"
#include "common.cuh"
#include "hydro.cuh"
#include "launch.h"

namespace orcha {

// Per-block signal-speed maxima (bits of non-negative doubles) of every call
// of orcha_cfl_dt_noalloc. Every GPU that loads the library holds this array
// (512 KiB) until the process exits.
static __device__ __align__(256) unsigned long long g_noalloc_smax[ORCHA_NOALLOC_MAX_BLOCKS];

// Device address of g_noalloc_smax in the current context. Host code must
// never pass the symbol itself. Outside stream capture the address is looked
// up on every call (cheap once the module is loaded), so a context the caller
// reset or replaced since an earlier call never gets a stale pointer. Inside
// a capture the lookup could load the module, which capture forbids, so the
// address that the last uncaptured call on this device saw is used.
static std::mutex g_addr_mu;
static unsigned long long* g_addr[64] = {};

static orcha_status scratch_address(cudaStream_t s, unsigned long long** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "cfl_dt_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= 64) return set_error(ORCHA_ERR_UNSUPPORTED, "cfl_dt_noalloc: device index above 63");
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess) return cuda_error(e, "cfl_dt_noalloc: cudaStreamIsCapturing");
    std::lock_guard<std::mutex> lock(g_addr_mu);
    if (cs == cudaStreamCaptureStatusNone) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_smax);
        if (e != cudaSuccess) return cuda_error(e, "cfl_dt_noalloc: cudaGetSymbolAddress");
        g_addr[dev] = static_cast<unsigned long long*>(p);
    } else if (!g_addr[dev]) {
        return set_error(ORCHA_ERR_INVALID,
                         "cfl_dt_noalloc: the first call on a device must come before any stream capture");
    }
    *out = g_addr[dev];
    return ORCHA_OK;
}

}  // namespace orcha

extern "C" orcha_status orcha_cfl_dt_noalloc(const orcha_mesh_desc* desc, int32_t current, int32_t* err_dev,
                                             void* stream) {
    orcha::MeshDev m;
    long long nblk = 0;
    orcha_status st = orcha::mesh_dev_from_desc(desc, &m, &nblk);
    if (st) return st;
    if (current != 0 && current != 1) return orcha::set_error(ORCHA_ERR_INVALID, "cfl_dt_noalloc: current must be 0 or 1");
    const double* U = desc->state_dev[current];
    if (!U || !desc->dt_dev || !err_dev)
        return orcha::set_error(ORCHA_ERR_INVALID, "cfl_dt_noalloc: state buffer, dt_dev and err_dev are required");
    if ((((uintptr_t)U) | ((uintptr_t)desc->dt_dev)) & 7 || ((uintptr_t)err_dev) & 3)
        return orcha::set_error(ORCHA_ERR_INVALID, "cfl_dt_noalloc: misaligned buffer");
    if (nblk > ORCHA_NOALLOC_MAX_BLOCKS) {
        char msg[160];
        snprintf(msg, sizeof(msg), "cfl_dt_noalloc: mesh has %lld blocks, above the no-allocation limit of %d",
                 nblk, ORCHA_NOALLOC_MAX_BLOCKS);
        return orcha::set_error(ORCHA_ERR_INVALID, msg);
    }
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long* smax = nullptr;
    if ((st = orcha::scratch_address(s, &smax))) return st;
    m.smax = smax;
    m.err = err_dev;
    // the array keeps the previous call's contents: clear the slots this call raises
    cudaError_t e = cudaMemsetAsync(smax, 0, sizeof(unsigned long long) * (size_t)nblk, s);
    if (e != cudaSuccess) return orcha::cuda_error(e, "cfl_dt_noalloc: clear");
    // one CTA per block of the mesh (no block-id list, which would need memory)
    e = orcha::launch_signal_speed_all(m, (int)nblk, U, s);
    if (e != cudaSuccess) return orcha::cuda_error(e, "cfl_dt_noalloc: signal-speed launch");
    e = orcha::launch_dt_reduce(m, (int)nblk, desc->dt_dev, s);
    if (e != cudaSuccess) return orcha::cuda_error(e, "cfl_dt_noalloc: reduce launch");
    return ORCHA_OK;
}
