// amr.cu -- two-level block AMR with flux correction (orcha_amr_*).
//
// The paper's Flash-X runs on an AMR mesh: when two adjacent blocks are at
// different refinement levels, their boundary fluxes must be reconciled
// (flux correction), which the paper leaves to a second, low-intensity step
// outside its task functions (section "Experiments", Spark paragraph). Here
// the whole step stays on the device:
//   restrict   parents <- the average of their children (current buffers);
//   guards     coarse: the uniform guard fill (parents included); fine: from
//              the fine blocks, or the containing coarse cell (injection);
//   hydro      every coarse leaf and every fine block in one launch (the
//              packet sweep, recording the fluxes through each block's faces);
//   reflux     coarse leaf cells next to a refined block take the average of
//              the fine fluxes through their face instead of their own;
//   restrict   parents of the new coarse state;
//   dt         signal speeds of the new leaf cells of both levels, one dt.
// The fine level is stored as its own list of blocks (block f is child
// f % 2^ndim, octant bits x | y << 1 | z << 2, of refined[f >> ndim]) with
// half the coarse cell width; both levels advance with the same dt.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../../include/orcha.h"
#include "hydro.cuh"
#include "launch.h"
#include "runtime.h"

namespace orcha {
namespace {

// Fine-level guard cells of fine block f (grid.y = position in the list,
// grid.x x threads over the padded cells): from the fine block that holds the
// cell, or the coarse cell containing it; the fine level's boundary rule
// applies in its own index space.
__global__ void amr_guard_fill_kernel(const MeshDev c, const MeshDev f, const int* __restrict__ refined,
                                      const int* __restrict__ child0, const double* __restrict__ Uc,
                                      double* __restrict__ Uf) {
    const int fb = blockIdx.y;
    const long long cell = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= f.var_stride) return;
    const int nd = c.ndim, nv = c.nvar;
    int q[3];
    q[0] = (int)(cell % f.pad[0]);
    q[1] = (int)((cell / f.pad[0]) % f.pad[1]);
    q[2] = (int)(cell / ((long long)f.pad[0] * f.pad[1]));
    bool guard = false;
    for (int d = 0; d < nd; ++d) guard = guard || q[d] < kGuard || q[d] >= kGuard + c.bs[d];
    if (!guard) return;
    const int pr = refined[fb >> nd], o = fb & ((1 << nd) - 1);
    const int pc[3] = {pr % c.nb[0], (pr / c.nb[0]) % c.nb[1], pr / (c.nb[0] * c.nb[1])};
    int g[3], gc[3], bc[3];
    for (int d = 0; d < 3; ++d) {
        if (d >= nd) { g[d] = 0; gc[d] = 0; bc[d] = 0; continue; }
        const int n = 2 * c.nb[d] * c.bs[d];
        int x = (2 * pc[d] + ((o >> d) & 1)) * c.bs[d] + q[d] - kGuard;
        if (c.periodic[d]) { x %= n; x = x < 0 ? x + n : x; }
        else x = x < 0 ? 0 : (x > n - 1 ? n - 1 : x);
        g[d] = x;
        gc[d] = x / 2;
        bc[d] = gc[d] / c.bs[d];
    }
    const int b = bc[0] + c.nb[0] * (bc[1] + c.nb[1] * bc[2]);
    const double* src;
    long long off;
    if (child0[b] < 0) {
        src = Uc + (long long)b * c.blk_stride;
        off = ((long long)(nd == 3 ? gc[2] % c.bs[2] + kGuard : 0) * c.pad[1] + (gc[1] % c.bs[1] + kGuard)) * c.pad[0] +
              (gc[0] % c.bs[0] + kGuard);
    } else {
        int oo = 0;
        for (int d = 0; d < nd; ++d) oo |= ((g[d] / c.bs[d]) & 1) << d;
        src = Uf + (long long)(child0[b] + oo) * f.blk_stride;
        off = ((long long)(nd == 3 ? g[2] % c.bs[2] + kGuard : 0) * c.pad[1] + (g[1] % c.bs[1] + kGuard)) * c.pad[0] +
              (g[0] % c.bs[0] + kGuard);
    }
    double* dst = Uf + (long long)fb * f.blk_stride + cell;
    for (int v = 0; v < nv; ++v) dst[(long long)v * f.var_stride] = src[off + (long long)v * c.var_stride];
}

// Parent p = refined[blockIdx.y] <- pairwise sum of its children's 2^ndim
// fine cells (x fastest) times 1/2^ndim, per interior cell.
__global__ void amr_restrict_kernel(const MeshDev c, const int* __restrict__ refined, const double* __restrict__ Uf,
                                    double* __restrict__ Uc) {
    const int r = blockIdx.y, nd = c.ndim;
    const int ncell = c.bs[0] * c.bs[1] * c.bs[2];
    const int cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= ncell) return;
    const int loc[3] = {cell % c.bs[0], (cell / c.bs[0]) % c.bs[1], cell / (c.bs[0] * c.bs[1])};
    int o = 0, fl[3] = {0, 0, 0};
    for (int d = 0; d < nd; ++d) {
        o |= ((2 * loc[d]) / c.bs[d]) << d;
        fl[d] = (2 * loc[d]) % c.bs[d];
    }
    const double* src = Uf + (long long)((r << nd) + o) * c.blk_stride;
    double* dst = Uc + (long long)refined[r] * c.blk_stride;
    const double w = nd == 3 ? 0.125 : 0.25;
    auto at = [&](int ex, int ey, int ez) {
        return ((long long)(nd == 3 ? fl[2] + ez + kGuard : 0) * c.pad[1] + (fl[1] + ey + kGuard)) * c.pad[0] +
               (fl[0] + ex + kGuard);
    };
    const long long dc = ((long long)(nd == 3 ? loc[2] + kGuard : 0) * c.pad[1] + (loc[1] + kGuard)) * c.pad[0] +
                         (loc[0] + kGuard);
    for (int v = 0; v < c.nvar; ++v) {
        const double* s = src + (long long)v * c.var_stride;
        double t = __dadd_rn(__dadd_rn(s[at(0, 0, 0)], s[at(1, 0, 0)]), __dadd_rn(s[at(0, 1, 0)], s[at(1, 1, 0)]));
        if (nd == 3)
            t = __dadd_rn(t, __dadd_rn(__dadd_rn(s[at(0, 0, 1)], s[at(1, 0, 1)]), __dadd_rn(s[at(0, 1, 1)], s[at(1, 1, 1)])));
        dst[(long long)v * c.var_stride + dc] = __dmul_rn(w, t);
    }
}

// Flux correction of one coarse leaf block (one CTA): for each of its faces
// next to a refined block, in the order (x low, x high, y low, ...), every
// face cell's adjacent coarse cell gets (dt/dx) (F_coarse - F_fine average)
// added (high face) or subtracted (low face); faces in turn, so a corner cell
// next to two refined blocks takes its corrections in that order.
struct RefluxEntry {
    int b;          // coarse leaf block
    int mask;       // bit 2d + side: the face has a refined neighbour
    int nbr[6];     // that neighbour's coarse block id
};

__global__ void amr_reflux_kernel(const MeshDev c, const RefluxEntry* __restrict__ ents,
                                  const int* __restrict__ child0, const double* __restrict__ regc,
                                  const double* __restrict__ regf, int fsz, double* __restrict__ Uc) {
    const RefluxEntry e = ents[blockIdx.x];
    const int nd = c.ndim, nv = c.nvar;
    const double dt = *c.dt;
    for (int d = 0; d < nd; ++d) {
        const int a1 = d == 0 ? 1 : 0, a2 = d == 2 ? 1 : 2;
        const int n1 = c.bs[a1], n2 = a2 < nd ? c.bs[a2] : 1;
        const double cdc = __dmul_rn(dt, c.idx[d]);
        for (int side = 0; side < 2; ++side) {
            if (!((e.mask >> (2 * d + side)) & 1)) continue;
            const int N = e.nbr[2 * d + side];
            for (int t = threadIdx.x; t < n1 * n2; t += blockDim.x) {
                const int t1 = t % n1, t2 = t / n1;
                int loc[3] = {0, 0, 0};
                loc[d] = side ? c.bs[d] - 1 : 0;
                loc[a1] = t1;
                if (a2 < nd) loc[a2] = t2;
                const int s1 = (2 * t1) / n1, s2 = a2 < nd ? (2 * t2) / n2 : 0;
                const int o = ((side ? 0 : 1) << d) | (s1 << a1) | (s2 << a2);
                const long long fb = child0[N] + o;
                const int f1 = 2 * t1 - s1 * n1, f2 = a2 < nd ? 2 * t2 - s2 * n2 : 0;
                const double* rf = regf + (fb * 6 + 2 * d + (side ? 0 : 1)) * (long long)nv * fsz;
                const double* rc = regc + ((long long)e.b * 6 + 2 * d + side) * (long long)nv * fsz;
                const long long uc = ((long long)(nd == 3 ? loc[2] + kGuard : 0) * c.pad[1] + (loc[1] + kGuard)) * c.pad[0] +
                                     (loc[0] + kGuard);
                double* U = Uc + (long long)e.b * c.blk_stride + uc;
                for (int v = 0; v < nv; ++v) {
                    const double* r = rf + (long long)v * fsz;
                    double avg;
                    if (nd == 3) {
                        const int i00 = f2 * n1 + f1;
                        avg = __dmul_rn(0.25, __dadd_rn(__dadd_rn(r[i00], r[i00 + 1]), __dadd_rn(r[i00 + n1], r[i00 + n1 + 1])));
                    } else {
                        avg = __dmul_rn(0.5, __dadd_rn(r[f1], r[f1 + 1]));
                    }
                    const double corr = __dmul_rn(cdc, __dsub_rn(rc[(long long)v * fsz + t], avg));
                    double* u = U + (long long)v * c.var_stride;
                    *u = side ? __dadd_rn(*u, corr) : __dsub_rn(*u, corr);
                }
            }
            __syncthreads();
        }
    }
}

// One level's part of the hydro launch: its view, its blocks, its buffers
// (by current buffer) and its flux registers.
struct AmrLevel {
    MeshDev m;
    const int* ids;
    const double* Uin;
    double* Uout;
    double* reg;
};

// Both levels' blocks in one launch (so one partial last wave, not two): the
// first n0 x tiles CTAs take the coarse leaves, the rest the fine blocks;
// every CTA runs the FP64 MUSCL-Hancock step of one block's column tile with
// its guards from the padded block and records the block's face fluxes.
template <int NDIM, int TX, int TY>
__global__ void __launch_bounds__(Tile<NDIM, TX, TY>::template nb<rd, false>())
amr_hydro_kernel(const AmrLevel* __restrict__ lv, int n0, int tiles_x, int tiles_y, int fsz) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ unsigned long long red[32];
    const int ntile = tiles_x * tiles_y;
    const int b = blockIdx.x / ntile, tile = blockIdx.x % ntile;
    const bool fine = b >= n0;
    const AmrLevel& L = lv[fine ? 1 : 0];
    FluxRegIO io;
    io.reg = L.reg;
    io.fsz = fsz;
    hydro_tile<NDIM, TX, TY, rd, false, false, false, FluxRegIO>(L.m, L.ids[fine ? b - n0 : b], (tile % tiles_x) * TX,
                                                                 (tile / tiles_x) * TY, L.Uin, L.Uout, smem_raw, red,
                                                                 0, -1, 0, io);
}

template <int NDIM, int TX, int TY>
cudaError_t launch_amr_hydro_t(const AmrLevel* lv, int n0, int n1, int tiles_x, int tiles_y, int fsz,
                               cudaStream_t st) {
    using Tl = Tile<NDIM, TX, TY>;
    const size_t smem = Tl::template smem_bytes<double>();
    auto kern = amr_hydro_kernel<NDIM, TX, TY>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<dim3((unsigned)((n0 + n1) * tiles_x * tiles_y)), dim3(Tl::template nb<rd, false>()), smem, st>>>(
        lv, n0, tiles_x, tiles_y, fsz);
    return cudaGetLastError();
}

// One FP64 MUSCL-Hancock step of the n0 coarse leaves and the n1 fine blocks
// of lv[0] and lv[1], filling their flux registers.
cudaError_t launch_amr_hydro(int ndim, const int bs[3], int tx, int ty, const AmrLevel* lv, int n0, int n1, int fsz,
                             cudaStream_t st) {
    if (n0 + n1 <= 0) return cudaSuccess;
    const int ntx = bs[0] / tx, nty = bs[1] / ty;
#define ORCHA_R(ND, X, Y) \
    if (ndim == ND && tx == X && ty == Y) return launch_amr_hydro_t<ND, X, Y>(lv, n0, n1, ntx, nty, fsz, st);
    ORCHA_R(3, 16, 16) ORCHA_R(3, 16, 8) ORCHA_R(3, 8, 8) ORCHA_R(2, 16, 16) ORCHA_R(2, 16, 8) ORCHA_R(2, 8, 8)
#undef ORCHA_R
    return cudaErrorInvalidConfiguration;
}

}  // namespace
}  // namespace orcha

struct orcha_amr {
    orcha_mesh* coarse = nullptr;         // level 0 over the caller's coarse buffers
    orcha::MeshDev md0{}, md1{};          // kernels' views of both levels (shared smax and err)
    double* fine[2] = {nullptr, nullptr}; // caller-owned fine state buffers
    int nref = 0, nfine = 0, nleaf = 0, fsz = 0, tx = 8, ty = 8;
    unsigned long long* smax = nullptr;   // coarse blocks, then fine blocks
    int* refined_dev = nullptr;
    int* child0_dev = nullptr;
    int* leaves_dev = nullptr;            // coarse leaf ids
    int* fine_ids_dev = nullptr;          // 0 .. nfine-1
    int* all_coarse_dev = nullptr;        // 0 .. nblk0-1
    double* reg0 = nullptr;               // flux registers of the coarse blocks
    double* reg1 = nullptr;               // and of the fine blocks
    orcha::RefluxEntry* reflux_dev = nullptr;
    int nreflux = 0;
    orcha::AmrLevel* levels_dev = nullptr; // [current buffer][coarse, fine]
    double* staging = nullptr;            // host load/store staging
};

namespace {

orcha_status amr_fail(cudaError_t e, const char* what) { return orcha::cuda_error(e, what); }

size_t fine_state_elems(const orcha_mesh_desc* d, int32_t nref) {
    const size_t per = orcha_state_elems(d) / ((size_t)d->nb[0] * d->nb[1] * d->nb[2]);
    return per * (size_t)nref * (1u << d->ndim);
}

}  // namespace

extern "C" {

size_t orcha_amr_fine_elems(const orcha_mesh_desc* coarse, int32_t nref) {
    if (!coarse || nref < 0 || orcha_state_elems(coarse) == 0) return 0;
    return fine_state_elems(coarse, nref);
}

orcha_status orcha_amr_destroy(orcha_amr* a) {
    if (!a) return ORCHA_OK;
    cudaDeviceSynchronize();
    cudaFree(a->smax);
    cudaFree(a->refined_dev);
    cudaFree(a->child0_dev);
    cudaFree(a->leaves_dev);
    cudaFree(a->fine_ids_dev);
    cudaFree(a->all_coarse_dev);
    cudaFree(a->reg0);
    cudaFree(a->reg1);
    cudaFree(a->reflux_dev);
    cudaFree(a->levels_dev);
    cudaFree(a->staging);
    orcha_mesh_destroy(a->coarse);
    delete a;
    return ORCHA_OK;
}

orcha_status orcha_amr_create(const orcha_mesh_desc* desc, const int32_t* refined, int32_t nref, double* fine0_dev,
                              double* fine1_dev, orcha_amr** out) {
    if (!desc || !out || nref < 0 || (nref > 0 && (!refined || !fine0_dev || !fine1_dev)))
        return orcha::set_error(ORCHA_ERR_INVALID, "amr_create: null argument or negative count");
    *out = nullptr;
    if ((((uintptr_t)fine0_dev) | ((uintptr_t)fine1_dev)) & 15)
        return orcha::set_error(ORCHA_ERR_INVALID, "amr_create: fine state buffers must be 16-byte aligned");
    orcha_amr* a = new orcha_amr();
    orcha_status s = orcha_mesh_create(desc, &a->coarse);
    if (s) { delete a; return s; }
    const orcha::MeshDev& c = a->coarse->dev;
    const int nblk0 = a->coarse->nblk, nd = c.ndim, nch = 1 << nd;
    std::vector<int> child0(nblk0, -1);
    for (int r = 0; r < nref; ++r) {
        if (refined[r] < 0 || refined[r] >= nblk0 || child0[refined[r]] >= 0) {
            orcha_amr_destroy(a);
            return orcha::set_error(ORCHA_ERR_INVALID, "amr_create: refined ids out of range or repeated");
        }
        child0[refined[r]] = r * nch;
    }
    a->nref = nref;
    a->nfine = nref * nch;
    a->fine[0] = fine0_dev;
    a->fine[1] = fine1_dev;
    a->tx = c.bs[0] >= 16 ? 16 : 8;
    a->ty = c.bs[1] >= 16 ? 16 : 8;
    a->fsz = 0;
    for (int d = 0; d < 3; ++d) {
        const int a1 = d == 0 ? 1 : 0, a2 = d == 2 ? 1 : 2;
        a->fsz = std::max(a->fsz, c.bs[a1] * c.bs[a2]);
    }
    std::vector<int> leaves, all_coarse(nblk0), fine_ids(a->nfine);
    for (int b = 0; b < nblk0; ++b) {
        all_coarse[b] = b;
        if (child0[b] < 0) leaves.push_back(b);
    }
    for (int f = 0; f < a->nfine; ++f) fine_ids[f] = f;
    a->nleaf = (int)leaves.size();
    // reflux entries: coarse leaves with a refined face neighbour (coarse boundary rule)
    std::vector<orcha::RefluxEntry> ents;
    for (int b : leaves) {
        const int bc[3] = {b % c.nb[0], (b / c.nb[0]) % c.nb[1], b / (c.nb[0] * c.nb[1])};
        orcha::RefluxEntry e{};
        e.b = b;
        for (int d = 0; d < nd; ++d)
            for (int side = 0; side < 2; ++side) {
                int nbc[3] = {bc[0], bc[1], bc[2]};
                nbc[d] += side ? 1 : -1;
                if (nbc[d] < 0 || nbc[d] >= c.nb[d]) {
                    if (!c.periodic[d]) continue;
                    nbc[d] = (nbc[d] + c.nb[d]) % c.nb[d];
                }
                const int N = nbc[0] + c.nb[0] * (nbc[1] + c.nb[1] * nbc[2]);
                if (child0[N] < 0) continue;
                e.mask |= 1 << (2 * d + side);
                e.nbr[2 * d + side] = N;
            }
        if (e.mask) ents.push_back(e);
    }
    a->nreflux = (int)ents.size();
    // the fine level's view: a list of nfine blocks, half the cell width
    a->md0 = c;
    a->md1 = c;
    a->md1.nb[0] = std::max(1, a->nfine);
    a->md1.nb[1] = a->md1.nb[2] = 1;
    for (int d = 0; d < 3; ++d) a->md1.idx[d] = d < nd ? 1.0 / ((desc->hi[d] - desc->lo[d]) / (double)(2 * c.nb[d] * c.bs[d])) : c.idx[d];
    const size_t regsz = (size_t)6 * c.nvar * a->fsz;
    cudaError_t e = cudaMalloc(&a->smax, sizeof(unsigned long long) * (size_t)(nblk0 + a->nfine));
    if (e == cudaSuccess) e = cudaMemset(a->smax, 0, sizeof(unsigned long long) * (size_t)(nblk0 + a->nfine));
    auto upload = [&](int** dst, const std::vector<int>& src) {
        if (e != cudaSuccess) return;
        e = cudaMalloc(dst, sizeof(int) * std::max<size_t>(1, src.size()));
        if (e == cudaSuccess && !src.empty())
            e = cudaMemcpy(*dst, src.data(), sizeof(int) * src.size(), cudaMemcpyHostToDevice);
    };
    upload(&a->refined_dev, std::vector<int>(refined, refined + nref));
    upload(&a->child0_dev, child0);
    upload(&a->leaves_dev, leaves);
    upload(&a->fine_ids_dev, fine_ids);
    upload(&a->all_coarse_dev, all_coarse);
    if (e == cudaSuccess) e = cudaMalloc(&a->reg0, sizeof(double) * regsz * nblk0);
    if (e == cudaSuccess) e = cudaMalloc(&a->reg1, sizeof(double) * regsz * std::max(1, a->nfine));
    if (e == cudaSuccess) e = cudaMalloc(&a->reflux_dev, sizeof(orcha::RefluxEntry) * std::max<size_t>(1, ents.size()));
    if (e == cudaSuccess && !ents.empty())
        e = cudaMemcpy(a->reflux_dev, ents.data(), sizeof(orcha::RefluxEntry) * ents.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = orcha::configure_hydro(nd, a->tx, a->ty);
    if (e != cudaSuccess) {
        orcha_status st = amr_fail(e, "amr_create");
        orcha_amr_destroy(a);
        return st;
    }
    a->md0.smax = a->smax;
    a->md1.smax = a->smax + nblk0;
    // the hydro launch's per-level arguments, for either current buffer
    orcha::AmrLevel lv[2][2];
    for (int cur = 0; cur < 2; ++cur) {
        lv[cur][0] = {a->md0, a->leaves_dev, desc->state_dev[cur], desc->state_dev[cur ^ 1], a->reg0};
        lv[cur][1] = {a->md1, a->fine_ids_dev, a->fine[cur], a->fine[cur ^ 1], a->reg1};
    }
    e = cudaMalloc(&a->levels_dev, sizeof(lv));
    if (e == cudaSuccess) e = cudaMemcpy(a->levels_dev, lv, sizeof(lv), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        orcha_status st = amr_fail(e, "amr_create");
        orcha_amr_destroy(a);
        return st;
    }
    *out = a;
    return ORCHA_OK;
}

// Copy both levels' interiors in or out of the current buffers:
// coarse [block][var][k][j][i] over all coarse blocks, fine [fine block]...
static orcha_status amr_copy(orcha_amr* a, double* coarse, double* fine, int host, bool in, cudaStream_t st) {
    const orcha::MeshDev& c = a->md0;
    const size_t ncell = (size_t)c.bs[0] * c.bs[1] * c.bs[2];
    const size_t n0 = (size_t)a->coarse->nblk * c.nvar * ncell, n1 = (size_t)a->nfine * c.nvar * ncell;
    const int cur = a->coarse->cur;
    if (host && !a->staging) {
        cudaError_t e = cudaMalloc(&a->staging, sizeof(double) * std::max<size_t>(1, std::max(n0, n1)));
        if (e != cudaSuccess) return amr_fail(e, "amr staging");
    }
    for (int lev = 0; lev < 2; ++lev) {
        const size_t n = lev ? n1 : n0;
        if (n == 0) continue;
        double* user = lev ? fine : coarse;
        double* state = lev ? a->fine[cur] : a->coarse->desc.state_dev[cur];
        const orcha::MeshDev& m = lev ? a->md1 : a->md0;
        double* dev = host ? a->staging : user;
        cudaError_t e = cudaSuccess;
        if (in) {
            if (host) e = cudaMemcpyAsync(dev, user, n * sizeof(double), cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess) e = orcha::launch_pack(m, dev, state, st);
        } else {
            e = orcha::launch_unpack(m, state, dev, st);
            if (e == cudaSuccess && host) e = cudaMemcpyAsync(user, dev, n * sizeof(double), cudaMemcpyDeviceToHost, st);
        }
        if (e == cudaSuccess && host) e = cudaStreamSynchronize(st);   // the staging buffer is reused
        if (e != cudaSuccess) return amr_fail(e, in ? "amr_load" : "amr_store");
    }
    return ORCHA_OK;
}

orcha_status orcha_amr_load(orcha_amr* a, const double* coarse, const double* fine, int32_t host_ptr, void* stream) {
    if (!a || !coarse || (a->nfine && !fine)) return orcha::set_error(ORCHA_ERR_INVALID, "amr_load: null argument");
    return amr_copy(a, const_cast<double*>(coarse), const_cast<double*>(fine), host_ptr, true, (cudaStream_t)stream);
}

orcha_status orcha_amr_store(orcha_amr* a, double* coarse, double* fine, int32_t host_ptr, void* stream) {
    if (!a || !coarse || (a->nfine && !fine)) return orcha::set_error(ORCHA_ERR_INVALID, "amr_store: null argument");
    return amr_copy(a, coarse, fine, host_ptr, false, (cudaStream_t)stream);
}

orcha_status orcha_amr_advance(orcha_amr* a, int32_t nsteps, int32_t init_dt, void* stream) {
    if (!a || nsteps < 0) return orcha::set_error(ORCHA_ERR_INVALID, "amr_advance: bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    const orcha::MeshDev& c = a->md0;
    const int nblk0 = a->coarse->nblk, nd = c.ndim;
    const int ncell = c.bs[0] * c.bs[1] * c.bs[2];
    const unsigned rgrid = (unsigned)((ncell + 255) / 256);
    const unsigned ggrid = (unsigned)((a->md1.var_stride + 255) / 256);
    auto restrict_into = [&](int buf) -> cudaError_t {
        if (!a->nref) return cudaSuccess;
        orcha::amr_restrict_kernel<<<dim3(rgrid, (unsigned)a->nref), 256, 0, st>>>(
            c, a->refined_dev, a->fine[buf], a->coarse->desc.state_dev[buf]);
        return cudaGetLastError();
    };
    auto leaf_speeds_dt = [&](int buf) -> cudaError_t {
        cudaError_t e = cudaMemsetAsync(a->smax, 0, sizeof(unsigned long long) * (size_t)(nblk0 + a->nfine), st);
        if (e == cudaSuccess && a->nleaf)
            e = orcha::launch_signal_speed(a->md0, a->leaves_dev, a->nleaf, a->coarse->desc.state_dev[buf], st);
        if (e == cudaSuccess && a->nfine)
            e = orcha::launch_signal_speed(a->md1, a->fine_ids_dev, a->nfine, a->fine[buf], st);
        if (e == cudaSuccess) e = orcha::launch_dt_reduce(a->md0, nblk0 + a->nfine, a->coarse->desc.dt_dev, st);
        return e;
    };
    int cur = a->coarse->cur;
    cudaError_t e = restrict_into(cur);
    if (e == cudaSuccess && init_dt) e = leaf_speeds_dt(cur);
    for (int n = 0; n < nsteps && e == cudaSuccess; ++n) {
        double* Uc = a->coarse->desc.state_dev[cur];
        double* Uc1 = a->coarse->desc.state_dev[cur ^ 1];
        double* Uf = a->fine[cur];
        e = orcha::launch_guard_fill(c, a->all_coarse_dev, nblk0, Uc, st);
        if (e == cudaSuccess && a->nfine) {
            orcha::amr_guard_fill_kernel<<<dim3(ggrid, (unsigned)a->nfine), 256, 0, st>>>(
                c, a->md1, a->refined_dev, a->child0_dev, Uc, Uf);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess)
            e = orcha::launch_amr_hydro(nd, c.bs, a->tx, a->ty, a->levels_dev + 2 * cur, a->nleaf, a->nfine, a->fsz, st);
        if (e == cudaSuccess && a->nreflux) {
            orcha::amr_reflux_kernel<<<(unsigned)a->nreflux, 256, 0, st>>>(c, a->reflux_dev, a->child0_dev, a->reg0,
                                                                         a->reg1, a->fsz, Uc1);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = restrict_into(cur ^ 1);
        if (e == cudaSuccess) e = leaf_speeds_dt(cur ^ 1);
        cur ^= 1;
        a->coarse->cur = cur;
    }
    if (e != cudaSuccess) return amr_fail(e, "amr_advance");
    return ORCHA_OK;
}

orcha_status orcha_amr_poll(orcha_amr* a, void* stream, int32_t* device_error) {
    if (!a) return orcha::set_error(ORCHA_ERR_INVALID, "amr_poll: null argument");
    return orcha_mesh_poll(a->coarse, stream, device_error);
}

}  // extern "C"
