// api.cu -- host runtime behind include/orcha.h: mesh and packet objects,
// argument checks, kernel launches, CUDA-graph capture of whole steps.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/orcha.h"
#include "common.cuh"
#include "launch.h"
#include "worklist.h"

using orcha::MeshDev;

namespace {

thread_local std::string g_last_error;

orcha_status fail(orcha_status code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

orcha_status cuda_fail(cudaError_t e, const char* what) {
    return fail(e == cudaErrorMemoryAllocation ? ORCHA_ERR_OOM : ORCHA_ERR_CUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

#define ORCHA_CUDA(call, what)                         \
    do {                                               \
        cudaError_t e_ = (call);                       \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

bool valid_bs(int b) { return b == 8 || b == 16 || b == 32; }



}  // namespace

#include "runtime.h"

extern "C" {

size_t orcha_state_elems(const orcha_mesh_desc* d) {
    if (!d || (d->ndim != 2 && d->ndim != 3)) return 0;
    size_t n = (size_t)(d->ndim + 2);
    for (int a = 0; a < 3; ++a) {
        if (d->nb[a] < 1 || d->bs[a] < 1) return 0;
        n *= (size_t)d->nb[a] * (size_t)(a < d->ndim ? d->bs[a] + 2 * orcha::kGuard : 1);
    }
    return n;
}

}  // extern "C"

namespace orcha {

orcha_status set_error(orcha_status code, const char* msg) { return fail(code, "%s", msg); }

orcha_status cuda_error(cudaError_t e, const char* what) { return cuda_fail(e, what); }

// Check a descriptor and fill the kernels' view of it (without the smax and
// err scratch pointers). Host-only; touches no device state.
orcha_status mesh_dev_from_desc(const orcha_mesh_desc* d, MeshDev* out, long long* nblk_out) {
    if (!d || !out) return fail(ORCHA_ERR_INVALID, "null descriptor");
    if (d->ndim != 2 && d->ndim != 3) return fail(ORCHA_ERR_INVALID, "mesh: ndim must be 2 or 3");
    for (int a = 0; a < 3; ++a) {
        if (d->nb[a] < 1) return fail(ORCHA_ERR_INVALID, "mesh: nb[%d] < 1", a);
        if (a < d->ndim && !valid_bs(d->bs[a]))
            return fail(ORCHA_ERR_INVALID, "mesh: bs[%d] = %d (must be 8, 16 or 32)", a, d->bs[a]);
        if (a >= d->ndim && (d->bs[a] != 1 || d->nb[a] != 1))
            return fail(ORCHA_ERR_INVALID, "mesh: 2D meshes need nb[2] = bs[2] = 1");
        if (a < d->ndim && !(d->hi[a] > d->lo[a])) return fail(ORCHA_ERR_INVALID, "mesh: hi[%d] <= lo[%d]", a, a);
        if (d->periodic[a] != 0 && d->periodic[a] != 1) return fail(ORCHA_ERR_INVALID, "mesh: periodic flag");
    }
    if (!(d->gamma > 1.0) || !(d->cfl > 0.0)) return fail(ORCHA_ERR_INVALID, "mesh: need gamma > 1, cfl > 0");
    const long long nblk = (long long)d->nb[0] * d->nb[1] * d->nb[2];
    if (nblk > (1LL << 30)) return fail(ORCHA_ERR_INVALID, "mesh: too many blocks");
    MeshDev v{};
    v.ndim = d->ndim;
    v.nvar = d->ndim + 2;
    for (int a = 0; a < 3; ++a) {
        v.nb[a] = d->nb[a];
        v.bs[a] = d->bs[a];
        v.pad[a] = a < d->ndim ? d->bs[a] + 2 * orcha::kGuard : 1;
        v.periodic[a] = d->periodic[a];
        // dx_d = (hi_d - lo_d) / N_d and 1/dx_d, formed in FP64 exactly as the definition does
        const double dx = (d->hi[a] - d->lo[a]) / (double)(d->nb[a] * d->bs[a]);
        v.idx[a] = 1.0 / dx;
    }
    v.var_stride = (long long)v.pad[0] * v.pad[1] * v.pad[2];
    v.blk_stride = v.var_stride * v.nvar;
    v.gamma = d->gamma;
    v.gm1 = d->gamma - 1.0;
    v.igm1 = 1.0 / (d->gamma - 1.0);
    v.cfl = d->cfl;
    v.dt = d->dt_dev;
    *out = v;
    if (nblk_out) *nblk_out = nblk;
    return ORCHA_OK;
}

}  // namespace orcha

extern "C" {

orcha_status orcha_mesh_create(const orcha_mesh_desc* d, orcha_mesh** out) {
    if (!d || !out) return fail(ORCHA_ERR_INVALID, "mesh_create: null argument");
    *out = nullptr;
    MeshDev v;
    long long nblk = 0;
    orcha_status st = orcha::mesh_dev_from_desc(d, &v, &nblk);
    if (st) return st;
    if (!d->state_dev[0] || !d->state_dev[1] || !d->dt_dev || d->state_dev[0] == d->state_dev[1])
        return fail(ORCHA_ERR_INVALID, "mesh_create: two distinct state buffers and dt_dev are required");
    // the hydro kernels load x-neighbour pairs of the state as 16-byte vectors
    if ((((uintptr_t)d->state_dev[0] | (uintptr_t)d->state_dev[1]) & 15) || ((uintptr_t)d->dt_dev & 7))
        return fail(ORCHA_ERR_INVALID, "mesh_create: state buffers must be 16-byte aligned, dt_dev 8-byte aligned");

    orcha_mesh* m = new orcha_mesh();
    m->desc = *d;
    m->nblk = (int)nblk;
    cudaGetDevice(&m->device);
    m->dev = v;
    m->ncell = (long long)d->bs[0] * d->bs[1] * d->bs[2];

    cudaError_t e = cudaMalloc(&m->smax, sizeof(unsigned long long) * nblk);
    if (e == cudaSuccess) e = cudaMalloc(&m->err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(m->smax, 0, sizeof(unsigned long long) * nblk);
    if (e == cudaSuccess) e = cudaMemset(m->err, 0, sizeof(int));
    // default tile: 16 wide where the block allows it
    m->tile_x = d->bs[0] >= 16 ? 16 : 8;
    m->tile_y = d->bs[1] >= 16 ? 16 : 8;
    if (e == cudaSuccess) e = orcha::configure_hydro(d->ndim, m->tile_x, m->tile_y);
    if (e != cudaSuccess) {
        orcha_status s = cuda_fail(e, "mesh_create");
        orcha_mesh_destroy(m);
        return s;
    }
    m->dev.smax = m->smax;
    m->dev.err = m->err;
    *out = m;
    return ORCHA_OK;
}

orcha_status orcha_mesh_destroy(orcha_mesh* m) {
    if (!m) return ORCHA_OK;
    cudaDeviceSynchronize();
    for (auto& g : m->graphs) cudaGraphExecDestroy(g.exec);
    cudaFree(m->smax);
    cudaFree(m->err);
    cudaFree(m->staging);
    delete m;
    return ORCHA_OK;
}

int32_t orcha_mesh_current(const orcha_mesh* m) { return m ? m->cur : -1; }

orcha_status orcha_mesh_swap(orcha_mesh* m) {
    if (!m) return fail(ORCHA_ERR_INVALID, "mesh_swap: null mesh");
    m->cur ^= 1;
    return ORCHA_OK;
}

orcha_status orcha_mesh_set_tile(orcha_mesh* m, int32_t tx, int32_t ty) {
    if (!m) return fail(ORCHA_ERR_INVALID, "mesh_set_tile: null mesh");
    if (!orcha::hydro_tile_supported(m->dev.ndim, tx, ty))
        return fail(ORCHA_ERR_UNSUPPORTED, "mesh_set_tile: no %dx%d tile variant", tx, ty);
    if (m->dev.bs[0] % tx || m->dev.bs[1] % ty)
        return fail(ORCHA_ERR_INVALID, "mesh_set_tile: %dx%d does not divide the block", tx, ty);
    ORCHA_CUDA(orcha::configure_hydro(m->dev.ndim, tx, ty), "mesh_set_tile");
    m->tile_x = tx;
    m->tile_y = ty;
    return ORCHA_OK;
}

orcha_status orcha_mesh_get_tile(const orcha_mesh* m, int32_t* tx, int32_t* ty) {
    if (!m || !tx || !ty) return fail(ORCHA_ERR_INVALID, "mesh_get_tile: null argument");
    *tx = m->tile_x;
    *ty = m->tile_y;
    return ORCHA_OK;
}

static orcha_status ensure_staging(orcha_mesh* m) {
    if (m->staging) return ORCHA_OK;
    const size_t n = (size_t)m->nblk * m->dev.nvar * m->ncell;
    ORCHA_CUDA(cudaMalloc(&m->staging, n * sizeof(double)), "staging buffer");
    return ORCHA_OK;
}

orcha_status orcha_mesh_load(orcha_mesh* m, const double* interior, int32_t host_ptr, void* stream) {
    if (!m || !interior) return fail(ORCHA_ERR_INVALID, "mesh_load: null argument");
    cudaStream_t st = (cudaStream_t)stream;
    const double* src = interior;
    if (host_ptr) {
        orcha_status s = ensure_staging(m);
        if (s) return s;
        const size_t bytes = (size_t)m->nblk * m->dev.nvar * m->ncell * sizeof(double);
        ORCHA_CUDA(cudaMemcpyAsync(m->staging, interior, bytes, cudaMemcpyHostToDevice, st), "mesh_load H2D");
        src = m->staging;
    }
    ORCHA_CUDA(orcha::launch_pack(m->dev, src, m->desc.state_dev[m->cur], st), "mesh_load pack");
    return ORCHA_OK;
}

orcha_status orcha_mesh_store(orcha_mesh* m, double* interior, int32_t host_ptr, void* stream) {
    if (!m || !interior) return fail(ORCHA_ERR_INVALID, "mesh_store: null argument");
    cudaStream_t st = (cudaStream_t)stream;
    if (host_ptr) {
        orcha_status s = ensure_staging(m);
        if (s) return s;
        ORCHA_CUDA(orcha::launch_unpack(m->dev, m->desc.state_dev[m->cur], m->staging, st), "mesh_store unpack");
        const size_t bytes = (size_t)m->nblk * m->dev.nvar * m->ncell * sizeof(double);
        ORCHA_CUDA(cudaMemcpyAsync(interior, m->staging, bytes, cudaMemcpyDeviceToHost, st), "mesh_store D2H");
        return ORCHA_OK;
    }
    ORCHA_CUDA(orcha::launch_unpack(m->dev, m->desc.state_dev[m->cur], interior, st), "mesh_store unpack");
    return ORCHA_OK;
}

orcha_status orcha_mesh_init_region(orcha_mesh* m, int32_t kind, const int32_t region[4], const double u_in[5],
                                    const double u_out[5], void* stream) {
    if (!m || !region || !u_in || !u_out) return fail(ORCHA_ERR_INVALID, "mesh_init_region: null argument");
    if (kind != ORCHA_INIT_SPHERE && kind != ORCHA_INIT_HALF_SPACE)
        return fail(ORCHA_ERR_INVALID, "mesh_init_region: kind must be SPHERE or HALF_SPACE");
    if (kind == ORCHA_INIT_HALF_SPACE && (region[0] < 0 || region[0] >= m->dev.ndim))
        return fail(ORCHA_ERR_INVALID, "mesh_init_region: axis outside [0, ndim)");
    orcha::RegionStates rs;
    for (int v = 0; v < 5; ++v) {
        rs.in[v] = u_in[v];
        rs.out[v] = u_out[v];
    }
    ORCHA_CUDA(orcha::launch_region_init(m->dev, m->desc.state_dev[m->cur], kind,
                                         make_int4(region[0], region[1], region[2], region[3]), rs,
                                         (cudaStream_t)stream),
               "mesh_init_region");
    return ORCHA_OK;
}

orcha_status orcha_packet_create(orcha_mesh* m, const int32_t* ids, int32_t n, orcha_packet** out) {
    if (!m || !ids || !out) return fail(ORCHA_ERR_INVALID, "packet_create: null argument");
    *out = nullptr;
    if (n < 1) return fail(ORCHA_ERR_INVALID, "packet_create: empty packet");
    if (n > m->nblk) return fail(ORCHA_ERR_INVALID, "packet_create: more ids than blocks");
    std::vector<char> seen((size_t)m->nblk, 0);
    for (int i = 0; i < n; ++i) {
        if (ids[i] < 0 || ids[i] >= m->nblk)
            return fail(ORCHA_ERR_INVALID, "packet_create: block id %d outside [0, %d)", ids[i], m->nblk);
        if (seen[ids[i]]) return fail(ORCHA_ERR_INVALID, "packet_create: block id %d repeated", ids[i]);
        seen[ids[i]] = 1;
    }
    orcha_packet* p = new orcha_packet();
    p->mesh = m;
    p->n = n;
    p->ids.assign(ids, ids + n);
    cudaError_t e = cudaMalloc(&p->ids_dev, sizeof(int) * n);
    if (e == cudaSuccess) e = cudaMemcpy(p->ids_dev, ids, sizeof(int) * n, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(p->ids_dev);
        delete p;
        return cuda_fail(e, "packet_create");
    }
    *out = p;
    return ORCHA_OK;
}

orcha_status orcha_packet_destroy(orcha_packet* p) {
    if (!p) return ORCHA_OK;
    cudaDeviceSynchronize();
    cudaFree(p->ids_dev);
    cudaFree(p->staging);
    delete p;
    return ORCHA_OK;
}

static orcha_status ensure_packet_staging(orcha_packet* p) {
    if (p->staging) return ORCHA_OK;
    const size_t n = (size_t)p->n * p->mesh->dev.nvar * p->mesh->ncell;
    ORCHA_CUDA(cudaMalloc(&p->staging, n * sizeof(double)), "packet staging buffer");
    return ORCHA_OK;
}

orcha_status orcha_packet_unpack(orcha_packet* p, double* dst, int32_t dst_is_host, void* stream) {
    if (!p) return fail(ORCHA_ERR_INVALID, "packet_unpack: null packet");
    if (!dst) return ORCHA_OK;                       // blocks are resident and were updated in place
    orcha_mesh* m = p->mesh;
    cudaStream_t st = (cudaStream_t)stream;
    const double* U = m->desc.state_dev[m->cur];
    if (!dst_is_host) {
        ORCHA_CUDA(orcha::launch_unpack_ids(m->dev, p->ids_dev, p->n, U, dst, st), "packet_unpack");
        return ORCHA_OK;
    }
    orcha_status s = ensure_packet_staging(p);
    if (s) return s;
    ORCHA_CUDA(orcha::launch_unpack_ids(m->dev, p->ids_dev, p->n, U, p->staging, st), "packet_unpack");
    const size_t bytes = (size_t)p->n * m->dev.nvar * m->ncell * sizeof(double);
    ORCHA_CUDA(cudaMemcpyAsync(dst, p->staging, bytes, cudaMemcpyDeviceToHost, st), "packet_unpack D2H");
    return ORCHA_OK;
}

orcha_status orcha_packet_pack(orcha_packet* p, const double* src, int32_t src_is_host, void* stream) {
    if (!p || !src) return fail(ORCHA_ERR_INVALID, "packet_pack: null argument");
    orcha_mesh* m = p->mesh;
    cudaStream_t st = (cudaStream_t)stream;
    const double* from = src;
    if (src_is_host) {
        orcha_status s = ensure_packet_staging(p);
        if (s) return s;
        const size_t bytes = (size_t)p->n * m->dev.nvar * m->ncell * sizeof(double);
        ORCHA_CUDA(cudaMemcpyAsync(p->staging, src, bytes, cudaMemcpyHostToDevice, st), "packet_pack H2D");
        from = p->staging;
    }
    ORCHA_CUDA(orcha::launch_pack_ids(m->dev, p->ids_dev, p->n, from, m->desc.state_dev[m->cur], st), "packet_pack");
    return ORCHA_OK;
}

orcha_status orcha_packet_run(orcha_packet* p, orcha_task task, void* stream) {
    if (!p) return fail(ORCHA_ERR_INVALID, "packet_run: null packet");
    orcha_mesh* m = p->mesh;
    if (!m->dev.smax || !m->dev.err || m->dev.dt != m->desc.dt_dev)
        return fail(ORCHA_ERR_INVALID, "packet_run: mesh scratch not set up");
    cudaStream_t st = (cudaStream_t)stream;
    double* cur = m->desc.state_dev[m->cur];
    double* nxt = m->desc.state_dev[m->cur ^ 1];
    cudaError_t e;
    switch (task) {
        case ORCHA_TASK_GUARD_FILL: e = orcha::launch_guard_fill(m->dev, p->ids_dev, p->n, cur, st); break;
        case ORCHA_TASK_HYDRO_FP64:
        case ORCHA_TASK_HYDRO_F32FLUX:
        case ORCHA_TASK_HYDRO_F32FLUX_FFSUM:
        case ORCHA_TASK_HYDRO_FF:
        case ORCHA_TASK_RK2_STAGE1:
        case ORCHA_TASK_RK2_STAGE2:
        case ORCHA_TASK_RK2_F32FLUX_STAGE1:
        case ORCHA_TASK_RK2_F32FLUX_STAGE2:
        case ORCHA_TASK_RK2_FF_STAGE1:
        case ORCHA_TASK_RK2_FF_STAGE2:
            e = orcha::launch_hydro(m->dev, m->tile_x, m->tile_y, orcha::prec_of(task), p->ids_dev, p->n, cur, nxt,
                                    orcha::stage_of(task), st);
            break;
        case ORCHA_TASK_SIGNAL_SPEED: e = orcha::launch_signal_speed(m->dev, p->ids_dev, p->n, cur, st); break;
        default: return fail(ORCHA_ERR_INVALID, "packet_run: unknown task %d", (int)task);
    }
    if (e != cudaSuccess) return cuda_fail(e, "packet_run launch");
    return ORCHA_OK;
}

orcha_status orcha_dt_reduce(orcha_mesh* m, void* stream) {
    if (!m) return fail(ORCHA_ERR_INVALID, "dt_reduce: null mesh");
    if (!m->dev.smax || !m->dev.err) return fail(ORCHA_ERR_INVALID, "dt_reduce: mesh scratch not set up");
    ORCHA_CUDA(orcha::launch_dt_reduce(m->dev, m->nblk, m->desc.dt_dev, (cudaStream_t)stream), "dt_reduce launch");
    return ORCHA_OK;
}

static orcha_status enqueue_steps(orcha_mesh* m, orcha_packet* const* pk, int npk, orcha_task task, int nsteps,
                                  int init_dt, void* stream) {
    orcha_status s;
    if (init_dt) {
        // the packets cover every block: one launch over the whole mesh
        ORCHA_CUDA(orcha::launch_signal_speed_all(m->dev, m->nblk, m->desc.state_dev[m->cur], (cudaStream_t)stream,
                                                  orcha::prec_f32_dt(orcha::prec_of(task))),
                   "advance signal speed");
        if ((s = orcha_dt_reduce(m, stream))) return s;
    }
    // a Heun step is two sweeps (stage 1, swap, stage 2, swap), every other
    // step one; each sweep refreshes the guards of the state it reads
    const bool rk = orcha::is_rk_step_task(task);
    const orcha_task sweeps[2] = {rk ? orcha::rk_stage_task(task, 1) : task, orcha::rk_stage_task(task, 2)};
    for (int n = 0; n < nsteps; ++n) {
        for (int k = 0; k < (rk ? 2 : 1); ++k) {
            for (int i = 0; i < npk; ++i)
                if ((s = orcha_packet_run(pk[i], ORCHA_TASK_GUARD_FILL, stream))) return s;
            for (int i = 0; i < npk; ++i)
                if ((s = orcha_packet_run(pk[i], sweeps[k], stream))) return s;
            if (!rk || k == 1)
                if ((s = orcha_dt_reduce(m, stream))) return s;
            m->cur ^= 1;
        }
    }
    return ORCHA_OK;
}

orcha_status orcha_mesh_advance(orcha_mesh* m, orcha_packet* const* pk, int32_t npk, orcha_task task, int32_t nsteps,
                                int32_t init_dt, int32_t use_graph, void* stream) {
    if (!m || (!pk && npk > 0) || npk < 0 || nsteps < 0) return fail(ORCHA_ERR_INVALID, "mesh_advance: bad argument");
    if (!orcha::is_step_task(task))
        return fail(ORCHA_ERR_INVALID, "mesh_advance: task must be a whole-step hydro task");
    if (orcha::prec_is_fused(orcha::prec_of(task)))
        return fail(ORCHA_ERR_UNSUPPORTED, "mesh_advance: fused two-application tasks run through orcha_batch_advance");
    long long covered = 0;
    for (int i = 0; i < npk; ++i) {
        if (!pk[i] || pk[i]->mesh != m) return fail(ORCHA_ERR_INVALID, "mesh_advance: packet %d not of this mesh", i);
        covered += pk[i]->n;
    }
    if (covered != m->nblk)
        return fail(ORCHA_ERR_INVALID, "mesh_advance: packets cover %lld ids, the mesh has %d blocks", covered, m->nblk);
    if (!use_graph) return enqueue_steps(m, pk, npk, task, nsteps, init_dt, stream);

    cudaStream_t st = (cudaStream_t)stream;
    if (st == nullptr) return fail(ORCHA_ERR_INVALID, "mesh_advance: graph capture needs a non-default stream");
    const int start = m->cur;
    for (auto& g : m->graphs) {
        if (g.task == task && g.nsteps == nsteps && g.init_dt == init_dt && g.start_cur == start &&
            g.packets.size() == (size_t)npk && std::equal(g.packets.begin(), g.packets.end(), pk)) {
            ORCHA_CUDA(cudaGraphLaunch(g.exec, st), "mesh_advance graph launch");
            m->cur = start ^ ((orcha::is_rk_step_task(task) ? 0 : nsteps) & 1);
            return ORCHA_OK;
        }
    }
    ORCHA_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal), "begin capture");
    orcha_status s = enqueue_steps(m, pk, npk, task, nsteps, init_dt, stream);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(st, &graph);
    m->cur = start;
    if (s) { if (graph) cudaGraphDestroy(graph); return s; }
    if (e != cudaSuccess) return cuda_fail(e, "end capture");
    orcha::GraphEntry g;
    g.packets.assign(pk, pk + npk);
    g.task = task;
    g.nsteps = nsteps;
    g.init_dt = init_dt;
    g.start_cur = start;
    e = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "graph instantiate");
    m->graphs.push_back(g);
    ORCHA_CUDA(cudaGraphLaunch(g.exec, st), "mesh_advance graph launch");
    m->cur = start ^ ((orcha::is_rk_step_task(task) ? 0 : nsteps) & 1);
    return ORCHA_OK;
}

// ---------------------------------------------------------------- batches (persistent path)

orcha_status orcha_batch_destroy(orcha_batch* b) {
    if (!b) return ORCHA_OK;
    cudaDeviceSynchronize();
    for (auto& g : b->graphs) cudaGraphExecDestroy(g.exec);
    for (auto& l : b->lists) {
        cudaFree(l.items_dev);
        cudaFree(l.slots_dev);
        cudaFree(l.done_dev);
        cudaFree(l.scratch);
        cudaFree(l.smax2);
        cudaFree(l.sub);
    }
    cudaFree(b->queue);
    cudaFree(b->cur_dev);
    delete b;
    return ORCHA_OK;
}

orcha_status orcha_batch_create(orcha_packet* const* pk, int32_t npk, int32_t tx, int32_t ty, orcha_batch** out) {
    if (!pk || !out || npk < 1) return fail(ORCHA_ERR_INVALID, "batch_create: need at least one packet");
    *out = nullptr;
    std::vector<orcha_mesh*> meshes;
    for (int i = 0; i < npk; ++i) {
        if (!pk[i]) return fail(ORCHA_ERR_INVALID, "batch_create: null packet %d", i);
        if (std::find(meshes.begin(), meshes.end(), pk[i]->mesh) == meshes.end()) meshes.push_back(pk[i]->mesh);
    }
    const int ndim = meshes[0]->dev.ndim;
    if (tx == 0 && ty == 0) {           // default: the widest variant every mesh's blocks allow
        tx = 16;
        ty = 16;
        for (auto* m : meshes) {
            if (m->dev.bs[0] < 16) tx = 8;
            if (m->dev.bs[1] < 16) ty = 8;
        }
    }
    if (!orcha::hydro_tile_supported(ndim, tx, ty))
        return fail(ORCHA_ERR_UNSUPPORTED, "batch_create: no %dx%d tile variant", tx, ty);
    for (auto* m : meshes) {
        if (!m->dev.smax || !m->dev.err) return fail(ORCHA_ERR_INVALID, "batch_create: mesh scratch not set up");
        if (m->dev.ndim != ndim) return fail(ORCHA_ERR_INVALID, "batch_create: meshes of different ndim");
        if (m->dev.bs[0] % tx || m->dev.bs[1] % ty)
            return fail(ORCHA_ERR_INVALID, "batch_create: tile %dx%d does not divide a mesh's blocks", tx, ty);
    }
    // each mesh's packets must cover its blocks exactly once (the step ends with that mesh's dt)
    for (size_t s_ = 0; s_ < meshes.size(); ++s_) {
        orcha_mesh* m = meshes[s_];
        std::vector<char> seen((size_t)m->nblk, 0);
        long long cnt = 0;
        for (int i = 0; i < npk; ++i) {
            if (pk[i]->mesh != m) continue;
            for (int id : pk[i]->ids) {
                if (seen[id]) return fail(ORCHA_ERR_INVALID, "batch_create: block %d of a mesh in two packets", id);
                seen[id] = 1;
                ++cnt;
            }
        }
        if (cnt != m->nblk)
            return fail(ORCHA_ERR_INVALID, "batch_create: packets cover %lld of a mesh's %d blocks", cnt, m->nblk);
    }
    orcha_batch* b = new orcha_batch();
    b->meshes = meshes;
    b->packets.assign(pk, pk + npk);
    b->ndim = ndim;
    b->tx = tx;
    b->ty = ty;
    for (int i = 0; i < npk; ++i) {
        const int slot = (int)(std::find(meshes.begin(), meshes.end(), pk[i]->mesh) - meshes.begin());
        const orcha_mesh* m = pk[i]->mesh;
        const int ntile = (m->dev.bs[0] / tx) * (m->dev.bs[1] / ty);
        for (int id : pk[i]->ids)
            for (int t = 0; t < ntile; ++t) b->base_items.push_back({slot, id, t, 0});
    }
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaMalloc(&b->queue, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMalloc(&b->cur_dev, sizeof(int) * meshes.size());
    if (e == cudaSuccess) e = orcha::configure_hydro(ndim, tx, ty);
    if (e != cudaSuccess) {
        orcha_status st = cuda_fail(e, "batch_create");
        orcha_batch_destroy(b);
        return st;
    }
    *out = b;
    return ORCHA_OK;
}

// Work list of a 3D batch: z ranges of block columns (worklist.h); 2D batches
// keep one item per block and tile.
static std::vector<orcha::Item> column_items(const orcha_batch* b, long long G) {
    std::vector<orcha::ColumnSource> src;
    for (size_t s = 0; s < b->meshes.size(); ++s) {
        const orcha::MeshDev& d = b->meshes[s]->dev;
        src.push_back({(int)s, {d.nb[0], d.nb[1], d.nb[2]}, {d.bs[0], d.bs[1], d.bs[2]},
                       (d.bs[0] / b->tx) * (d.bs[1] / b->ty)});
    }
    return orcha::column_items(src, G);
}

static orcha_status ensure_list(orcha_batch* b, int prec) {
    if (prec < 0 || prec >= orcha::kNumPrec) return fail(ORCHA_ERR_INVALID, "batch: not a hydro task variant");
    orcha_batch::List& L = b->lists[prec];
    if (L.built) return ORCHA_OK;
    const bool fused = orcha::prec_is_fused(prec);
    int per_sm = 0;
    ORCHA_CUDA(fused ? orcha::fused_occupancy(b->ndim, b->tx, b->ty, prec, &per_sm)
                     : orcha::persistent_occupancy(b->ndim, b->tx, b->ty, prec, &per_sm),
               "batch occupancy");
    if (per_sm < 1) return fail(ORCHA_ERR_UNSUPPORTED, "batch: persistent kernel does not fit on an SM");
    const long long G = (long long)per_sm * b->num_sms;
    // z ranges of block columns (3D; a column's planes must fit the 15-bit
    // fields of Item::zr), else one item per block and tile; the fused
    // variants take whole blocks (their scratch holds one block's planes)
    bool columns = b->ndim == 3 && !fused;
    for (auto* m : b->meshes) columns = columns && orcha::column_items_fit(m->dev);
    std::vector<orcha::Item> items = columns ? column_items(b, G) : b->base_items;
    const size_t ns = b->meshes.size();
    std::vector<int> per_mesh(ns, 0);
    for (auto& it : items) ++per_mesh[it.slot];
    std::vector<orcha::SlotDev> sl(ns);
    cudaError_t e = cudaMalloc(&L.done_dev, sizeof(unsigned) * ns);
    if (e == cudaSuccess) e = cudaMemset(L.done_dev, 0, sizeof(unsigned) * ns);
    for (size_t i = 0; i < ns; ++i) {
        orcha_mesh* m = b->meshes[i];
        sl[i].m = m->dev;
        sl[i].state[0] = m->desc.state_dev[0];
        sl[i].state[1] = m->desc.state_dev[1];
        sl[i].dt = m->desc.dt_dev;
        sl[i].cur = b->cur_dev + i;
        sl[i].done = L.done_dev + i;
        sl[i].nitems = per_mesh[i];
        sl[i].nblk = m->nblk;
        sl[i].tiles_x = m->dev.bs[0] / b->tx;
        sl[i].tiles_y = m->dev.bs[1] / b->ty;
    }
    const long long grid = std::min<long long>((long long)items.size(), G);
    if (fused && e == cudaSuccess) {
        int bz = 1;
        for (auto* m : b->meshes) bz = std::max(bz, b->ndim == 3 ? m->dev.bs[2] : 1);
        L.per_cta = orcha::fused_scratch_doubles(b->ndim, b->tx, b->ty, bz);
        e = cudaMalloc(&L.scratch, sizeof(double) * (size_t)(L.per_cta * grid));
        long long nb_all = 0;
        for (auto* m : b->meshes) nb_all += m->nblk;
        if (e == cudaSuccess && orcha::prec_is_tb2(prec)) {
            e = cudaMalloc(&L.smax2, sizeof(unsigned long long) * (size_t)nb_all);
            if (e == cudaSuccess) e = cudaMemset(L.smax2, 0, sizeof(unsigned long long) * (size_t)nb_all);
            long long off = 0;
            for (size_t i = 0; i < ns; ++i) {
                sl[i].smax2 = L.smax2 + off;
                off += b->meshes[i]->nblk;
            }
        }
    }
    if (!fused && e == cudaSuccess) {
        // one-step variants: the signal-speed filter's per-block bounds (hydro.cuh, SpeedBound)
        long long nb_all = 0;
        for (auto* m : b->meshes) nb_all += m->nblk;
        // + one word per mesh: the first dt's scratch (orcha::launch_first_dt)
        e = cudaMalloc(&L.sub, sizeof(unsigned long long) * (size_t)(nb_all + (long long)ns));
        if (e == cudaSuccess) e = cudaMemset(L.sub, 0, sizeof(unsigned long long) * (size_t)(nb_all + (long long)ns));
        long long off = 0;
        for (size_t i = 0; i < ns; ++i) {
            sl[i].m.sub = L.sub + off;
            off += b->meshes[i]->nblk;
        }
    }
    if (e == cudaSuccess) e = cudaMalloc(&L.slots_dev, sizeof(orcha::SlotDev) * ns);
    if (e == cudaSuccess) e = cudaMalloc(&L.items_dev, sizeof(orcha::Item) * items.size());
    if (e == cudaSuccess) e = cudaMemcpy(L.slots_dev, sl.data(), sizeof(orcha::SlotDev) * ns, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(L.items_dev, items.data(), sizeof(orcha::Item) * items.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "batch work list");
    L.nitems = (int)items.size();
    L.grid = (int)grid;
    L.built = true;
    return ORCHA_OK;
}

// Persistent launches that nsteps time steps of `task` take.
static int batch_launches(orcha_task task, int nsteps) {
    const int prec = orcha::prec_of(task);
    if (orcha::prec_is_tb2(prec)) return nsteps / 2;       // two steps per launch
    if (orcha::prec_is_fused(prec)) return nsteps;         // a whole Heun step per launch
    return nsteps * (orcha::is_rk_step_task(task) ? 2 : 1);
}

static orcha_status enqueue_batch_steps(orcha_batch* b, orcha_task task, int nsteps, cudaStream_t st) {
    const int prec = orcha::prec_of(task);
    const orcha_batch::List& L = b->lists[prec];
    if (orcha::prec_is_fused(prec)) {
        for (int n = 0; n < batch_launches(task, nsteps); ++n) {
            ORCHA_CUDA(cudaMemsetAsync(b->queue, 0, sizeof(unsigned), st), "batch queue reset");
            ORCHA_CUDA(orcha::launch_fused(b->ndim, b->tx, b->ty, prec, L.slots_dev, L.items_dev, L.nitems, b->queue,
                                           L.scratch, L.per_cta, L.grid, st),
                       "batch fused launch");
        }
        return ORCHA_OK;
    }
    const int stages = orcha::is_rk_step_task(task) ? 2 : 1;     // a Heun step is two launches
    for (int n = 0; n < nsteps; ++n) {
        for (int k = 1; k <= stages; ++k) {
            ORCHA_CUDA(cudaMemsetAsync(b->queue, 0, sizeof(unsigned), st), "batch queue reset");
            ORCHA_CUDA(orcha::launch_persistent(b->ndim, b->tx, b->ty, prec, L.slots_dev, L.items_dev, L.nitems,
                                                b->queue, L.grid, stages == 2 ? k : 0, st),
                       "batch launch");
        }
    }
    return ORCHA_OK;
}

orcha_status orcha_batch_advance(orcha_batch* b, orcha_task task, int32_t nsteps, int32_t init_dt, int32_t use_graph,
                                 void* stream) {
    if (!b || nsteps < 0) return fail(ORCHA_ERR_INVALID, "batch_advance: bad argument");
    if (!orcha::is_step_task(task))
        return fail(ORCHA_ERR_INVALID, "batch_advance: task must be a whole-step hydro task");
    if (orcha::prec_is_tb2(orcha::prec_of(task)) && nsteps % 2)
        return fail(ORCHA_ERR_INVALID, "batch_advance: a two-step task needs an even nsteps");
    cudaStream_t st = (cudaStream_t)stream;
    orcha_status s;
    if ((s = ensure_list(b, orcha::prec_of(task)))) return s;
    if (init_dt) {
        // one launch per mesh over all its blocks (the batch covers every block);
        // an FP64 rule with the list's filter bounds takes the filtered first dt
        const orcha_batch::List& L = b->lists[orcha::prec_of(task)];
        long long nb_all = 0;
        for (auto* m : b->meshes) nb_all += m->nblk;
        long long off = 0;
        for (size_t i = 0; i < b->meshes.size(); ++i) {
            orcha_mesh* m = b->meshes[i];
            if (L.sub && !orcha::prec_f32_dt(orcha::prec_of(task))) {
                orcha::MeshDev md = m->dev;
                md.sub = L.sub + off;
                ORCHA_CUDA(orcha::launch_first_dt(md, m->nblk, m->desc.state_dev[m->cur], m->desc.dt_dev,
                                                  L.sub + nb_all + (long long)i, st),
                           "batch first dt");
            } else {
                ORCHA_CUDA(orcha::launch_signal_speed_all(m->dev, m->nblk, m->desc.state_dev[m->cur], st,
                                                          orcha::prec_f32_dt(orcha::prec_of(task))),
                           "batch signal speed");
                if ((s = orcha_dt_reduce(m, stream))) return s;
            }
            off += m->nblk;
        }
    }
    // the device copy of each mesh's current buffer index, as of this point in the stream
    std::vector<int> cur(b->meshes.size());
    for (size_t i = 0; i < cur.size(); ++i) cur[i] = b->meshes[i]->cur;
    ORCHA_CUDA(cudaMemcpyAsync(b->cur_dev, cur.data(), sizeof(int) * cur.size(), cudaMemcpyHostToDevice, st),
               "batch cur upload");
    if (nsteps == 0) return ORCHA_OK;
    if (!use_graph) {
        if ((s = enqueue_batch_steps(b, task, nsteps, st))) return s;
    } else {
        if (st == nullptr) return fail(ORCHA_ERR_INVALID, "batch_advance: graph capture needs a non-default stream");
        cudaGraphExec_t exec = nullptr;
        for (auto& g : b->graphs)
            if (g.task == task && g.nsteps == nsteps) exec = g.exec;
        if (!exec) {
            ORCHA_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal), "begin capture");
            s = enqueue_batch_steps(b, task, nsteps, st);
            cudaGraph_t graph = nullptr;
            cudaError_t e = cudaStreamEndCapture(st, &graph);
            if (s) { if (graph) cudaGraphDestroy(graph); return s; }
            if (e != cudaSuccess) return cuda_fail(e, "end capture");
            e = cudaGraphInstantiate(&exec, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) return cuda_fail(e, "graph instantiate");
            b->graphs.push_back({task, nsteps, exec});
        }
        ORCHA_CUDA(cudaGraphLaunch(exec, st), "batch graph launch");
    }
    const int flips = batch_launches(task, nsteps);     // one per launch
    for (auto* m : b->meshes) m->cur ^= (flips & 1);
    return ORCHA_OK;
}

orcha_status orcha_mesh_poll(orcha_mesh* m, void* stream, int32_t* device_error) {
    if (!m || !device_error) return fail(ORCHA_ERR_INVALID, "mesh_poll: null argument");
    cudaStream_t st = (cudaStream_t)stream;
    ORCHA_CUDA(cudaStreamSynchronize(st), "mesh_poll sync");
    int h = 0;
    ORCHA_CUDA(cudaMemcpy(&h, m->err, sizeof(int), cudaMemcpyDeviceToHost), "mesh_poll read");
    ORCHA_CUDA(cudaMemset(m->err, 0, sizeof(int)), "mesh_poll clear");
    *device_error = h;
    if (h)
        return fail(ORCHA_ERR_NONFINITE,
                    "device error word %d (1 non-physical state, 2 non-finite dt, 8 two-step launch beyond its "
                    "stability limit)", h);
    return ORCHA_OK;
}

orcha_status orcha_selftest_conversions(uint64_t first_pattern, uint64_t count, uint64_t seed, uint64_t* mismatches) {
    if (!mismatches) return fail(ORCHA_ERR_INVALID, "selftest: null argument");
    unsigned long long* bad = nullptr;
    ORCHA_CUDA(cudaMalloc(&bad, sizeof(unsigned long long)), "selftest alloc");
    cudaError_t e = cudaMemset(bad, 0, sizeof(unsigned long long));
    if (e == cudaSuccess) e = orcha::launch_selftest(first_pattern, count, seed, bad, nullptr);
    unsigned long long h = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&h, bad, sizeof(h), cudaMemcpyDeviceToHost);
    cudaFree(bad);
    if (e != cudaSuccess) return cuda_fail(e, "selftest");
    *mismatches = h;
    return ORCHA_OK;
}

orcha_status orcha_selftest_fp64_emulation(uint64_t count, uint64_t seed, uint64_t* mismatches) {
    if (!mismatches) return fail(ORCHA_ERR_INVALID, "selftest: null argument");
    unsigned long long* bad = nullptr;
    ORCHA_CUDA(cudaMalloc(&bad, sizeof(unsigned long long)), "selftest alloc");
    cudaError_t e = cudaMemset(bad, 0, sizeof(unsigned long long));
    if (e == cudaSuccess) e = orcha::launch_selftest_fp64(count, seed, bad, nullptr);
    unsigned long long h = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&h, bad, sizeof(h), cudaMemcpyDeviceToHost);
    cudaFree(bad);
    if (e != cudaSuccess) return cuda_fail(e, "selftest");
    *mismatches = h;
    return ORCHA_OK;
}

orcha_status orcha_selftest_dword(uint64_t count, uint64_t seed, double max_err[6]) {
    if (!max_err) return fail(ORCHA_ERR_INVALID, "selftest: null argument");
    unsigned long long* err = nullptr;
    ORCHA_CUDA(cudaMalloc(&err, 6 * sizeof(unsigned long long)), "selftest alloc");
    cudaError_t e = cudaMemset(err, 0, 6 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = orcha::launch_selftest_dword(count, seed, err, nullptr);
    unsigned long long h[6] = {};
    if (e == cudaSuccess) e = cudaMemcpy(h, err, sizeof(h), cudaMemcpyDeviceToHost);
    cudaFree(err);
    if (e != cudaSuccess) return cuda_fail(e, "selftest");
    for (int k = 0; k < 6; ++k) std::memcpy(&max_err[k], &h[k], sizeof(double));
    return ORCHA_OK;
}

orcha_status orcha_selftest_speed_bound(uint64_t count, uint64_t seed, uint64_t counts[3], double* max_ratio) {
    if (!counts || !max_ratio) return fail(ORCHA_ERR_INVALID, "selftest: null argument");
    unsigned long long* res = nullptr;
    ORCHA_CUDA(cudaMalloc(&res, 5 * sizeof(unsigned long long)), "selftest alloc");
    cudaError_t e = cudaMemset(res, 0, 5 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = orcha::launch_selftest_speed_bound(count, seed, res, nullptr);
    unsigned long long h[4] = {};
    if (e == cudaSuccess) e = cudaMemcpy(h, res, sizeof(h), cudaMemcpyDeviceToHost);
    cudaFree(res);
    if (e != cudaSuccess) return cuda_fail(e, "selftest");
    for (int k = 0; k < 3; ++k) counts[k] = h[k];
    std::memcpy(max_ratio, &h[3], sizeof(double));
    return ORCHA_OK;
}

const char* orcha_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
