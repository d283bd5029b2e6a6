// server.cu -- continuous-batching serving loop with resident block state.
//
// A request is an independent simulation (its own block grid, initial
// state, step count and time step). The paper's runtime moves data packets
// between host and device on GPU streams so that transfers hide behind
// computation, and keeps enough packets in flight to occupy the GPU
// (sections "Milhoja" and "Sedov Blast Wave Results"). Here one worker
// thread owns the device and runs, per iteration:
//   admit    pending requests in arrival order while their state fits the
//            HBM budget (one device pool allocated up front): H2D copy of
//            the initial interiors, pack into the padded layout, first dt --
//            all on a copy stream, overlapping the compute stream;
//   step     ONE persistent launch that advances every active request by
//            one time step (each with its own dt, formed on the device);
//            requests join as soon as their admission completes and leave
//            after their last step; the work list's buffers are sized at
//            creation (the loop allocates no device memory);
//   complete finished requests on the copy stream: unpack, D2H, error word;
//            their pool memory is released when the copy has landed.
// At most two steps are in flight, so new requests join within two steps.
// A request's arithmetic does not depend on what else is in the launch, so
// its result is bitwise the one it gets alone.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/orcha.h"
#include "launch.h"
#include "runtime.h"

namespace {

using Clock = std::chrono::steady_clock;
constexpr size_t kAlign = 256;
constexpr int kInflight = 2;      // persistent steps queued ahead of the device

size_t round_up(size_t n) { return (n + kAlign - 1) / kAlign * kAlign; }

// First-fit allocator with coalescing over one device allocation.
struct Pool {
    char* base = nullptr;
    size_t size = 0, used = 0, peak = 0;
    std::map<size_t, size_t> free_;   // offset -> bytes

    cudaError_t init(size_t bytes) {
        size = round_up(bytes);
        cudaError_t e = cudaMalloc(&base, size);
        if (e == cudaSuccess) free_[0] = size;
        return e;
    }
    long long alloc(size_t bytes) {
        bytes = round_up(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            const size_t off = it->first, rem = it->second - bytes;
            free_.erase(it);
            if (rem) free_[off + bytes] = rem;
            used += bytes;
            peak = std::max(peak, used);
            return (long long)off;
        }
        return -1;
    }
    void release(size_t off, size_t bytes) {
        bytes = round_up(bytes);
        used -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

enum class RS { Pending, Admitting, Active, Finishing, Done };

struct Req {
    int64_t ticket = 0;
    orcha_request_desc d{};
    orcha::MeshDev m{};
    long long nblk = 0, ncell = 0;
    size_t interior_bytes = 0, state_elems = 0, bytes = 0, off = 0;
    double* state[2] = {nullptr, nullptr};
    double* dt = nullptr;
    unsigned long long* smax = nullptr;
    unsigned long long* sub = nullptr;   // the signal-speed filter's per-block bounds (hydro.cuh, SpeedBound)
    int* cur = nullptr;
    unsigned* done = nullptr;
    int* err = nullptr;
    double* totals = nullptr;
    double* partial = nullptr;       // nblk x 5 doubles: per-block sums of the totals reduction
    int cur_host = 0, steps_left = 0, nitems = 0, err_slot = -1;
    int kind = 0, tx = 8, ty = 8;    // tile kind and column tile of the hydro launch this request joins
    int prec = orcha::kF64;          // arithmetic variant of the hydro task (orcha::Prec)
    cudaEvent_t ev = nullptr;        // admission done / completion landed
    RS st = RS::Pending;
    orcha_request_stats stats{};
};

// One launch per (ndim 2 or 3) x (FP64, FP32 flux, FF or FP32-flux shortcut) x tile kind (0: 8x8,
// 1: 16x8, 2: 16x16): blocks 8 cells across x use the 8x8 tile; wider ones
// the autotuner's choice for 16^3 blocks on a B300, 16x16 for FP64 and FF in
// 3D when the blocks are 16 or more cells across y too, else 16x8.
constexpr int kServePrec = 4;        // kF64, kF32, kFF, kF32X (Runge-Kutta steps are not served)
constexpr int kTileKinds = 3;
constexpr int kGroups = 2 * kServePrec * kTileKinds;
constexpr int serve_index(int prec) { return prec == orcha::kF32X ? 3 : prec; }
constexpr int served_prec(int i) { return i == 3 ? (int)orcha::kF32X : i; }
constexpr int group_ndim(int g) { return 2 + (g & 1); }
constexpr int group_prec(int g) { return served_prec((g >> 1) % kServePrec); }
constexpr int group_kind(int g) { return (g >> 1) / kServePrec; }
constexpr int group_tx(int g) { return group_kind(g) >= 1 ? 16 : 8; }
constexpr int group_ty(int g) { return group_kind(g) == 2 ? 16 : 8; }
constexpr int group_of(int ndim, int prec, int kind) { return (ndim - 2) | ((serve_index(prec) + kind * kServePrec) << 1); }
constexpr bool serve_f32(int prec) { return prec == orcha::kF32 || prec == orcha::kF32X; }
constexpr int tile_kind(int ndim, int prec, const int* bs) {
    return bs[0] < 16 ? 0 : (ndim == 3 && !serve_f32(prec) && bs[1] >= 16 ? 2 : 1);
}
static_assert(group_of(group_ndim(17), group_prec(17), group_kind(17)) == 17, "group index round trip");
static_assert(group_of(group_ndim(23), group_prec(23), group_kind(23)) == 23, "group index round trip");

// Work-list buffers of one in-flight step, sized once at server creation so
// the step loop never allocates: slots for at most max_active requests and
// items for at most cap_items (an item needs at least 4 KiB of its request's
// pool memory -- two state buffers over a tile of >= 64 cells x >= 4
// variables x 8 bytes -- so pool bytes / 4096 items always suffice). The
// device arrays are carved from the budgeted pool; each launch group takes
// the next sub-range. Items are written on the device from the slots.
struct StepSlot {
    orcha::SlotDev* slots_pin = nullptr;     // host staging of the slots (pinned)
    orcha::SlotDev* slots_d = nullptr;       // in the pool
    orcha::Item* items_d = nullptr;          // in the pool
    unsigned* queue_d = nullptr;             // in the pool: one work counter per group
    cudaEvent_t ev = nullptr;
    bool busy = false;
};

}  // namespace

struct orcha_server {
    size_t budget = 0;
    int max_active = 0, device = 0, num_sms = 0;
    Pool pool;
    cudaStream_t compute = nullptr, copy = nullptr;
    Clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv_done;
    std::deque<Req*> submitted;                  // guarded by mu
    std::unordered_map<int64_t, Req*> tickets;   // guarded by mu
    int64_t next_ticket = 1;                     // guarded by mu
    orcha_server_stats totals{};                 // guarded by mu
    std::string fail_msg;                        // guarded by mu
    orcha_status fail_status = ORCHA_OK;         // guarded by mu
    // worker-owned
    std::vector<Req*> pending, admitting, active, finishing;
    StepSlot ring[kInflight];
    int ring_i = 0;
    size_t cap_items = 0;                        // items one step can hold (see StepSlot)
    long long items_held = 0;                    // items of the requests holding pool memory
    struct Result { double totals[5]; double dt; int err; int pad; };
    Result* res_pin = nullptr;                   // pinned results, one slot per live request
    std::vector<int> err_free;
    std::thread worker;
    std::atomic<bool> stop{false};

    double now_us() const { return std::chrono::duration<double, std::micro>(Clock::now() - t0).count(); }
    void run();
    bool fail(orcha_status s, const std::string& msg);
    bool admit(Req* r);
    bool launch_step(bool* launched);
    int occ[kGroups] = {};                       // resident CTAs per SM of each group's variant
    bool complete(Req* r);
};

bool orcha_server::fail(orcha_status s, const std::string& msg) {
    std::lock_guard<std::mutex> lock(mu);
    if (fail_status == ORCHA_OK) {
        fail_status = s;
        fail_msg = msg;
    }
    cv_done.notify_all();
    return false;
}

#define SRV_CUDA(call, what)                                                                      \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess) return fail(ORCHA_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// Reserve pool memory for a request and enqueue its admission on the copy stream.
bool orcha_server::admit(Req* r) {
    if ((size_t)(items_held + r->nitems) > cap_items) return false;   // bounded by construction; kept as a guard
    const long long off = pool.alloc(r->bytes);
    if (off < 0) return false;   // does not fit now; retried when memory frees up
    items_held += r->nitems;
    r->off = (size_t)off;
    char* p = pool.base + r->off;
    const size_t sb = round_up(r->state_elems * sizeof(double));
    r->state[0] = (double*)p;
    r->state[1] = (double*)(p + sb);
    char* tail = p + 2 * sb;
    r->smax = (unsigned long long*)tail;
    r->sub = (unsigned long long*)(tail + round_up(r->nblk * sizeof(unsigned long long)));
    r->dt = (double*)(tail + 2 * round_up(r->nblk * sizeof(unsigned long long)));
    r->cur = (int*)((char*)r->dt + kAlign);
    r->done = (unsigned*)((char*)r->cur + kAlign);
    r->err = (int*)((char*)r->done + kAlign);
    r->totals = (double*)((char*)r->err + kAlign);
    r->partial = (double*)((char*)r->totals + kAlign);
    const size_t tail_bytes = (size_t)((char*)r->totals + kAlign - tail);
    r->m.dt = r->dt;
    r->m.smax = r->smax;
    r->m.sub = r->sub;
    r->m.err = r->err;
    r->err_slot = err_free.back();
    err_free.pop_back();
    r->stats.t_admit_us = now_us();
    if (r->d.init_kind == ORCHA_INIT_FROM_HOST) {
        // initial interiors land in state[1] (used as staging), are packed into state[0]
        SRV_CUDA(cudaMemcpyAsync(r->state[1], r->d.init_host, r->interior_bytes, cudaMemcpyHostToDevice, copy),
                 "admit H2D");
        SRV_CUDA(orcha::launch_pack(r->m, r->state[1], r->state[0], copy), "admit pack");
    } else {
        orcha::RegionStates rs;
        for (int v = 0; v < 5; ++v) {
            rs.in[v] = r->d.u_in[v];
            rs.out[v] = r->d.u_out[v];
        }
        const int4 reg = make_int4(r->d.region[0], r->d.region[1], r->d.region[2], r->d.region[3]);
        SRV_CUDA(orcha::launch_region_init(r->m, r->state[0], r->d.init_kind, reg, rs, copy), "admit recipe");
    }
    SRV_CUDA(cudaMemsetAsync(tail, 0, tail_bytes, copy), "admit clear");
    if (orcha::prec_f32_dt(r->prec)) {
        SRV_CUDA(orcha::launch_signal_speed_all(r->m, (int)r->nblk, r->state[0], copy, true), "admit signal speed");
        SRV_CUDA(orcha::launch_dt_reduce(r->m, (int)r->nblk, r->dt, copy), "admit dt");
    } else {
        // FP64 speeds only where a cell can hold the maximum; the first word of
        // the request's totals (written again when it completes) is the scratch
        SRV_CUDA(orcha::launch_first_dt(r->m, (int)r->nblk, r->state[0], r->dt,
                                        reinterpret_cast<unsigned long long*>(r->totals), copy),
                 "admit dt");
    }
    SRV_CUDA(cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming), "admit event");
    SRV_CUDA(cudaEventRecord(r->ev, copy), "admit record");
    r->st = RS::Admitting;
    return true;
}

// One persistent launch per (ndim, precision) group advancing every active
// request one step. Sets *launched; returns false on failure.
bool orcha_server::launch_step(bool* launched) {
    *launched = false;
    StepSlot& s = ring[ring_i];
    if (s.busy) {
        const cudaError_t q = cudaEventQuery(s.ev);
        if (q == cudaErrorNotReady) return true;        // both slots in flight: try again later
        SRV_CUDA(q, "step slot");
        s.busy = false;
    }
    // the slots of every group, group after group, into this step's staging
    struct Span { int gi, slot0, nslots, item0, nitems; };
    std::vector<Span> spans;
    std::vector<Req*> finished;
    int nslot = 0, nitem = 0;
    for (int gi = 0; gi < kGroups; ++gi) {
        const int gtx = group_tx(gi), gty = group_ty(gi);
        Span sp{gi, nslot, 0, nitem, 0};
        for (Req* r : active) {
            if (group_of(r->m.ndim, r->prec, r->kind) != gi) continue;
            orcha::SlotDev sd{};
            sd.m = r->m;
            sd.state[0] = r->state[0];
            sd.state[1] = r->state[1];
            sd.dt = r->dt;
            sd.cur = r->cur;
            sd.done = r->done;
            sd.nitems = r->nitems;
            sd.nblk = (int)r->nblk;
            sd.tiles_x = r->m.bs[0] / gtx;
            sd.tiles_y = r->m.bs[1] / gty;
            sd.item0 = sp.nitems;                      // relative to the group's first item
            s.slots_pin[nslot++] = sd;
            sp.nslots += 1;
            sp.nitems += r->nitems;
            r->cur_host ^= 1;
            if (--r->steps_left == 0) finished.push_back(r);
        }
        if (sp.nslots == 0) continue;
        nitem += sp.nitems;
        spans.push_back(sp);
    }
    if ((size_t)nitem > cap_items || nslot > max_active)
        return fail(ORCHA_ERR_CUDA, "step: work list above its preallocated capacity");
    SRV_CUDA(cudaMemcpyAsync(s.slots_d, s.slots_pin, (size_t)nslot * sizeof(orcha::SlotDev), cudaMemcpyHostToDevice,
                             compute), "step upload");
    SRV_CUDA(cudaMemsetAsync(s.queue_d, 0, sizeof(unsigned) * kGroups, compute), "step queues");
    for (const Span& sp : spans) {
        const int gi = sp.gi;
        SRV_CUDA(orcha::launch_expand_items(s.slots_d + sp.slot0, sp.nslots, s.items_d + sp.item0, compute),
                 "step items");
        const int grid = std::max(1, std::min(sp.nitems, occ[gi] * num_sms));
        SRV_CUDA(orcha::launch_persistent(group_ndim(gi), group_tx(gi), group_ty(gi), group_prec(gi),
                                          s.slots_d + sp.slot0, s.items_d + sp.item0, sp.nitems, s.queue_d + gi,
                                          grid, 0, compute), "step launch");
        std::lock_guard<std::mutex> lock(mu);
        totals.steps_launched += 1;
    }
    SRV_CUDA(cudaEventRecord(s.ev, compute), "step record");
    s.busy = true;
    *launched = true;
    ring_i = (ring_i + 1) % kInflight;
    for (Req* r : finished) {
        active.erase(std::find(active.begin(), active.end(), r));
        if (!complete(r)) return false;
        finishing.push_back(r);
    }
    return true;
}

// Enqueue the copy-out of a request after its last step.
bool orcha_server::complete(Req* r) {
    StepSlot& last = ring[(ring_i + kInflight - 1) % kInflight];
    SRV_CUDA(cudaStreamWaitEvent(copy, last.ev, 0), "complete wait");
    double* cur = r->state[r->cur_host];
    double* stage = r->state[r->cur_host ^ 1];
    Result* res = res_pin + r->err_slot;
    SRV_CUDA(orcha::launch_totals(r->m, (int)r->nblk, cur, r->partial, r->totals, copy), "complete totals");
    if (r->d.out_host) {
        SRV_CUDA(orcha::launch_unpack(r->m, cur, stage, copy), "complete unpack");
        SRV_CUDA(cudaMemcpyAsync(r->d.out_host, stage, r->interior_bytes, cudaMemcpyDeviceToHost, copy),
                 "complete D2H");
    }
    SRV_CUDA(cudaMemcpyAsync(res->totals, r->totals, sizeof(double) * 5, cudaMemcpyDeviceToHost, copy), "complete totals D2H");
    SRV_CUDA(cudaMemcpyAsync(&res->dt, r->dt, sizeof(double), cudaMemcpyDeviceToHost, copy), "complete dt D2H");
    SRV_CUDA(cudaMemcpyAsync(&res->err, r->err, sizeof(int), cudaMemcpyDeviceToHost, copy), "complete err");
    SRV_CUDA(cudaEventRecord(r->ev, copy), "complete record");
    r->st = RS::Finishing;
    return true;
}

void orcha_server::run() {
    cudaSetDevice(device);
    while (!stop.load()) {
        bool progress = false;
        {
            std::lock_guard<std::mutex> lock(mu);
            if (fail_status != ORCHA_OK) break;
            while (!submitted.empty()) {
                pending.push_back(submitted.front());
                submitted.pop_front();
            }
        }
        // admit in arrival order while memory and slots allow
        while (!pending.empty() && (int)(admitting.size() + active.size() + finishing.size()) < max_active &&
               !err_free.empty()) {
            Req* r = pending.front();
            if (!admit(r)) {
                if (fail_status != ORCHA_OK) return;
                break;
            }
            pending.erase(pending.begin());
            admitting.push_back(r);
            progress = true;
        }
        // admitted requests join the next step
        for (size_t i = 0; i < admitting.size();) {
            const cudaError_t q = cudaEventQuery(admitting[i]->ev);
            if (q == cudaErrorNotReady) { ++i; continue; }
            if (q != cudaSuccess) { fail(ORCHA_ERR_CUDA, std::string("admission: ") + cudaGetErrorString(q)); return; }
            admitting[i]->stats.t_ready_us = now_us();
            admitting[i]->st = RS::Active;
            active.push_back(admitting[i]);
            admitting.erase(admitting.begin() + i);
            progress = true;
        }
        if (!active.empty()) {
            bool launched = false;
            if (!launch_step(&launched)) return;
            progress = progress || launched;
        }
        // completions that landed
        for (size_t i = 0; i < finishing.size();) {
            Req* r = finishing[i];
            const cudaError_t q = cudaEventQuery(r->ev);
            if (q == cudaErrorNotReady) { ++i; continue; }
            if (q != cudaSuccess) { fail(ORCHA_ERR_CUDA, std::string("completion: ") + cudaGetErrorString(q)); return; }
            cudaEventDestroy(r->ev);
            r->ev = nullptr;
            pool.release(r->off, r->bytes);
            items_held -= r->nitems;
            const Result& res = res_pin[r->err_slot];
            r->stats.device_error = res.err;
            for (int v = 0; v < 5; ++v) r->stats.totals[v] = v < r->m.nvar ? res.totals[v] : 0.0;
            r->stats.dt_next = res.dt;
            err_free.push_back(r->err_slot);
            r->stats.status = r->stats.device_error ? ORCHA_ERR_NONFINITE : ORCHA_OK;
            r->stats.t_done_us = now_us();
            finishing.erase(finishing.begin() + i);
            {
                std::lock_guard<std::mutex> lock(mu);
                r->st = RS::Done;
                totals.completed += 1;
                totals.zone_updates += r->stats.zone_updates;
                totals.pool_peak_bytes = pool.peak;
            }
            cv_done.notify_all();
            progress = true;
        }
        if (!progress) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

extern "C" {

orcha_status orcha_server_create(size_t hbm_budget_bytes, int32_t max_active, orcha_server** out) {
    if (!out || hbm_budget_bytes < (1u << 20) || max_active < 1)
        return orcha::set_error(ORCHA_ERR_INVALID, "server_create: need out, a budget >= 1 MiB and max_active >= 1");
    *out = nullptr;
    orcha_server* s = new orcha_server();
    s->budget = hbm_budget_bytes;
    s->max_active = max_active;
    s->t0 = Clock::now();
    cudaError_t e = cudaGetDevice(&s->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, s->device);
    if (e == cudaSuccess) e = s->pool.init(hbm_budget_bytes);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->compute, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->copy, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMallocHost(&s->res_pin, sizeof(orcha_server::Result) * (size_t)max_active);
    // the step loop's work-list buffers, once: slots and items carved from the pool
    s->cap_items = s->pool.size / 4096;
    for (int i = 0; e == cudaSuccess && i < kInflight; ++i) {
        StepSlot& r = s->ring[i];
        e = cudaEventCreateWithFlags(&r.ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMallocHost(&r.slots_pin, sizeof(orcha::SlotDev) * (size_t)max_active);
        const long long a = s->pool.alloc(sizeof(orcha::SlotDev) * (size_t)max_active);
        const long long b = s->pool.alloc(sizeof(orcha::Item) * s->cap_items);
        const long long c = s->pool.alloc(sizeof(unsigned) * kGroups);
        if (e == cudaSuccess && (a < 0 || b < 0 || c < 0)) e = cudaErrorMemoryAllocation;
        if (e == cudaSuccess) {
            r.slots_d = (orcha::SlotDev*)(s->pool.base + a);
            r.items_d = (orcha::Item*)(s->pool.base + b);
            r.queue_d = (unsigned*)(s->pool.base + c);
        }
    }
    for (int nd = 2; e == cudaSuccess && nd <= 3; ++nd) {
        e = orcha::configure_hydro(nd, 8, 8);
        if (e == cudaSuccess) e = orcha::configure_hydro(nd, 16, 8);
        if (e == cudaSuccess) e = orcha::configure_hydro(nd, 16, 16);
    }
    for (int gi = 0; e == cudaSuccess && gi < kGroups; ++gi)
        e = orcha::persistent_occupancy(group_ndim(gi), group_tx(gi), group_ty(gi), group_prec(gi), &s->occ[gi]);
    if (e != cudaSuccess) {
        orcha_status st = orcha::cuda_error(e, "server_create");
        s->stop = true;
        orcha_server_destroy(s);
        return st;
    }
    for (int i = max_active - 1; i >= 0; --i) s->err_free.push_back(i);
    s->totals.pool_bytes = s->pool.size;
    s->worker = std::thread([s] { s->run(); });
    *out = s;
    return ORCHA_OK;
}

orcha_status orcha_server_destroy(orcha_server* s) {
    if (!s) return ORCHA_OK;
    s->stop = true;
    if (s->worker.joinable()) s->worker.join();
    if (s->compute) cudaStreamSynchronize(s->compute);
    if (s->copy) cudaStreamSynchronize(s->copy);
    std::vector<Req*> all;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        for (auto& kv : s->tickets) all.push_back(kv.second);
        s->tickets.clear();
    }
    for (Req* r : all) {
        if (r->ev) cudaEventDestroy(r->ev);
        delete r;
    }
    for (auto& sl : s->ring) {
        if (sl.ev) cudaEventDestroy(sl.ev);
        cudaFreeHost(sl.slots_pin);          // the device arrays live in the pool
    }
    cudaFreeHost(s->res_pin);
    if (s->compute) cudaStreamDestroy(s->compute);
    if (s->copy) cudaStreamDestroy(s->copy);
    cudaFree(s->pool.base);
    delete s;
    return ORCHA_OK;
}

orcha_status orcha_server_submit(orcha_server* s, const orcha_request_desc* rd, int64_t* ticket) {
    if (!s || !rd || !ticket) return orcha::set_error(ORCHA_ERR_INVALID, "server_submit: null argument");
    if (rd->nsteps < 1) return orcha::set_error(ORCHA_ERR_INVALID, "server_submit: nsteps < 1");
    if (rd->task != ORCHA_TASK_HYDRO_FP64 && rd->task != ORCHA_TASK_HYDRO_F32FLUX && rd->task != ORCHA_TASK_HYDRO_FF &&
        rd->task != ORCHA_TASK_HYDRO_F32FLUX_FFSUM)
        return orcha::set_error(ORCHA_ERR_INVALID,
                                "server_submit: task must be HYDRO_FP64, HYDRO_F32FLUX, HYDRO_F32FLUX_FFSUM or HYDRO_FF");
    if (rd->init_kind == ORCHA_INIT_FROM_HOST && !rd->init_host)
        return orcha::set_error(ORCHA_ERR_INVALID, "server_submit: FROM_HOST needs init_host");
    if (rd->init_kind == ORCHA_INIT_HALF_SPACE && (rd->region[0] < 0 || rd->region[0] >= rd->ndim))
        return orcha::set_error(ORCHA_ERR_INVALID, "server_submit: half-space axis outside [0, ndim)");
    if (rd->init_kind < ORCHA_INIT_FROM_HOST || rd->init_kind > ORCHA_INIT_HALF_SPACE)
        return orcha::set_error(ORCHA_ERR_INVALID, "server_submit: unknown init_kind");
    orcha_mesh_desc md{};
    md.ndim = rd->ndim;
    for (int a = 0; a < 3; ++a) {
        md.nb[a] = rd->nb[a];
        md.bs[a] = rd->bs[a];
        md.periodic[a] = rd->periodic[a];
        md.lo[a] = rd->lo[a];
        md.hi[a] = rd->hi[a];
    }
    md.gamma = rd->gamma;
    md.cfl = rd->cfl;
    Req* r = new Req();
    orcha_status st = orcha::mesh_dev_from_desc(&md, &r->m, &r->nblk);
    if (st) { delete r; return st; }
    r->d = *rd;
    r->prec = orcha::prec_of((orcha_task)rd->task);
    r->ncell = (long long)rd->bs[0] * rd->bs[1] * (rd->ndim == 3 ? rd->bs[2] : 1);
    r->interior_bytes = (size_t)r->nblk * r->m.nvar * r->ncell * sizeof(double);
    r->state_elems = orcha_state_elems(&md);
    r->bytes = 2 * round_up(r->state_elems * sizeof(double)) + 2 * round_up(r->nblk * sizeof(unsigned long long)) +
               5 * kAlign + round_up(r->nblk * 5 * sizeof(double));
    r->steps_left = rd->nsteps;
    r->kind = tile_kind(rd->ndim, r->prec, rd->bs);
    r->tx = group_tx(group_of(rd->ndim, r->prec, r->kind));
    r->ty = group_ty(group_of(rd->ndim, r->prec, r->kind));
    r->nitems = (int)r->nblk * (rd->bs[0] / r->tx) * (rd->bs[1] / r->ty);
    r->stats.zone_updates = (int64_t)r->nblk * r->ncell * rd->nsteps;
    if (r->bytes > s->pool.size || (size_t)r->nitems > s->cap_items) {
        delete r;
        return orcha::set_error(ORCHA_ERR_OOM, "server_submit: request larger than the whole HBM budget");
    }
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->fail_status != ORCHA_OK) {
        delete r;
        return orcha::set_error(s->fail_status, ("server failed: " + s->fail_msg).c_str());
    }
    r->ticket = s->next_ticket++;
    r->stats.t_submit_us = s->now_us();
    s->tickets[r->ticket] = r;
    s->submitted.push_back(r);
    s->totals.submitted += 1;
    *ticket = r->ticket;
    return ORCHA_OK;
}

orcha_status orcha_server_wait(orcha_server* s, int64_t ticket, int32_t timeout_ms, orcha_request_stats* stats) {
    if (!s) return orcha::set_error(ORCHA_ERR_INVALID, "server_wait: null server");
    std::unique_lock<std::mutex> lock(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return orcha::set_error(ORCHA_ERR_INVALID, "server_wait: unknown ticket");
    Req* r = it->second;
    const auto pred = [&] { return r->st == RS::Done || s->fail_status != ORCHA_OK; };
    if (timeout_ms < 0) s->cv_done.wait(lock, pred);
    else if (!s->cv_done.wait_for(lock, std::chrono::milliseconds(timeout_ms), pred))
        return orcha::set_error(ORCHA_ERR_TIMEOUT, "server_wait: request not finished within the timeout");
    if (r->st != RS::Done) return orcha::set_error(s->fail_status, ("server failed: " + s->fail_msg).c_str());
    if (stats) *stats = r->stats;
    s->tickets.erase(it);
    const orcha_status st = r->stats.status;
    delete r;
    if (st) return orcha::set_error(st, "request finished with a device error (see stats.device_error)");
    return ORCHA_OK;
}

orcha_status orcha_server_get_stats(orcha_server* s, orcha_server_stats* out) {
    if (!s || !out) return orcha::set_error(ORCHA_ERR_INVALID, "server_get_stats: null argument");
    std::lock_guard<std::mutex> lock(s->mu);
    *out = s->totals;
    out->now_us = s->now_us();
    return s->fail_status;
}

}  // extern "C"
