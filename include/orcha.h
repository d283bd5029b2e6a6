/*
 * orcha.h -- C ABI of the B300 block-hydro packet engine.
 *
 * Model (arXiv 2507.09337, "ORCHA"): a task function is a group of API
 * calls executed on one device with no data transfer in between (section
 * "Code Generators", definitions); the data item that feeds a device task is
 * a data packet, one flattened structure moved as a single unit (same
 * section); an AMR application concatenates n blocks into one packet because
 * a single block is too small to occupy a GPU, with n chosen at run time
 * (section "DataItem Generators"). Blocks all have the same cell count and a
 * uniform cell size (section "Flash-X"); a halo of guard cells around each
 * block is refreshed before the task runs, and tasks contain no
 * communication (sections "Experiments" and "Milhoja").
 *
 * Here a mesh is a uniform grid of equal blocks whose state lives in device
 * memory; a packet is a list of block ids; the task run on a packet is one
 * step of a compressible-Euler finite-volume update on ideal gamma-law gas
 * (MUSCL-Hancock reconstruction with minmod limiting, HLL fluxes, unsplit
 * conservative update) plus the per-block signal speeds that give the next
 * CFL time step.
 *
 * Conventions for every call:
 *  - Pointers named *_dev are device pointers, all others host pointers.
 *  - The caller owns the two state buffers and the dt scalar (any device
 *    allocator, e.g. PyTorch); the library owns only its descriptors, small
 *    per-block scratch arrays and staging buffers, freed by the matching
 *    destroy call.
 *  - Calls taking a stream are asynchronous and stream-ordered; none of them
 *    synchronises the device except orcha_mesh_poll and the destroy calls.
 *  - Host-detected errors are returned immediately as a negative
 *    orcha_status, with a message in orcha_last_error() (per thread).
 *    Errors found on the device (non-physical state, a non-finite time
 *    step, a two-step launch beyond its stability limit) are OR-ed into the
 *    mesh's device error word and reported by orcha_mesh_poll. No kernel
 *    waits on another CTA or launch, so none has a timeout.
 *  - Not thread-safe per mesh: calls on one mesh must come from one thread
 *    at a time. Different meshes are independent.
 */
#ifndef ORCHA_H
#define ORCHA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define ORCHA_API __attribute__((visibility("default")))
#else
#define ORCHA_API
#endif

typedef int32_t orcha_status;

#define ORCHA_OK 0
#define ORCHA_ERR_INVALID (-1)   /* bad argument: null pointer, size, id out of range or repeated */
#define ORCHA_ERR_OOM (-2)       /* a device allocation failed, or an HBM budget would be exceeded */
#define ORCHA_ERR_CUDA (-3)      /* a CUDA runtime call failed (text in orcha_last_error) */
#define ORCHA_ERR_TIMEOUT (-4)   /* a bounded wait ran out */
#define ORCHA_ERR_NONFINITE (-5) /* the device found rho <= 0, p <= 0 or a non-finite value */
#define ORCHA_ERR_UNSUPPORTED (-6) /* valid request outside the built configurations */

/* Bits of the device error word (orcha_mesh_poll). */
#define ORCHA_DEVERR_NONPHYSICAL 1 /* an interior cell had rho <= 0 or p <= 0 (or NaN) */
#define ORCHA_DEVERR_BAD_DT 2      /* the reduced signal speed was not positive and finite */
#define ORCHA_DEVERR_CFL 8         /* a two-step launch's dt exceeded the second step's stability limit */

/* Initial states (orcha_mesh_init_region, serving requests). FROM_HOST copies
 * host data in. The two
 * recipes write the initial state on the device (no host transfer): cell g
 * (global index per axis) is inside the region when, in half-cell units
 * (cell centre at 2g + 1), sum_d (2 g_d + 1 - region[d])^2 <= region[3]
 * (SPHERE), or when g[region[0]] < region[1] (HALF_SPACE); inside cells take
 * the conserved state u_in, the others u_out (Sedov-like and Sod-like
 * problems). */
#define ORCHA_INIT_FROM_HOST 0
#define ORCHA_INIT_SPHERE 1
#define ORCHA_INIT_HALF_SPACE 2

/* Tasks a packet can run (orcha_packet_run). */
typedef enum {
    /* Refresh the two guard layers of every packet block in the current
     * state buffer from the neighbouring blocks' interiors; on the domain
     * edge the boundary rule applies (outflow: zero-gradient copy of the
     * nearest interior cell, per axis; periodic: wrap). Pure FP64 copy. */
    ORCHA_TASK_GUARD_FILL = 0,
    /* One MUSCL-Hancock/HLL step of every packet block in FP64: reads the
     * current buffer (guards filled) and the device dt, writes the interiors
     * of the other buffer and the blocks' largest signal speed
     * sum_d (|u_d| + c) / dx_d of the new state. The default library fuses a
     * product into the sum or difference the scheme writes it in (one FMA)
     * and rounds every other operation as written, so every tile shape and
     * both the packet and the persistent path give the same bits; the
     * library built with ORCHA_FP64_CONTRACT=0 (liborcha_exact.so) fuses
     * nothing and reproduces an unfused FP64 evaluation bit for bit. */
    ORCHA_TASK_HYDRO_FP64 = 1,
    /* As HYDRO_FP64 with primitives, reconstruction, predictor and HLL fluxes
     * in FP32 (from the FP64 state rounded to nearest). Each face flux is
     * promoted to FP64 before the difference; the differences, their dt/dx_d
     * scaling, the x+y+z sum and the conservative update are FP64, as are the
     * guard fill, the new state's per-cell signal speed and the dt
     * reduction. */
    ORCHA_TASK_HYDRO_F32FLUX = 2,
    /* Only the blocks' largest signal speed of the current buffer (to form
     * the first time step). */
    ORCHA_TASK_SIGNAL_SPEED = 3,
    /* As HYDRO_FP64 with primitives, reconstruction, predictor and HLL fluxes
     * in double-word ("float-float") arithmetic: each value a pair of FP32
     * numbers, about 48 significant bits, on the FP32 pipe. The flux
     * differences are double-word, the conservative update, the guard fill
     * and the dt reduction FP64. Not in the paper: a variant of its task
     * for a GPU whose FP64 rate is a small fraction of its FP32 rate. */
    ORCHA_TASK_HYDRO_FF = 4,
    /* The first stage of Heun's two-stage Runge-Kutta step (the paper's
     * Spark solver is explicit finite volume with 2nd-order Runge-Kutta,
     * section "Experiments") with the plain MUSCL operator L (minmod slopes
     * of the primitives, face states W -+ dW/2, no half step, HLL), FP64:
     * other buffer = current + dt L(current). Raises no signal speed. */
    ORCHA_TASK_RK2_STAGE1 = 5,
    /* The second stage: other buffer = 0.5 * (other + (current + dt L(current))),
     * i.e. with the stage-1 state current (after a swap) and the step's
     * initial state in the other buffer, the new state replaces the initial
     * one. Raises the blocks' signal speeds of the new state. The guard fill
     * must refresh the current (stage-1) buffer before it. */
    ORCHA_TASK_RK2_STAGE2 = 6,
    /* For orcha_mesh_advance, orcha_batch_advance and orcha_autotune: whole
     * Heun steps (stage 1, swap, guard fill, stage 2, dt reduce, swap). */
    ORCHA_TASK_HYDRO_RK2 = 7,
    /* The two Heun stages and the whole Heun step with the plain MUSCL
     * operator evaluated as in HYDRO_F32FLUX (FP32 primitives, slopes and HLL
     * fluxes; FP64 flux differences, update, stage-2 average, signal speed
     * and dt). */
    ORCHA_TASK_RK2_F32FLUX_STAGE1 = 8,
    ORCHA_TASK_RK2_F32FLUX_STAGE2 = 9,
    ORCHA_TASK_HYDRO_RK2_F32FLUX = 10,
    /* The same with the operator evaluated as in HYDRO_FF (double-word
     * arithmetic on the FP32 pipe, FP64 update, stage-2 average and dt). */
    ORCHA_TASK_RK2_FF_STAGE1 = 11,
    ORCHA_TASK_RK2_FF_STAGE2 = 12,
    ORCHA_TASK_HYDRO_RK2_FF = 13,
    /* HYDRO_F32FLUX with a cheaper update: each difference dt/dx_d (F_hi -
     * F_lo) of the FP32 face fluxes is formed exactly as a float pair and the
     * x+y+z sum is float-float (about 46 bits, within ~1e-14 of the summed
     * terms); only U+ = U - sum is FP64. The new state's signal speed is
     * evaluated in FP32 and rounded up by 1 + 2^-18 (FP64 where the FP32
     * pressure is not positive); the max-reduction and dt = cfl / max stay
     * FP64, and the first dt uses the same rule. Not in the paper: it moves
     * the per-cell FP64 work off this GPU's scarce FP64 pipe. */
    ORCHA_TASK_HYDRO_F32FLUX_FFSUM = 14,
    /* Batch tasks (orcha_batch_advance only) that apply the operator twice
     * per persistent launch, with one read and one write of the state for
     * both: the paper's doubled halo (both Runge-Kutta stages with no guard
     * refresh between them, the first stage computed redundantly on the
     * inner halo; section "Experiments", Spark paragraph), here to save the
     * intermediate state's round trip through HBM. A CTA advances its tile
     * grown by 2 cells (2 planes in z) into an L2-resident scratch, then the
     * tile itself from the scratch. Each application gives the bits the
     * one-step task gives.
     * TB2: two MUSCL-Hancock steps (as HYDRO_FP64 / HYDRO_F32FLUX) per
     * launch, both with the dt formed from the state at the start of the
     * pair (nsteps must be even); the launch checks dt * s(U1) <= 1 for the
     * intermediate state U1 (the summed-direction rule's stability limit)
     * and sets ORCHA_DEVERR_CFL otherwise. */
    ORCHA_TASK_HYDRO_TB2 = 15,
    ORCHA_TASK_HYDRO_F32FLUX_TB2 = 16,
    /* One whole Heun step (as HYDRO_RK2 / HYDRO_RK2_F32FLUX) per launch. */
    ORCHA_TASK_HYDRO_RK2_FUSED = 17,
    ORCHA_TASK_HYDRO_RK2_F32FLUX_FUSED = 18
} orcha_task;

/* Mesh geometry and the caller's device buffers. */
typedef struct orcha_mesh_desc {
    int32_t ndim;        /* 2 or 3 */
    int32_t nb[3];       /* blocks per axis (nb[2] = 1 in 2D) */
    int32_t bs[3];       /* interior cells per block per axis; bs[0], bs[1] (and bs[2] in 3D)
                            each 8, 16 or 32; bs[2] = 1 in 2D */
    int32_t periodic[3]; /* per axis: 0 outflow (zero-gradient), 1 periodic */
    double gamma;        /* ratio of specific heats (> 1) */
    double cfl;          /* Courant number of the summed-direction rule
                            dt = cfl / max_cells sum_d (|u_d| + c) / dx_d (> 0) */
    double lo[3], hi[3]; /* domain box; dx_d = (hi_d - lo_d) / (nb_d * bs_d) */
    double* state_dev[2];/* two caller-owned device buffers of orcha_state_elems() doubles each,
                            layout [block][var][k][j][i] over the padded block
                            (bs + 4 cells per active axis, i fastest), vars
                            (rho, m_x, m_y[, m_z], E); 16-byte aligned (the
                            kernels load pairs of x-neighbours as one vector) */
    double* dt_dev;      /* caller-owned device double: the current time step (8-byte aligned) */
} orcha_mesh_desc;

typedef struct orcha_mesh orcha_mesh;     /* opaque */
typedef struct orcha_packet orcha_packet; /* opaque */

/* Number of doubles in one state buffer of this geometry (0 if invalid). */
ORCHA_API size_t orcha_state_elems(const orcha_mesh_desc* desc);

/* Validate desc and create a mesh over the caller's buffers. State buffer 0
 * is current. Allocates the per-block signal-speed array and the error word
 * on the current device. Errors: INVALID (geometry, null buffers), OOM, CUDA. */
ORCHA_API orcha_status orcha_mesh_create(const orcha_mesh_desc* desc, orcha_mesh** out);

/* Free the library's allocations (not the caller's buffers). Waits for the
 * device. NULL is accepted. */
ORCHA_API orcha_status orcha_mesh_destroy(orcha_mesh* mesh);

/* Index (0 or 1) of the current state buffer. */
ORCHA_API int32_t orcha_mesh_current(const orcha_mesh* mesh);

/* Make the other state buffer current (after all packets have run a hydro
 * task for this step). Host-side only; stream order is the caller's. */
ORCHA_API orcha_status orcha_mesh_swap(orcha_mesh* mesh);

/* Column tile of the hydro kernel: one CTA sweeps a tx x ty column tile of a
 * block along z. Built variants: 8x8, 16x8, 16x16; tx must divide bs[0] and
 * ty must divide bs[1]. The tile does not change any result bit (each face
 * flux is evaluated by the same expression whatever the tiling). Errors:
 * UNSUPPORTED (no such variant), INVALID (does not divide the block), CUDA. */
ORCHA_API orcha_status orcha_mesh_set_tile(orcha_mesh* mesh, int32_t tx, int32_t ty);
ORCHA_API orcha_status orcha_mesh_get_tile(const orcha_mesh* mesh, int32_t* tx, int32_t* ty);

/* Pack: copy interior cells into the current state buffer. `interior` holds
 * [block][var][k][j][i] over the interior cells only (nblocks * nvar * cells
 * per block doubles). host_ptr != 0: `interior` is host memory (pinned for
 * true asynchrony), staged through a library device buffer; otherwise it is
 * a device pointer. Guards are not filled. Errors: INVALID, OOM, CUDA. */
ORCHA_API orcha_status orcha_mesh_load(orcha_mesh* mesh, const double* interior, int32_t host_ptr, void* stream);

/* Unpack: copy the interiors of the current state buffer out to `interior`
 * (same layout and host_ptr meaning as orcha_mesh_load). */
ORCHA_API orcha_status orcha_mesh_store(orcha_mesh* mesh, double* interior, int32_t host_ptr, void* stream);

/* Write a two-region initial state (ORCHA_INIT_SPHERE or ORCHA_INIT_HALF_SPACE,
 * rule as for serving requests below) into the interiors of the current
 * state buffer on the device. Errors: INVALID, CUDA. */
ORCHA_API orcha_status orcha_mesh_init_region(orcha_mesh* mesh, int32_t kind, const int32_t region[4],
                                              const double u_in[5], const double u_out[5], void* stream);

/* Create a packet over n distinct block ids of the mesh (host array, copied).
 * Errors: INVALID (n < 1, an id outside [0, nblocks) or repeated), OOM, CUDA. */
ORCHA_API orcha_status orcha_packet_create(orcha_mesh* mesh, const int32_t* block_ids, int32_t n, orcha_packet** out);

ORCHA_API orcha_status orcha_packet_destroy(orcha_packet* packet);

/* Enqueue `task` for every block of the packet on `stream` (a cudaStream_t;
 * NULL = legacy default stream). Hydro and signal-speed tasks raise the
 * blocks' entries of the mesh's signal-speed array; orcha_dt_reduce consumes
 * them. Errors: INVALID, UNSUPPORTED (block size), CUDA (launch). */
ORCHA_API orcha_status orcha_packet_run(orcha_packet* packet, orcha_task task, void* stream);

/* Unpack a packet (the paper's "moving data back", section "DataItem
 * Generators"): copy the interiors of the packet's blocks, in packet order
 * ([position in the packet][var][k][j][i] doubles), from the mesh's current
 * state buffer to dst: host memory when dst_is_host (pinned for the copy to
 * be asynchronous; staged through a device buffer the packet owns), else
 * device memory. The blocks stay resident: a hydro task already wrote them in
 * place, so dst = NULL is a no-op, and the copy is made only on request.
 * Stream-ordered. Errors: INVALID (null packet), OOM, CUDA. */
ORCHA_API orcha_status orcha_packet_unpack(orcha_packet* packet, double* dst, int32_t dst_is_host, void* stream);

/* Pack a packet: write the interiors of its blocks from src (same layout and
 * host/device meaning as orcha_packet_unpack) into the mesh's current state
 * buffer; the other blocks are untouched. Errors: INVALID (null argument),
 * OOM, CUDA. */
ORCHA_API orcha_status orcha_packet_pack(orcha_packet* packet, const double* src, int32_t src_is_host, void* stream);

/* dt_dev = cfl / (largest signal speed raised since the previous reduce, over
 * all blocks), then clear the signal-speed array. A non-positive or
 * non-finite maximum sets ORCHA_DEVERR_BAD_DT and leaves dt_dev unchanged. */
ORCHA_API orcha_status orcha_dt_reduce(orcha_mesh* mesh, void* stream);

/* Whole steps over a set of packets that covers the mesh:
 *   if (init_dt) SIGNAL_SPEED on every packet, dt_reduce;
 *   repeat nsteps: GUARD_FILL on every packet; hydro_task on every packet;
 *                  dt_reduce; swap.
 * For HYDRO_F32FLUX_FFSUM the first dt uses that task's FP32 signal-speed
 * rule (as every later step's dt does); otherwise the FP64 SIGNAL_SPEED task.
 * hydro_task: HYDRO_FP64, HYDRO_F32FLUX, HYDRO_F32FLUX_FFSUM, HYDRO_FF, or
 * HYDRO_RK2 (and its FP32-flux and double-word forms), whose step
 * is GUARD_FILL, RK2_STAGE1, swap, GUARD_FILL, RK2_STAGE2, dt_reduce, swap
 * (the current buffer is the same before and after a step).
 * use_graph != 0 captures the nsteps-step sequence in a CUDA graph the first
 * time and replays it afterwards (the graph is cached on the mesh, keyed by
 * the packet set, task, step count and current buffer). Errors: INVALID
 * (packets not covering the mesh, not a whole-step task, graph capture on
 * the legacy default stream), CUDA. */
ORCHA_API orcha_status orcha_mesh_advance(orcha_mesh* mesh, orcha_packet* const* packets, int32_t npackets,
                                orcha_task hydro_task, int32_t nsteps, int32_t init_dt,
                                int32_t use_graph, void* stream);

/* ------------------------------------------------------------------ batches
 * A batch is a fixed set of packets (of one or more meshes) whose steps run
 * as ONE persistent launch per time step: resident CTAs drain a device work
 * queue of (mesh, block, column tile) items, read each tile's halo directly
 * from the neighbouring blocks (no guard-fill pass; the padded guard layers
 * are left untouched), and the CTA finishing a mesh's last item forms that
 * mesh's next dt and flips its current buffer on the device. The packets of
 * each mesh in the batch must cover all of its blocks exactly once. All
 * meshes need the same ndim, and the tile must divide every mesh's blocks. */
typedef struct orcha_batch orcha_batch;

/* tx = ty = 0 picks the widest built tile that divides every mesh's blocks.
 * Errors: INVALID (coverage, mixed ndim, tile does not divide), UNSUPPORTED,
 * OOM, CUDA. The packets and meshes must outlive the batch. */
ORCHA_API orcha_status orcha_batch_create(orcha_packet* const* packets, int32_t npackets, int32_t tx, int32_t ty,
                                          orcha_batch** out);
ORCHA_API orcha_status orcha_batch_destroy(orcha_batch* batch);

/* nsteps steps of every mesh in the batch on `stream` (hydro_task as for
 * orcha_mesh_advance; a HYDRO_RK2 step is two launches, one per stage).
 * init_dt != 0 first forms each mesh's dt from its current state (the
 * value of the signal-speed task + dt reduce; for the FP64 speed rule the
 * FP64 speed is evaluated only where FP32 bounds leave a cell that can hold
 * the maximum, with the same bits); otherwise each mesh's dt_dev must already
 * hold its time step. use_graph != 0 captures the nsteps steps' launches
 * once per (task, nsteps) and replays the graph (needs a non-default
 * stream). After the call each mesh's current buffer is the one its last
 * step wrote. Errors: INVALID, UNSUPPORTED (the variant does not fit an SM),
 * OOM, CUDA. */
ORCHA_API orcha_status orcha_batch_advance(orcha_batch* batch, orcha_task hydro_task, int32_t nsteps,
                                           int32_t init_dt, int32_t use_graph, void* stream);

/* ------------------------------------------------------------------ serving
 * A server advances independent simulations ("requests") with continuous
 * batching. The paper's runtime keeps data packets moving between host and
 * device on GPU streams so transfers hide behind computation (sections
 * "Milhoja" and "Sedov Blast Wave Results"); here one worker thread owns the
 * device: it admits requests in arrival order while their state fits an
 * HBM budget (one device pool reserved at creation; a request that does not
 * fit waits, it is not failed), copies their initial state in on a copy
 * stream, advances every admitted request by one time step per persistent
 * launch (requests join and leave between launches; at most two launches
 * are queued ahead), and copies finished requests out on the copy stream.
 * Each request keeps its own dt. A request's result does not depend on the
 * other requests in flight. */
typedef struct orcha_server orcha_server;


typedef struct orcha_request_desc {
    int32_t ndim, nb[3], bs[3], periodic[3]; /* as in orcha_mesh_desc */
    double gamma, cfl, lo[3], hi[3];
    int32_t nsteps;           /* time steps to advance (>= 1); the first dt comes from the initial state */
    int32_t task;             /* ORCHA_TASK_HYDRO_FP64, _F32FLUX, _F32FLUX_FFSUM or _FF */
    int32_t init_kind;        /* ORCHA_INIT_* */
    int32_t region[4];
    double u_in[5], u_out[5]; /* conserved states (rho, m_x, m_y[, m_z], E) of the recipes */
    const double* init_host;  /* FROM_HOST: interior cells [block][var][k][j][i]; host memory (pinned
                                 for overlap) valid until the request completes */
    double* out_host;         /* NULL, or the same layout: receives the final state */
} orcha_request_desc;

typedef struct orcha_request_stats {
    double t_submit_us, t_admit_us, t_ready_us, t_done_us; /* server clock (us since creation) */
    int64_t zone_updates;     /* interior cells x steps */
    double totals[5];         /* final sum over interior cells of each conserved variable (fixed order) */
    double dt_next;           /* the time step the final state gives */
    int32_t device_error;     /* ORCHA_DEVERR_* bits this request raised */
    int32_t status;           /* ORCHA_OK, or ORCHA_ERR_NONFINITE when device_error != 0 */
} orcha_request_stats;

typedef struct orcha_server_stats {
    int64_t submitted, completed, steps_launched, zone_updates;
    double now_us;
    size_t pool_bytes, pool_peak_bytes;
} orcha_server_stats;

/* Reserve a device pool of hbm_budget_bytes and start the worker on the
 * current device. max_active bounds the requests holding device memory at
 * once. The pool also holds the step loop's work lists, sized here once
 * (two in-flight steps x (max_active request slots + one 16-byte item per
 * 4 KiB of pool), about 0.8 % of the budget), so the worker never allocates
 * or frees device memory while serving. Errors: INVALID, OOM, CUDA. */
ORCHA_API orcha_status orcha_server_create(size_t hbm_budget_bytes, int32_t max_active, orcha_server** out);
/* Stop the worker, wait for the device, free everything. Requests not yet
 * waited for are dropped. */
ORCHA_API orcha_status orcha_server_destroy(orcha_server* server);
/* Queue a request (thread-safe, returns at once). Errors: INVALID
 * (geometry, steps, task, buffers), OOM (larger than the whole budget). */
ORCHA_API orcha_status orcha_server_submit(orcha_server* server, const orcha_request_desc* request, int64_t* ticket);
/* Block until the request is done (timeout_ms < 0: no limit) and release its
 * ticket; stats may be NULL. Errors: TIMEOUT (still running, ticket kept),
 * NONFINITE (finished with a device error), INVALID, CUDA (server failed). */
ORCHA_API orcha_status orcha_server_wait(orcha_server* server, int64_t ticket, int32_t timeout_ms,
                                         orcha_request_stats* stats);
ORCHA_API orcha_status orcha_server_get_stats(orcha_server* server, orcha_server_stats* out);

/* ------------------------------------------------------------------ autotuning
 * Pick the fastest built column tile (tx, ty) of the hydro kernel for blocks
 * of bs[0] x bs[1] (x bs[2] in 3D) cells and the given hydro task: each
 * variant dividing the block is timed on a synthetic periodic mesh of about
 * `nblocks` blocks through the persistent batch path (2 warm-up + 5 timed
 * steps). All variants give the same result bits; the choice only affects
 * speed. With cache_path != NULL the answer is read from / written to that
 * JSON file, keyed by GPU name, ndim, block size and task, so tuning runs once
 * per machine. ms_out (may be NULL) receives the best time per step (-1 when a
 * cache entry has none). Allocates and frees its own temporary mesh;
 * synchronises the device. The paper names auto-tuned kernel generation as
 * future work (section "Conclusions"). Errors: INVALID, UNSUPPORTED, OOM,
 * CUDA. */
ORCHA_API orcha_status orcha_autotune(int32_t ndim, const int32_t bs[3], orcha_task hydro_task, int32_t nblocks,
                                      const char* cache_path, int32_t* tx, int32_t* ty, double* ms_out);

/* ------------------------------------------------------------------ two-level AMR
 * Block AMR with flux correction. The paper's application runs on an AMR
 * mesh, where adjacent blocks at different refinement levels need their
 * boundary fluxes reconciled (flux correction); the paper does that in a
 * second, low-intensity step outside its task functions (section
 * "Experiments", Spark paragraph). Here the whole two-level step runs on the
 * device.
 *
 * The coarse level is the uniform block grid of a mesh descriptor (its two
 * state buffers and dt_dev). Each of the nref coarse blocks in `refined` is
 * covered by 2^ndim fine blocks of the same cell count and half the cell
 * width; fine block f is child f % 2^ndim (octant bits x | y << 1 | z << 2)
 * of refined[f >> ndim], stored in two caller-owned fine buffers of
 * orcha_amr_fine_elems() doubles each ([fine block][var][k][j][i] over the
 * padded block, 16-byte aligned). A refined coarse block (a parent) holds the
 * average of its children and is not advanced. One step, both levels with
 * the same dt (FP64 MUSCL-Hancock):
 *   parents <- restriction of their children (pairwise sums, times 2^-ndim);
 *   guard fill: coarse from the coarse level (parents included); fine from
 *     the fine blocks, or the coarse cell that contains the guard cell
 *     (piecewise-constant prolongation); the boundary rule applies on each
 *     level's own index space;
 *   every coarse leaf and every fine block advances, recording the fluxes
 *     through its faces;
 *   flux correction: a coarse leaf cell next to a refined block is corrected
 *     by (dt/dx)(F_coarse - average of the 2^(ndim-1) fine fluxes) through
 *     that face, so the total of U dV over the leaf cells is conserved;
 *   parents <- restriction; dt = cfl / max over leaf cells of both levels of
 *     sum_d (|u_d| + c) / dx_d.
 * Calls are stream-ordered like the mesh calls; create allocates the flux
 * registers (6 faces x nvar x the largest face of a block, per block) and
 * small index arrays. */
typedef struct orcha_amr orcha_amr;

/* Doubles in one fine state buffer (0 if the descriptor is invalid). */
ORCHA_API size_t orcha_amr_fine_elems(const orcha_mesh_desc* coarse, int32_t nref);
/* Errors: INVALID (descriptor, ids out of range or repeated, buffers), OOM, CUDA. */
ORCHA_API orcha_status orcha_amr_create(const orcha_mesh_desc* coarse, const int32_t* refined, int32_t nref,
                                        double* fine_state0_dev, double* fine_state1_dev, orcha_amr** out);
ORCHA_API orcha_status orcha_amr_destroy(orcha_amr* amr);
/* Copy interiors into / out of the current buffers of both levels: coarse
 * [block][var][k][j][i] over all coarse blocks (a parent's cells are
 * replaced by its children's average at the next advance), fine [fine
 * block][var][k][j][i]. host_ptr != 0: host memory (staged; the call waits
 * for the copy), else device memory. */
ORCHA_API orcha_status orcha_amr_load(orcha_amr* amr, const double* coarse, const double* fine, int32_t host_ptr,
                                      void* stream);
ORCHA_API orcha_status orcha_amr_store(orcha_amr* amr, double* coarse, double* fine, int32_t host_ptr, void* stream);
/* nsteps two-level steps; init_dt != 0 first forms dt from the current leaf
 * cells, otherwise dt_dev must hold it; each step leaves the next dt there. */
ORCHA_API orcha_status orcha_amr_advance(orcha_amr* amr, int32_t nsteps, int32_t init_dt, void* stream);
/* As orcha_mesh_poll, for both levels. */
ORCHA_API orcha_status orcha_amr_poll(orcha_amr* amr, void* stream, int32_t* device_error);

/* ------------------------------------------------------------------ no-allocation CFL step
 * The paper has no counterpart to this call. It serves callers that cannot
 * let a library allocate device memory (for example a host code whose own
 * allocator owns all of HBM, or a time loop where allocation is forbidden).
 *
 * Computes dt_dev = cfl / (largest signal speed sum_d (|u_d| + c) / dx_d over
 * the interior cells of desc->state_dev[current]) -- the same value that the
 * SIGNAL_SPEED task followed by orcha_dt_reduce gives -- without creating a
 * mesh and without any allocation: no cudaMalloc, no cudaFree, no allocating
 * library routine. Its per-block scratch is a file-scope device array of
 * ORCHA_NOALLOC_MAX_BLOCKS entries that every GPU loading the library holds
 * until exit; meshes with more blocks are rejected with ORCHA_ERR_INVALID.
 * The caller passes the inputs and outputs: desc (geometry, state buffers,
 * dt_dev) and err_dev, a device int32 into which ORCHA_DEVERR_* bits are
 * OR-ed (the caller clears it); guards need not be filled.
 * Each call outside stream capture looks up the array's device address in
 * the current context (so a context reset between calls is safe); a call
 * made while `stream` is capturing reuses the address that the last
 * uncaptured call on this device saw, so make a first call on each device
 * before any stream capture (a capture after a context reset needs another
 * uncaptured call first). Every call shares the one array and clears the entries it uses
 * at its start, so calls that overlap on the GPU (other streams, other host
 * threads) race and must be serialised by the caller. Asynchronous on
 * `stream`. Errors: INVALID (descriptor, buffers, size limit), UNSUPPORTED,
 * CUDA. */
#define ORCHA_NOALLOC_MAX_BLOCKS 65536
ORCHA_API orcha_status orcha_cfl_dt_noalloc(const orcha_mesh_desc* desc, int32_t current, int32_t* err_dev,
                                            void* stream);

/* Wait for `stream`, then read the device error word into *device_error (0 =
 * none) and clear it. Returns NONFINITE when a bit is set. */
ORCHA_API orcha_status orcha_mesh_poll(orcha_mesh* mesh, void* stream, int32_t* device_error);

/* Diagnostics: the FP32-flux task converts between binary64 and binary32 on
 * the integer pipe (bit-field arithmetic from the IEEE-754 formats, with the
 * hardware conversion for subnormal, infinite and NaN cases). This checks
 * them against the hardware conversions on the current device: binary32 ->
 * binary64 for the `count` patterns starting at first_pattern, and binary64 ->
 * binary32 (round to nearest even) for `count` pseudo-random patterns derived
 * from `seed`; *mismatches receives the number of results whose bits differ
 * (NaN payloads excepted). Synchronous. Errors: INVALID, CUDA. */
ORCHA_API orcha_status orcha_selftest_conversions(uint64_t first_pattern, uint64_t count, uint64_t seed,
                                                  uint64_t* mismatches);

/* Diagnostics: part of the FP64 task's adds, subtracts and multiplies are
 * computed with integer instructions (the FP64 pipe is the bound of that
 * task on this GPU), exactly as IEEE-754 round-to-nearest-even defines them.
 * This checks them against the hardware instructions on `count`
 * pseudo-random operand pairs derived from `seed` (biased toward carries,
 * ties, cancellation and zeros); *mismatches receives the number of results
 * whose bits differ (NaN results excepted). The same pairs also check the
 * FP64 task's integer-pipe sign tests (x > 0, x < 0, x >= 0, x <= 0), the
 * order of its HLL wave speeds (x < y, except that -0 counts below +0),
 * minmod and the halving 0.5 * x against FP64 comparisons and the hardware
 * multiply (NaN operands excepted), and the FP32 tasks' minmod (a median of
 * three) against its sign-test definition on binary32 pairs cut from the
 * same operands, bit for bit; each disagreement counted as a mismatch.
 * Synchronous. */
ORCHA_API orcha_status orcha_selftest_fp64_emulation(uint64_t count, uint64_t seed, uint64_t* mismatches);

/* Diagnostics: the FF task computes in double-word arithmetic (pairs of
 * binary32 numbers). This measures its building blocks against FP64
 * references on `count` pseudo-random operands derived from `seed`
 * (magnitudes 2^-30 .. 2^30, both signs, half of the sum operands nearly
 * cancelling) and writes the largest errors to max_err: [0] binary64 ->
 * double-word (relative), [1] sum (relative to |x| + |y|), [2] product,
 * [3] reciprocal, [4] reciprocal square root, [5] sound speed
 * sqrt(x / rho) (relative). Synchronous. Errors: INVALID, CUDA. */
ORCHA_API orcha_status orcha_selftest_dword(uint64_t count, uint64_t seed, double max_err[6]);

/* Diagnostics: the persistent one-step tasks skip the FP64 signal speed of a
 * cell whose FP32 upper bound lies below a quarter of the previous step's
 * largest speed (the dt rule CFL / max_cells sum_d (|u_d| + c) / dx_d needs
 * only the maximum; the step's reducer re-evaluates in FP64 whenever a
 * skipped bound could exceed it, so dt keeps its bits). This checks the
 * bound against the FP64 speed on `count` pseudo-random 3D states derived
 * from `seed` (densities 2^-20 .. 2^20, speeds up to 10^6, pressures down to
 * 10^-14 of the kinetic energy density): counts[0] = states where the bound
 * applied but lies below the FP64 speed, or where the lower bound that the
 * first time step's filter pairs with it (the same conditions, the same upper
 * bits) lies above the FP64 speed (0 when both are sound),
 * counts[1] = states where it applied, counts[2] = states where it applied
 * although the FP64 evaluation finds the state non-physical (0 when sound);
 * *max_ratio = the largest bound / speed ratio. Synchronous. Errors:
 * INVALID, CUDA. No counterpart in the paper (a check of this build's
 * arithmetic). */
ORCHA_API orcha_status orcha_selftest_speed_bound(uint64_t count, uint64_t seed, uint64_t counts[3], double* max_ratio);

/* Diagnostics: the FP64 pipe's throughput on the current device, in lane
 * operations per second (one FMA, add or multiply = one operation): op 0
 * FMA, 1 add, 2 multiply, 3 an add issued as an FMA with a run-time 1.0,
 * 4 a multiply issued as an FMA with a run-time -0.0 (the same bits). Every SM runs its maximum resident warps, each
 * thread eight independent chains of the operation; best of five timed
 * launches after one warm-up (about 0.1 s each). This is the ceiling of the
 * FP64 hydro task, which the FP64 pipe bounds on this GPU (the task's
 * operations per zone are counted in the same unit). Synchronous; allocates
 * and frees 8 bytes and one stream. Errors: INVALID, CUDA. */
ORCHA_API orcha_status orcha_measure_fp64_rate(int32_t op, double* lane_ops_per_s);

/* Message of the last error returned on this thread ("" if none). */
ORCHA_API const char* orcha_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* ORCHA_H */
