/*
 * d2q37.h - C ABI of the GB300 (sm_103a) thermal D2Q37 lattice Boltzmann step.
 *
 * One time step of the method of Calore et al., "Massively parallel lattice
 * Boltzmann codes on large GPU clusters": pbc (periodic x halos) -> propagate
 * (pull form, Eq. master2) -> bc (top/bottom walls) -> collide (BGK relaxation
 * to the shifted equilibrium of Eq. MASTERSHIFT3, Eq. discrete), or a fused
 * propagate+collide pass (Sec. "Performance Analysis", last paragraph, and the
 * fused kernels of Sec. "2D Splitting").
 *
 * Conventions shared by every entry point:
 *  - Return value: LBM_OK (0) on success, a negative LBM_E* code on failure;
 *    lbm_strerror() gives its text.  No entry point aborts the process.
 *  - Lattice: Lx x Ly physical sites, x periodic, y bounded by a bottom wall
 *    (y = 0 side, temperature T_bot) and a top wall (y = Ly - 1 side, T_top)
 *    unless periodic_y is set.  Gravity g = (0, -g0).  Lengths are in lattice
 *    sites, time in steps, velocities and temperatures in the thermal units
 *    of the quadrature (reference temperature 1).
 *  - Host field arrays are caller-owned FP64, site (x, y) at index x*Ly + y.
 *    Population arrays are [37][Lx][Ly], population order as returned by
 *    lbm_velocity_set().
 *  - All work is enqueued on the handle's CUDA stream and is asynchronous
 *    unless an entry point says it synchronises.  A handle is not thread-safe;
 *    separate handles may be driven from separate threads and streams.
 *  - The library never frees memory it did not allocate.
 */
#ifndef D2Q37_H
#define D2Q37_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_Q 37

#define LBM_OK 0
#define LBM_EINVAL (-1)   /* bad argument: NULL, Lx < 3, Ly < 6, tau <= 0.5, bad phase mask */
#define LBM_ENOMEM (-2)   /* device allocation failed, or caller buffer too small */
#define LBM_ECUDA (-3)    /* a CUDA call or kernel launch failed */
#define LBM_ETIMEOUT (-4) /* reserved for bounded device waits */
#define LBM_ESTATE (-5)   /* call out of order, e.g. a step before any initial state */
#define LBM_ETOOBIG (-6)  /* more lattices than lbm_batch_step_static's fixed table holds */

/* Phase bits for lbm_run_phases(). */
#define LBM_PHASE_PROPAGATE 1 /* pbc + pull propagate (Sec. "Code Organization") */
#define LBM_PHASE_BC 2        /* wall bc; only together with LBM_PHASE_PROPAGATE */
#define LBM_PHASE_COLLIDE 4   /* BGK collide (Eq. discrete) */
#define LBM_PHASE_ALL 7

/* Storage precisions for lbm_params.precision. */
#define LBM_PRECISION_FP64 0      /* FP64 populations, FP64 arithmetic */
#define LBM_PRECISION_FP32_FP64 1 /* FP32 deviations f - w; FP64 for rho, u, T and T-dependent terms */
#define LBM_PRECISION_FP32_DF 2   /* FP32 deviations; those terms in double-float on the FP32 pipes */

/* Kernel schedules for lbm_params.kernel. */
#define LBM_KERNEL_SEPARATE 0 /* pbc, propagate, bc, collide as separate kernels */
#define LBM_KERNEL_FUSED 1    /* pbc, then one fused propagate+bc+collide kernel */
#define LBM_KERNEL_FUSED_SERIAL 2 /* as FUSED; the FP64 wall-band kernel starts only after the sites
                                     kernel has finished (FUSED lets it start in that kernel's tail);
                                     the results are the same bit for bit */

typedef struct lbm_t lbm_t;

typedef struct {
  double tau;     /* BGK relaxation time in steps, > 0.5 (paper: symbol tau, value not given) */
  double g0;      /* gravity magnitude; g = (0, -g0) */
  double T_top;   /* top wall temperature */
  double T_bot;   /* bottom wall temperature */
  int precision;  /* LBM_PRECISION_*: populations stored as FP64, or as FP32 deviations
                     d_l = f_l - w_l from the lattice weights (half the memory traffic) with the
                     moment sums exact in 64-bit integers and rho, u, T and the temperature-
                     dependent equilibrium terms in FP64 or in double-float */
  int kernel;     /* LBM_KERNEL_SEPARATE, LBM_KERNEL_FUSED or LBM_KERNEL_FUSED_SERIAL */
  int periodic_y; /* 1: no walls, y periodic too (used by tests of pure propagation) */
} lbm_params;

/* Defaults: tau 0.8, g0 1e-4, T_top 0.5, T_bot 1.5, FP64, fused, walls. */
void lbm_default_params(lbm_params* p);

/* The 37 integer hops c_l = (cx[l], cy[l]) in this library's population
 * order (Sec. "Lattice Boltzmann methods": labels are arbitrary).  cx, cy are
 * caller arrays of 37 ints.  Host only; never fails for non-NULL pointers. */
int lbm_velocity_set(int* cx, int* cy);

/* Thermal scale s (xi_l = s c_l) and the 37 weights w_l in population order,
 * solved by this library at first use.  Host only. */
int lbm_quadrature(double* s, double* w);

/* Device bytes needed for an Lx x Ly lattice: two population copies of
 * 37 x (Lx+6) x NY sites (FP64: NY = Ly + 32 rounded up to 16; FP32
 * storage: NY = Ly + 64 rounded up to 32) plus a scratch of 4 Lx Ly
 * doubles.  0 for invalid sizes or parameters. */
size_t lbm_required_bytes(int Lx, int Ly, const lbm_params* p);

/* Create a lattice on the current CUDA device; allocates its own device
 * memory (cudaMalloc) and its own stream.  *out is set only on success. */
int lbm_create(int Lx, int Ly, const lbm_params* p, lbm_t** out);

/* As lbm_create, but the device memory is the caller's: dev_buf (256-byte
 * aligned, at least lbm_required_bytes) stays owned by the caller and must
 * outlive the handle; cuda_stream is a cudaStream_t (NULL: legacy default
 * stream) on which all work of this handle is enqueued. */
int lbm_create_ext(int Lx, int Ly, const lbm_params* p, void* dev_buf, size_t bytes, void* cuda_stream,
                   lbm_t** out);

/* Rayleigh-Taylor initial state (the workload of Sec. "Overview of Physics
 * Results"): cold T_top fluid over hot T_bot fluid, interface
 * y_i(x) = Ly/2 + (Ly/64) sin(2 pi (x + 1/2) / Lx), T scaled by
 * 1 + 1e-3 (2U - 1), U = (splitmix64(seed + x Ly + y) >> 11) 2^-53;
 * rho = 1/T, u = 0, populations at equilibrium.  The temperature field is
 * built on the host (host-side scratch of 8 Lx Ly bytes) and uploaded; this
 * call synchronises the handle's stream. */
int lbm_init_rayleigh_taylor(lbm_t* h, uint64_t seed);

/* Upload / download all physical populations, host [37][Lx][Ly] FP64 in this
 * library's order.  Pinned host memory makes the copies asynchronous; the
 * download synchronises the stream before returning. */
int lbm_set_populations(lbm_t* h, const double* f);
int lbm_get_populations(lbm_t* h, double* f);

/* n full time steps (pbc -> propagate -> bc -> collide, Sec. "Code
 * Organization"), asynchronous on the handle's stream. */
int lbm_step(lbm_t* h, int n);

/* n repetitions of the selected phases (LBM_PHASE_* bits) with the separate
 * kernels, for phase-by-phase checking.  BC requires PROPAGATE. */
int lbm_run_phases(lbm_t* h, int n, int phases);

/* Macroscopic fields of the current populations (Sec. "Lattice Boltzmann
 * methods": rho = sum f, rho u = sum xi f, D rho T = sum |xi - u|^2 f).
 * Host arrays rho[Lx Ly], u[2 Lx Ly] (ux plane then uy plane), T[Lx Ly];
 * synchronises the stream. */
int lbm_fields(lbm_t* h, double* rho, double* u, double* T);

/* Same fields into caller device arrays, asynchronous on the stream. */
int lbm_fields_device(lbm_t* h, double* rho, double* u, double* T);

/* Wait for all work enqueued on the handle's stream; reports any
 * asynchronous CUDA error as LBM_ECUDA. */
int lbm_synchronize(lbm_t* h);

/* Number of CUDA kernels this handle has enqueued so far, graph replays
 * included: a fused FP64 step of a lattice with walls is two (the sites, then
 * the wall-band rows), a fused FP32-storage step or one without walls one; a
 * separate step one per phase run (propagate, bc with walls, collide); pbc
 * one. */
int64_t lbm_launch_count(const lbm_t* h);

/* Kernel kinds reported by lbm_kernel_times(). */
#define LBM_KIND_WRAP 0
#define LBM_KIND_PROPAGATE 1
#define LBM_KIND_BC 2
#define LBM_KIND_COLLIDE 3
#define LBM_KIND_FUSED 4
#define LBM_KIND_FIELDS 5
#define LBM_KIND_INIT 6
#define LBM_KIND_CONVERT 7 /* FP64 <-> FP32-deviation conversions of set/get populations */
#define LBM_KIND_COUNT 8

/* Per-kernel timing (not in the paper; measurement support).  enable != 0
 * records a CUDA event pair on the handle's stream around every later kernel
 * launch of this handle and clears the totals; 0 stops recording. */
int lbm_set_timing(lbm_t* h, int enable);

/* Totals since timing was enabled: ms[LBM_KIND_COUNT] of device time per
 * kernel kind and launches[LBM_KIND_COUNT] (either may be NULL).
 * Synchronises the stream. */
int lbm_kernel_times(lbm_t* h, double* ms, int64_t* launches);

/* Release the handle and the device memory it allocated.  NULL-safe. */
void lbm_destroy(lbm_t* h);

/* ---- batched stepping: many lattices, one launch per step -----------------
 * Not in the paper (its lattices are split across GPUs instead); this is the
 * single-GPU form for many independent jobs.  Every lattice keeps its own
 * memory, parameters and state (its lbm_t).  Launch shapes:
 *  - block_y > 0, blocks_per_sm = 0: one launch per step with one block per
 *    tile (one column by block_y rows) of every lattice.  FP64 batches whose
 *    lattices all have walls and the same tau and g (at most 64 lattices,
 *    offsets within 32 bits) run the wall rows in separate wall tiles of the
 *    same launch and read each lattice's offsets from the launch's parameters;
 *    FP32-storage batches of at most 128 lattices read each lattice's
 *    parameters from the launch's parameters; others use the table below.
 *  - block_y > 0, blocks_per_sm > 0: a persistent grid-stride kernel over the
 *    tiles, each lattice's parameters read from a device table.
 *  - block_y = 0: one launch of the single-lattice fused kernel per lattice,
 *    spread over four streams forked from the batch stream and joined back.
 * lbm_batch_step(n >= 4) replays a captured two-step CUDA graph.  Per-site
 * arithmetic is the fused kernel's, so a lattice's result is the same batched
 * or alone. */
typedef struct lbm_batch_t lbm_batch_t;

/* Group n lattices (same precision, each with a state) on cuda_stream (NULL:
 * legacy default stream).  Synchronises the lattices' own streams.  The
 * lattices must outlive the batch and must not be stepped through their own
 * handles while the batch is in use; call lbm_batch_synchronize() before
 * reading their fields or populations. */
int lbm_batch_create(int n, lbm_t* const* lattices, void* cuda_stream, lbm_batch_t** out);

/* n steps of every lattice, asynchronous on the batch stream. */
int lbm_batch_step(lbm_batch_t* b, int n);

/* Launch shape: block_y in {64, 128, 256} rows per tile; blocks_per_sm 0 for
 * one block per tile, else a persistent grid of blocks_per_sm x SM count
 * (at most the kernel's occupancy; LBM_EINVAL otherwise).  block_y = 0 with
 * blocks_per_sm = 0: one single-lattice launch per lattice and step (n
 * launches per step, counted by lbm_batch_launch_count). */
int lbm_batch_set_config(lbm_batch_t* b, int block_y, int blocks_per_sm);
int lbm_batch_get_config(const lbm_batch_t* b, int* block_y, int* blocks_per_sm);

/* Time every launch shape (block_y = 0 included) over trial_steps launches
 * and keep the fastest;
 * the trials recompute the same step, so the lattices' state does not
 * advance.  Outputs (any may be NULL): the chosen shape and its ms per step.
 * Synchronises the batch stream. */
int lbm_batch_autotune(lbm_batch_t* b, int trial_steps, int* block_y, int* blocks_per_sm, double* best_ms);

int lbm_batch_synchronize(lbm_batch_t* b);
int64_t lbm_batch_launch_count(const lbm_batch_t* b);

/* Release the batch (not its lattices).  NULL-safe. */
void lbm_batch_destroy(lbm_batch_t* b);

/* ---- batched stepping without device allocation ----------------------------
 * The paper has no counterpart; this exists for callers that cannot call
 * cudaMalloc: programs whose device memory all belongs to a caching allocator
 * or a pre-registered pool (an extra cudaMalloc would break their memory
 * budget, or fail on a full device), and loops that cannot afford the device
 * synchronisation cudaMalloc/cudaFree may bring.
 *
 * lbm_batch_step_static advances n lattices (same precision, each with a
 * state; their memory is the caller's, e.g. from lbm_create_ext) by `steps`
 * steps, one batched fused launch per step on cuda_stream, exactly as
 * lbm_batch_step with tiles of 128 rows.  It allocates no device memory and
 * calls no allocating library routine: its tile table lives in a file-scope
 * static device array of LBM_STATIC_BATCH_MAX entries (about 680 KB) that
 * every GPU loading this library holds until the process exits.
 *  - n > LBM_STATIC_BATCH_MAX returns LBM_ETOOBIG and does nothing.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress, once per device); make that first call before any
 *    stream capture.
 *  - Every call shares the one array per device and rewrites the entries it
 *    uses (nothing in it needs to start at zero); calls whose work overlaps on
 *    the GPU race on it, so order them (one stream, or events).
 *  - The caller orders the lattices' own pending work before this call; the
 *    lattices' current buffers are updated on return (work still in flight
 *    on cuda_stream).
 *  - The table reaches the device by a copy from pageable host memory, so
 *    each call waits on the host for the work already queued on cuda_stream.
 *  - Every lattice's memory must be on the current device (LBM_EINVAL
 *    otherwise), and cuda_stream must not be capturing (LBM_EINVAL): the
 *    current buffers are switched on the host at call time.
 *  - The batched launches are counted by no handle's lbm_launch_count (as
 *    lbm_batch_step's are counted on its batch, not on its lattices). */
#define LBM_STATIC_BATCH_MAX 256
int lbm_batch_step_static(int n, lbm_t* const* lattices, int steps, void* cuda_stream);

/* ---- serving: continuous batching of simulation jobs ----------------------
 * Not in the paper.  A job is a Rayleigh-Taylor lattice (size, parameters,
 * precision, seed) to advance a given number of steps.  Jobs queue on
 * submission and are admitted, in arrival order with later jobs allowed to
 * pass ones that do not fit yet, whenever their device memory
 * (lbm_required_bytes) fits in the free part of one pre-allocated pool of
 * hbm_budget_bytes.  Each lbm_server_tick first completes the jobs whose
 * fields have arrived (copies them to host memory, frees their device memory),
 * admits what fits, then advances every admitted job by
 * min(max_steps_per_tick, its steps left) steps of its fused step (as
 * lbm_step: replays of captured graphs) on the job's stream (one of eight,
 * assigned at admission to the one with the fewest active sites, so that the
 * jobs run side by side); a job that reaches its step count gets its fields
 * computed on the device, to be completed by a later tick.
 * All calls are from one host thread.  A tick waits for the GPU only to stay
 * at most two ticks ahead of it, or, when every active job is waiting for its
 * fields, for the first of them. */
typedef struct lbm_server_t lbm_server_t;

#define LBM_JOB_QUEUED 0
#define LBM_JOB_ACTIVE 1
#define LBM_JOB_DONE 2

typedef struct {
  int64_t submitted, completed, queued, active;
  int64_t ticks, steps, launches; /* ticks run, steps advanced (summed over jobs), kernels launched */
  size_t budget_bytes, bytes_in_use, largest_free_bytes;
} lbm_server_stats;

/* Allocates the pool (cudaMalloc of hbm_budget_bytes) and 3 streams on the
 * current device.  LBM_ENOMEM if the pool cannot be allocated. */
int lbm_server_create(size_t hbm_budget_bytes, int max_steps_per_tick, lbm_server_t** out);

/* Queue a job; *job_id receives its id (> 0).  p->kernel is ignored (fused).
 * LBM_EINVAL for invalid sizes or parameters, LBM_ENOMEM if the job alone
 * exceeds the budget. */
int lbm_server_submit(lbm_server_t* s, int Lx, int Ly, int steps, const lbm_params* p, uint64_t seed,
                      int64_t* job_id);

/* One scheduling round (see above); *steps_done (may be NULL) = the most
 * steps any job advanced in it, 0 when none did. */
int lbm_server_tick(lbm_server_t* s, int* steps_done);

/* Ids of jobs completed since the last poll (at most max_ids); *n = count. */
int lbm_server_poll(lbm_server_t* s, int64_t* ids, int max_ids, int* n);

/* State (LBM_JOB_*) and steps left of a job that has not been fetched. */
int lbm_server_job_state(const lbm_server_t* s, int64_t id, int* state, int* steps_left);

/* Copy a completed job's fields (layout of lbm_fields) and forget the job.
 * LBM_ESTATE if it has not completed. */
int lbm_server_fetch(lbm_server_t* s, int64_t id, double* rho, double* u, double* T);

int lbm_server_stats_get(const lbm_server_t* s, lbm_server_stats* out);

/* Release the pool, streams and every job.  NULL-safe. */
void lbm_server_destroy(lbm_server_t* s);

const char* lbm_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* D2Q37_H */
