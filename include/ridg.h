/*
 * ridg.h -- C ABI of the GB300 RIDG library (regionally-implicit discontinuous Galerkin).
 *
 * One RIDG time step (Sec. 2) on a uniform, fully periodic Cartesian mesh in 1, 2 or 3
 * dimensions has two parts:
 *   prediction  (Sec. 2.2, eq. pred_full_system): for every cell i the space-time DG
 *               system on its region R_i of 3^d vertex neighbours (eq. region) is solved
 *               and only the centre cell's space-time coefficients W_i are kept;
 *               for a linear flux this is a precomputed region-to-cell operator applied
 *               to every cell (over the region cells upstream of it, on which alone the
 *               centre depends with upwind face values), for a nonlinear flux a Newton
 *               iteration (Sec. 3) with the
 *               quasi-quadrature-free Jacobian (eqs. Jacproj, Jacobian2);
 *   correction  (Sec. 2.3): Q^{n+1}_i = Q^n_i + volume integral of grad Phi . F(w_i)
 *               - surface integral of the Rusanov flux, both from the predicted W.
 *
 * Conventions shared by every entry point
 *   - Basis: Phi_s = prod_d sqrt(2 b_d + 1) P_{b_d}(xi_d) on each cell, orthonormal in
 *     the element-average sense (Sec. 2.1), degree M per dimension, theta_S = (M+1)^d
 *     modes ordered with b_x fastest.  The space-time basis Psi_k = psi_a(tau) Phi_s has
 *     theta_T = (M+1)^(d+1) modes, k = a * theta_S + s (time slowest), so the first
 *     theta_S entries of W_i are its time mean.
 *   - Cells are numbered e = i_x + n_x (i_y + n_y i_z).
 *   - State layout ("canonical"): q[(e * m + r) * theta_S + s], r = conserved variable.
 *     Prediction layout: w[(e * m + r) * theta_T + k].
 *   - All arithmetic that defines the result is FP64 unless a mixed precision is chosen
 *     (see ridg_options.precision); the state is always held in FP64.
 *   - Every call returns an int status (RIDG_OK = 0); nothing is thrown across the ABI.
 *     The handle keeps a message for the last failure (ridg_last_error).
 *   - A handle is bound to the CUDA device that was current at ridg_create and issues all
 *     work on its stream (ridg_options.stream, or a non-blocking stream the handle creates
 *     when that is NULL; CUDA-graph capture needs a stream other than the legacy one).
 *     Device pointers passed in must be on that device; the caller orders them against
 *     the handle's stream.  A handle is not thread-safe.
 *   - Ownership: the caller owns every buffer it passes; the library owns its internal
 *     device state and releases it in ridg_destroy.
 */
#ifndef RIDG_H_
#define RIDG_H_

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ----- status codes ------------------------------------------------------------- */
enum {
  RIDG_OK = 0,
  RIDG_EINVAL = 1,      /* invalid argument, unsupported dimension / degree / flux      */
  RIDG_ENOMEM = 2,      /* host or device allocation failed                              */
  RIDG_ECUDA = 3,       /* a CUDA runtime call failed (message has the CUDA error)       */
  RIDG_ENONFINITE = 4,  /* a non-finite value was found in the state                     */
  RIDG_ENOCONV = 5,     /* Newton hit its iteration cap in some regions; the step still
                           completed and ridg_info reports how many regions                */
  RIDG_ETIMEOUT = 6,    /* a bounded device-side wait gave up                             */
  RIDG_ESTATE = 7,      /* call out of order (e.g. correct before predict, no dt yet)    */
  RIDG_ETOOBIG = 8      /* problem larger than the fixed scratch of ridg_l2_error_noalloc  */
};

/* ----- problem description -------------------------------------------------------- */
typedef struct {
  int dim;          /* 1, 2 or 3                                                        */
  int n[3];         /* cells per dimension (entries beyond dim ignored), each >= 3      */
  double lo[3];     /* domain [lo_d, hi_d], periodic on every face                      */
  double hi[3];
} ridg_mesh;

enum { RIDG_FLUX_ADVECTION = 0, RIDG_FLUX_BURGERS = 1, RIDG_FLUX_EULER = 2 };

typedef struct {
  int kind;         /* RIDG_FLUX_*                                                      */
  double vel[3];    /* advection velocity a (ADVECTION)                                 */
  double gamma;     /* ratio of specific heats (EULER, 2D only, m = 4)                  */
} ridg_flux;

enum {
  RIDG_PREC_FP64 = 0,        /* every step of the path in FP64                           */
  RIDG_PREC_MIXED_BF16 = 1,  /* linear prediction as a sliced BF16 tensor-core contraction
                                with FP32 accumulation recombined into double-float pairs
                                (split-operand refinement); in the step the contraction
                                also yields the correction's volume term and face traces
                                (one composed operator; in 3D at Q2 up to 4 slices, else
                                the time means), the face terms are summed in double-float
                                and the state update is FP64                              */
  RIDG_PREC_MIXED_FP32 = 2,  /* Newton linear solves in FP32 with the residual in FP64
                                (nonlinear flux)                                          */
  RIDG_PREC_MIXED_TF32 = 3,  /* Newton linear solves with the Schur-complement block
                                updates on the TF32 tensor cores (FP32 accumulation), FP32
                                pivot inverses, and refinement sweeps against the FP64
                                residual (nonlinear flux)                                 */
  RIDG_PREC_MIXED_FP16 = 4   /* as MIXED_BF16 with FP16 digit operands: the balanced
                                base-256 digits are exact in FP16 as in BF16 and every
                                digit product and FP32 sum is the same, so the results are
                                bit-identical to MIXED_BF16 at the same tensor rate        */
};

typedef void* (*ridg_alloc_fn)(size_t bytes, void* user);
typedef void (*ridg_free_fn)(void* ptr, void* user);

typedef struct {
  int precision;          /* RIDG_PREC_*                                                */
  int slices;             /* digit slices per operand for MIXED_BF16 / MIXED_FP16, 2..7
                             (0 = default 6)                                                */
  int newton_max_iters;   /* 0 = default 4                                              */
  double newton_tol;      /* <= 0 = default 1e-10: stop when ||dW||_inf <= tol max(1,||W||_inf) */
  void* stream;           /* cudaStream_t (not the legacy default stream) or NULL       */
  ridg_alloc_fn alloc;    /* optional device allocator (default cudaMalloc)             */
  ridg_free_fn free;      /* matching release (default cudaFree)                        */
  void* alloc_user;       /* passed to alloc / free                                     */
} ridg_options;

typedef struct ridg_handle ridg_t;

typedef struct {
  int dim, order, m;            /* dimension, degree M, conserved variables             */
  int theta_s, theta_t;         /* (M+1)^d, (M+1)^(d+1)                                  */
  long long cells;              /* number of cells                                       */
  double dt, t;                 /* current step size and time                            */
  long long steps;              /* steps taken since the last ridg_set_state              */
  long long newton_unconverged; /* regions that hit the Newton cap in the last prediction */
  int newton_iters_max;         /* largest Newton iteration count of the last prediction  */
  int precision, slices;
  long long newton_iters_total; /* Newton iterations summed over the regions of the last
                                   prediction (or of the steps of the last ridg_step)      */
  long long newton_hist[16];    /* regions by Newton iteration count over the same span
                                   (entry k: k iterations; entry 15: 15 or more)           */
  double mass[4];               /* sum over cells of |T| Q_{e, r, 0} per conserved variable
                                   r < m (Sec. 2.3: conserved by the correction); the
                                   entries beyond m are 0                                  */
} ridg_info_t;

/* ----- lifecycle -------------------------------------------------------------------- */

/* Build the tables and operators for degree `order` (M >= 0) and allocate device state.
 * Linear flux: the region system of eq. pred_full_system (Sec. 2.2) is solved on the host
 * in FP64 once -- by block substitution over the region cells upstream of the centre
 * (offsets {-1, 0} along a_d > 0, {0, +1} along a_d < 0, {0} where a_d = 0; the others do
 * not reach the centre) -- and the centre rows of its solution operator over those cells
 * (and their time mean) are copied to the device.  Nonlinear flux: the quadrature and
 * quasi-quadrature-free tables of Sec. 3 are built.  dt is set from `cfl` for advection
 * (dt = cfl h_min / max|a_d|); for nonlinear flux it is set by ridg_set_state.
 * Supported: ADVECTION d = 1 (M <= 11), d = 2, 3 (M <= 5; the mixed precisions M <= 3 in
 * 2D, M <= 2 in 3D); BURGERS d = 2 (M <= 4) and d = 3 (M = 1: FP64 or MIXED_FP32 region
 * solves, a dense LU of the 3 x 3 x 3 region's 432 unknowns per Newton iteration); EULER
 * d = 2 (M <= 2).  `opt` may be NULL.
 * On success *out owns the new handle.                                                 */
int ridg_create(const ridg_mesh* mesh, int order, const ridg_flux* flux, double cfl,
                const ridg_options* opt, ridg_t** out);

/* Release all device and host state of the handle (NULL is accepted).                  */
void ridg_destroy(ridg_t* h);

/* ----- state ------------------------------------------------------------------------ */

/* Copy the state in (canonical layout, cells * m * theta_S doubles); `on_device` != 0
 * means q is a device pointer.  A page-locked host buffer (16-byte aligned) is read by
 * the GPU's SMs directly, copy and finite check in one pass; other host memory goes
 * through a copy-engine copy.  Resets t = 0 and the step count.  For a nonlinear flux
 * dt = cfl h_min / (largest wave speed of q) is computed here unless ridg_set_dt fixed
 * it.  RIDG_ENONFINITE if q holds a NaN or Inf.  Synchronous.                          */
int ridg_set_state(ridg_t* h, const double* q, int on_device);

/* Copy the state out (same layout).  Synchronous with the handle's stream.              */
int ridg_get_state(ridg_t* h, double* q, int on_device);

/* Fix dt (> 0) for the following steps (used to land exactly on a final time).          */
int ridg_set_dt(ridg_t* h, double dt);

/* Shorten dt so that an integer number of steps reaches T: N = ceil(T / dt - 1e-9),
 * dt = T / N; *nsteps (may be NULL) receives N.                                         */
int ridg_set_final_time(ridg_t* h, double T, long long* nsteps);

/* ----- the step ---------------------------------------------------------------------- */

/* Prediction (Sec. 2.2): every cell's centre space-time coefficients W_i from the
 * current state.  With a mixed linear precision (2D, 3D) it runs the split-digit
 * tensor-core contraction of all theta_T rows (in 3D one launch per block of up to 64 rows,
 * 32 at 5-6 slices: a block of up to 32 rows written in FP64 by its own launch, a wider one
 * through a double-float buffer and a conversion pass).
 * If w_out is not NULL it receives cells * m * theta_T doubles (prediction layout; device
 * pointer if on_device).  The prediction is also kept for a
 * following ridg_correct.  Returns RIDG_ENOCONV (after completing) if Newton hit its cap
 * in some region.  Synchronous when w_out is a host pointer.                            */
int ridg_predict(ridg_t* h, double* w_out, int on_device);

/* Correction (Sec. 2.3) from the last prediction; advances t by dt.  Stream-ordered.  */
int ridg_correct(ridg_t* h);

/* n >= 1 full steps (prediction + correction), enqueued on the handle's stream; the
 * sequence is captured once into a CUDA graph per (n, dt) and replayed.  Returns after
 * enqueueing; ridg_sync waits.                                                          */
int ridg_step(ridg_t* h, int n);

/* Wait for all work of the handle; reports a device-side status (ENOCONV / ETIMEOUT).  */
int ridg_sync(ridg_t* h);

/* ----- diagnostics -------------------------------------------------------------------- */

/* Problem sizes, time, step count, Newton statistics of the last prediction / ridg_step and
 * the current mass (Sec. 2.3).  Computing the mass waits for the handle's stream.          */
int ridg_info(ridg_t* h, ridg_info_t* info);

/* sum over cells of |T| Q_{e, r, 0} for each conserved variable r (mass[m]).            */
int ridg_mass(ridg_t* h, double* mass);

/* Relative L2 error of eq. l2relerror against the exact solution's projection onto
 * Q(M+1): x holds cells * m * (M+2)^d coefficients (same ordering rules).              */
int ridg_l2_error(ridg_t* h, const double* x, int on_device, double* err);

/* The same relative L2 error as ridg_l2_error for a state q (cells * m * (order+1)^dim) and
 * exact coefficients x (cells * m * (order+2)^dim), both already in device memory on the
 * current device, with no handle and no allocation of any kind.  The paper has no
 * counterpart: this entry point is for callers that cannot call cudaMalloc where they need
 * the diagnostic -- code whose device memory is owned by a pool or arena that must see
 * every allocation, and time-critical loops that cannot afford the device synchronisation
 * of cudaMalloc / cudaFree.  Its scratch is a fixed file-scope device array of 1 MiB (65536
 * pairs of partial sums, one pair per 256 cells), held by every GPU that loads the library
 * until the process exits; larger problems (more than 16,777,216 cells) are rejected with
 * RIDG_ETOOBIG before any work.  The first call on a device looks up the array's device
 * address and keeps it; after a cudaDeviceReset of that device the kept address is stale
 * and the entry point must not be called again in that process.  Work is issued on
 * `stream` (NULL = legacy default stream) and the call copies the result back and waits
 * for it, so `stream` must not be capturing a CUDA graph: a capturing stream (or the legacy
 * stream while another stream captures in global mode) is refused with RIDG_ESTATE before
 * any work.  Every call shares the array: calls that overlap on the GPU race.            */
int ridg_l2_error_noalloc(const double* q, const double* x, long long cells, int m, int dim,
                          int order, void* stream, double* err);

/* Failure-detection check (no GPU fault involved): launches a one-thread kernel whose bounded
 * mbarrier wait -- the helper every tensor-core kernel waits with -- waits on an arrival
 * that never comes, so the wait runs out of polls and the kernel reports it and returns.
 * Returns RIDG_ETIMEOUT when that happened (the expected outcome), RIDG_OK if the wait
 * completed (it cannot), RIDG_ENOMEM / RIDG_ECUDA on allocation / launch errors.  The
 * device context stays usable.  seconds (nullable) receives the wait's device time.  Work
 * is issued on `stream` (NULL = legacy default stream) and the call waits for it.          */
int ridg_check_bounded_wait(void* stream, double* seconds);

/* ----- tracing ---------------------------------------------------------------------------- */

typedef struct {
  double predict_ms;     /* average device time of the prediction kernel per step           */
  double correct_ms;     /* average device time of the correction kernel per step           */
  double step_ms;        /* average device time of one whole step                            */
  int launches_per_step; /* kernels launched per step                                        */
} ridg_profile_t;

/* Run n steps (the same arithmetic as ridg_step) as individual launches bracketed by CUDA
 * events on the handle's stream, wait, and report the average device time of each
 * kernel.  Advances the state and t like ridg_step.                                       */
int ridg_profile_step(ridg_t* h, int n, ridg_profile_t* out);

/* ----- autotuning ------------------------------------------------------------------------ */

/* Time the launch choices of the handle's kernels on its own current state and keep the
 * fastest (tile shapes and schedules per polynomial order).  Tuned now: for the 3D mixed
 * path the depth of the GEMM's operand ring (the slots that fit, up to 8) and the
 * correction's block size (64, 128, 256 threads); for a nonlinear
 * flux the persistent Newton grid (1, 2, 4 or 8 CTAs per 4 SMs: fewer CTAs keep more of
 * their block storage in L2).  Each candidate runs a few real steps (CUDA events around
 * each launch); the state, t and the step count are restored afterwards, and captured
 * graphs are dropped.  The choices go into the process-wide cache under keys naming the
 * kernel family, degree, slices / conserved variables and precision, which ridg_create and
 * ridg_batch_create read for every later handle; if cache_path is not NULL the whole cache
 * is also written there (one "key value" line each).  The cache is first loaded from the
 * file named by the environment variable RIDG_TUNE_CACHE when that is set.  Other
 * configurations have nothing to tune and return RIDG_OK at once.  Synchronous.          */
int ridg_autotune(ridg_t* h, const char* cache_path);

/* The handle's current launch choices (any pointer may be NULL): 3D GEMM ring cap (0 = as
 * many slots as fit), 3D correction block size, Newton grid in CTAs.                      */
int ridg_get_tuning(ridg_t* h, int* gemm3_slots, int* corr3_block, int* newton_grid);

/* Merge the "key value" lines of a cache file into the process-wide cache
 * (RIDG_EINVAL if it cannot be read).                                                      */
int ridg_tune_load(const char* cache_path);

/* The cached value of `key` (RIDG_EINVAL if none is recorded).                            */
int ridg_tune_lookup(const char* key, int* value);

/* ----- batched ensemble ---------------------------------------------------------------- */

typedef struct ridg_batch ridg_batch_t;

/* `count` independent problems (meshes[i], orders[i], the same flux kind) advanced
 * together; ridg_batch_step runs n steps of every instance in one graph, each instance
 * with its own dt.                                                                      */
int ridg_batch_create(int count, const ridg_mesh* meshes, const int* orders,
                      const ridg_flux* flux, double cfl, const ridg_options* opt,
                      ridg_batch_t** out);
void ridg_batch_destroy(ridg_batch_t* b);
/* Instance i of the batch as an ordinary handle (owned by the batch).                    */
ridg_t* ridg_batch_instance(ridg_batch_t* b, int i);
/* ridg_set_state / ridg_get_state of instance i (RIDG_EINVAL for an index out of range).  */
int ridg_batch_set_state(ridg_batch_t* b, int i, const double* q, int on_device);
int ridg_batch_get_state(ridg_batch_t* b, int i, double* q, int on_device);
int ridg_batch_step(ridg_batch_t* b, int n);
/* The batch's schedule for a nonlinear flux (1: the whole ensemble's Newton prediction in one
 * launch -- every degree's regions, highest degree first, each CTA moving to the next
 * degree's queue as one runs out -- and every instance's correction in one more launch;
 * 0: one Newton launch per degree and one correction per instance) and the kernel launches
 * of one step.  Burgers batches default to 1 unless the autotuner recorded otherwise.     */
int ridg_batch_schedule(ridg_batch_t* b, int* schedule, int* launches_per_step);
/* Time one step in each schedule from the instances' current states (restored afterwards,
 * graphs dropped) and keep the faster; the choice goes into the autotuner's cache (and to
 * cache_path if not NULL) for later batches of the same flux and precision.               */
int ridg_batch_autotune(ridg_batch_t* b, const char* cache_path);
int ridg_batch_sync(ridg_batch_t* b);

/* ----- a mesh sharded into slabs (domain decomposition, Sec. 5) ------------------------- */

typedef struct ridg_shard ridg_shard_t;

/* Partition a linear-advection mesh into `count` slabs along its slowest axis (x in 1D, y in
 * 2D, z in 3D), slab i an ordinary handle on device devices[i] (NULL: every slab on the
 * current device), with its own stream (opt->stream must be NULL).  Each slab's local mesh
 * is its layers plus, when the velocity along the axis is nonzero, the two layers upstream
 * of it (the halo: its first layer's correction reads the time mean of the layer below it,
 * whose prediction reads one more layer), periodic locally; the local wrap only reaches
 * halo cells, whose results are discarded, so every owned cell is computed exactly as in
 * the unsharded step.  Every slab needs at least 2 layers.  The paper's decomposition uses
 * two exchanges per step (the state, then the boundary predictions); with upwind face
 * values one exchange of a two-layer state halo from the upstream slab suffices.          */
int ridg_shard_create(const ridg_mesh* mesh, int order, const ridg_flux* flux, double cfl,
                      const ridg_options* opt, int count, const int* devices,
                      ridg_shard_t** out);
void ridg_shard_destroy(ridg_shard_t* s);
/* Slab i as an ordinary handle (owned by the shard): its info, mass, profile.             */
ridg_t* ridg_shard_slab(ridg_shard_t* s, int i);
/* The whole problem's state in the canonical layout (host memory, or device memory of the
 * current device if on_device), scattered to / gathered from the slabs.  Synchronous.      */
int ridg_shard_set_state(ridg_shard_t* s, const double* q, int on_device);
int ridg_shard_get_state(ridg_shard_t* s, double* q, int on_device);
/* n steps: per step every slab's halo is copied from its upstream neighbour (one contiguous
 * copy, peer-to-peer between devices), ordered by events after that neighbour's previous
 * step, then every slab runs its step graph once the copy that reads its own state is done.
 * Returns after enqueueing; ridg_shard_sync waits (and reports a device-side status).     */
int ridg_shard_step(ridg_shard_t* s, int n);
int ridg_shard_sync(ridg_shard_t* s);

/* ----- errors ------------------------------------------------------------------------- */
const char* ridg_strerror(int status);
const char* ridg_last_error(const ridg_t* h);

#ifdef __cplusplus
}
#endif
#endif /* RIDG_H_ */
