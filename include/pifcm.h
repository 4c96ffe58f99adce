/*
 * pifcm.h - C ABI of the GB300 (sm_103a) implementation of the 3DPIFCM hot path.
 *
 * 3DPIFCM (Agranonik, Herman, Last, "Parallel 3DPIFCM Algorithm for Noisy Brain
 * MRI Images", arXiv 2002.01981) is fuzzy C-means whose distance carries two
 * neighbourhood terms weighted by (lambda, xi) (Eqs 1-10), with (lambda, xi)
 * chosen by a particle swarm whose fitness is the objective J_m (Algorithm 1).
 * This library runs the whole path on one GPU: min-max normalisation
 * (Algorithm 2 step 1), the FCM start (Algorithm 1 step 2), the batched fitness
 * evaluation of all particles (Algorithm 1 step 4: one IFCM run per particle),
 * the swarm update (steps 5-8) and the final IFCM run at the best particle
 * (step 11).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Volumes are float32 arrays [nz][ny][pitch_x], x fastest; elements with
 *   x >= nx are padding and are never read.  A 2D image is nz = 1.  pitch_x
 *   must be >= nx and a multiple of 4 (16-byte rows); base pointers must be
 *   16-byte aligned.
 * - Memberships are float32 arrays [c][nz][ny][pitch_x] (one plane per
 *   cluster); padding elements of outputs are unspecified.
 * - "device" pointers are CUDA device memory owned by the caller; "host"
 *   pointers are ordinary host memory owned by the caller.  The library does
 *   not allocate: its scratch is the caller's workspace `ws` of at least the
 *   size the matching *_workspace_bytes() call returns (256-byte aligned).
 *   The one exception is ifcm_fit_noalloc, whose scratch is a static 64 MiB
 *   device array of the library (see there).
 * - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are
 *   stream-ordered and return without synchronising, except the *_host entry
 *   points, which synchronise the stream before returning.
 * - Errors: every call returns an ifcm_status and never throws or aborts.
 *   IFCM_ERR_INVALID is returned for bad arguments before anything is
 *   launched.  Conditions found on the device (NaN/Inf or constant input
 *   volume, a bounded wait that ran out) are recorded in a device status word
 *   inside the workspace; the *_host calls and ifcm_device_status() report it.
 *   ifcm_last_error() holds a thread-local message for the last failure.
 */
#ifndef PIFCM_H
#define PIFCM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  IFCM_OK = 0,
  IFCM_ERR_INVALID = 1,      /* bad argument, shape, parameter or input volume */
  IFCM_ERR_NOMEM = 2,        /* workspace smaller than *_workspace_bytes()     */
  IFCM_ERR_CUDA = 3,         /* a CUDA runtime/driver call failed              */
  IFCM_ERR_TIMEOUT = 4,      /* a bounded device-side wait ran out             */
  IFCM_ERR_BOUNDS = 5,       /* a checked index fell outside its buffer        */
  IFCM_ERR_UNSUPPORTED = 6   /* valid per the paper but not built (e.g. V > 1) */
} ifcm_status;

/* Volume geometry.  nz = 1 selects the 2D 8-neighbourhood (Eq 9, L = 3). */
typedef struct {
  int32_t nx, ny, nz;
  int32_t pitch_x;           /* elements per row, >= nx, multiple of 4 */
} ifcm_shape;

/* Method parameters (Algorithm 1 / Algorithm 2 inputs). */
typedef struct {
  int32_t c;                 /* clusters, 2..8                                   */
  double m;                  /* fuzzifier m > 1 (Eqs 1-3); m = 2 has a fast path  */
  int32_t V;                 /* shells of Eq 10; only V = 1 (W_1 = 1) is built    */
  double h;                  /* decay of Eq 10 (unused for V = 1)                 */
  int32_t max_iter;          /* IFCM iterations per run, >= 1                     */
  double eps_u;              /* stop when max_ij |u' - u| < eps_u                 */
  double dist_floor;         /* lower bound of d^2 (reading R2), e.g. 1e-12       */
  int32_t u_dtype;           /* IFCM_U_FP32 (0) or IFCM_U_BF16 (1): see below     */
  int32_t reduce;            /* IFCM_REDUCE_FP64 (0) or IFCM_REDUCE_COMP32 (1)    */
} ifcm_params;

/* Storage of the memberships between the iterations of the batched runs
 * (ifcm_fit, pso_fitness_batch, pso_fitness_multi*, pifcm3d).  The paper
 * fixes no precision.  IFCM_U_BF16 stores U^t as bfloat16 (rounded to nearest
 * even once per iteration) while every arithmetic step stays FP32; it halves
 * the membership traffic.  max|du| of the stop rule compares the stored
 * values.  Inputs (u_init, u0) and outputs (u_out) stay FP32 arrays either
 * way.  The plain form (ifcm_fit_plain) and the FCM start always use FP32. */
#define IFCM_U_FP32 0
#define IFCM_U_BF16 1
/* Precision of the centre / objective sums above the warp level (Eqs 1, 3):
 * IFCM_REDUCE_FP64 sums warp partials and tile records in FP64;
 * IFCM_REDUCE_COMP32 sums them in FP32 with Neumaier compensation and takes
 * Eq 3 in FP32.  Within a thread and a warp the sums are FP32 either way. */
#define IFCM_REDUCE_FP64 0
#define IFCM_REDUCE_COMP32 1

/* Swarm state (Algorithm 1 steps 3-8).  All arrays are device memory owned by
 * the caller: x, v, pbest_x hold P*2 doubles (lambda, xi per particle),
 * pbest_f holds P doubles, gen one int32 (the generation counter that keys
 * the Philox draws). */
typedef struct {
  int32_t P;                 /* particles, 1..1024                              */
  int32_t radius;            /* ring radius of the topological neighbours, >= 0 */
  double vmax;               /* velocity clamp, > 0                              */
  uint64_t seed;             /* Philox4x32-10 key                               */
  double* x;
  double* v;
  double* pbest_x;
  double* pbest_f;
  int32_t* gen;
} pso_state;

/* Whole-run options of pifcm3d (Algorithm 1). */
typedef struct {
  int32_t P;                 /* particles                                         */
  int32_t generations;       /* swarm generations (fixed count, reading R9)       */
  int32_t radius;            /* ring radius                                       */
  double vmax;               /* velocity clamp                                    */
  uint64_t seed;             /* Philox key                                        */
  int32_t init_max_iter;     /* iterations of the FCM start (Algorithm 1 step 2)  */
  int32_t slice_z;           /* -1: whole volume; else segment slice z as 2D (Algorithm 1 step 1) */
  int32_t fitness_mode;      /* PIFCM_FITNESS_RESTART or PIFCM_FITNESS_ONESTEP     */
} pifcm_options;

/* What one fitness evaluation (Algorithm 1 step 4) is.
 * PIFCM_FITNESS_RESTART (reading R5): an IFCM run from the shared FCM start
 *   until max|du| < eps_u or max_iter iterations; fitness = its last J.
 * PIFCM_FITNESS_ONESTEP (Algorithm 2 steps 6-11 read literally): every
 *   particle keeps its own (U, C), starting from the FCM start, and each
 *   generation advances it by one IFCM iteration at the particle's current
 *   (lambda, xi); fitness = that iteration's J.  max_iter and eps_u then
 *   apply only to the final run (Algorithm 1 step 11). */
#define PIFCM_FITNESS_RESTART 0
#define PIFCM_FITNESS_ONESTEP 1

/* Result block written by pifcm3d (device or host copy). */
typedef struct {
  double centres[8];         /* C of the final IFCM run (first c used)            */
  double lambda, xi;         /* best particle's position                          */
  double J;                  /* objective of the final run's last iteration       */
  double best_fitness;       /* lowest personal-best fitness of the swarm         */
  int64_t updates;           /* voxel x particle x iteration updates executed     */
  int32_t iters_final;       /* iterations of the final run                       */
  int32_t iters_init;        /* iterations of the FCM start                       */
  int32_t status;            /* device status word (an ifcm_status)              */
  int32_t best_particle;
} pifcm_result;

const char* ifcm_status_string(ifcm_status s);
const char* ifcm_last_error(void);

/* Device status word recorded in `ws` by earlier calls (synchronises `stream`). */
ifcm_status ifcm_device_status(const void* ws, void* stream);

/* ---------------------------------------------------------------------------
 * Algorithm 2 step 1: x <- (x - min) / (max - min) over the whole volume.
 * vol: device, read; x_out: device, written (may equal vol).  A NaN/Inf or a
 * constant volume sets IFCM_ERR_INVALID in the device status word and leaves
 * x_out unspecified.
 */
size_t ifcm_normalize_workspace_bytes(ifcm_shape shape);
ifcm_status ifcm_normalize(const float* vol, float* x_out, ifcm_shape shape,
                           void* ws, size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------------------
 * One IFCM run (Eqs 1-10; Algorithm 1 steps 2 and 11).
 * Iteration t maps (U^t, C^t) to U^{t+1} (Eq 2 with the modified distance of
 * Eq 4, whose H and F come from U^t by Eqs 5-9), J^t (Eq 1 with that
 * distance) and C^{t+1} (Eq 3); the run stops when max|U^{t+1} - U^t| <
 * eps_u or after max_iter iterations.
 * x:       device, normalised volume [nz][ny][pitch_x].
 * lam_xi:  device, 2 doubles (lambda, xi), read when the run starts.
 * u_init:  device [c][nz][ny][pitch_x], or NULL for u_ij = 1/c.
 * c_init:  device, c doubles, or NULL for c_j = (j + 1/2)/c.
 * u_out:   device [c][nz][ny][pitch_x] (may be NULL): final memberships.
 * c_out:   device, c doubles (may be NULL): final centres.
 * J_out:   device, 1 double (may be NULL): J of the last iteration.
 * iters_out: device, 1 int32 (may be NULL): iterations executed.
 * With lambda = xi = 0 this is plain FCM, the start of Algorithm 1 step 2.
 */
size_t ifcm_fit_workspace_bytes(ifcm_shape shape, const ifcm_params* p);
ifcm_status ifcm_fit(const float* x, ifcm_shape shape, const ifcm_params* p,
                     const double* lam_xi, const float* u_init, const double* c_init,
                     float* u_out, double* c_out, double* J_out, int32_t* iters_out,
                     void* ws, size_t ws_bytes, void* stream);

/* The same run in the shape of the paper's Algorithm 2 (one particle, one
 * thread per voxel reading its neighbours from global memory, the host
 * checking convergence after every iteration).  Kept as the plain form that
 * the batched path is measured against.  Synchronises `stream` each
 * iteration; lambda and xi are host values; outputs are as for ifcm_fit. */
ifcm_status ifcm_fit_plain(const float* x, ifcm_shape shape, const ifcm_params* p,
                           double lambda, double xi, const float* u_init,
                           const double* c_init, float* u_out, double* c_out,
                           double* J_out, int32_t* iters_out,
                           void* ws, size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------------------
 * Algorithm 1 step 4 for a whole swarm: fitness_p = J of an IFCM run from the
 * shared start (u0, c0) at (lambda_p, xi_p) = lam_xi[2p], lam_xi[2p+1]
 * (reading R5), all P runs in one batch of launches.
 * lam_xi: device, P*2 doubles.  u0: device [c][nz][ny][pitch_x].  c0: device,
 * c doubles.  fitness: device, P doubles.  iters: device, P int32 (may be
 * NULL).  c_out: device, P*c doubles (may be NULL).
 */
size_t pso_fitness_batch_workspace_bytes(ifcm_shape shape, const ifcm_params* p, int32_t P);
ifcm_status pso_fitness_batch(const float* x, ifcm_shape shape, const ifcm_params* p,
                              const double* lam_xi, int32_t P,
                              const float* u0, const double* c0,
                              double* fitness, int32_t* iters, double* c_out,
                              void* ws, size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------------------
 * Work decomposition of the batched stencil launches (no arithmetic change
 * beyond the order of the FP64 partial sums).  A launch is cut into work
 * items of np particles (1, or 2 for c <= 5) x a 32-column tile x a z-chunk
 * of tz planes (in a 2D image: a run of tz tiles down the image, the tiles
 * taking the place of the planes).  Mode 0 (default): a built-in rule picks
 * the deepest chunks that still give every CTA four items.  Mode 1: the first
 * run of each (membership type, c, volume extents, particle counts) times the
 * candidate plans on its own buffers (a host synchronisation; never on a
 * stream being captured into a graph) and the fastest is cached for the
 * process.
 * Thread-safe.
 */
void ifcm_autotune_enable(int32_t mode);
void ifcm_autotune_reset(void);
/* Every later launch uses np particles per item (where c allows it: np = 2
 * only for c <= 5, else the usual choice) and `chunks` z-chunks per tile
 * (clamped so that chunks keep >= 8 planes).  np = 0 lifts it.  For tests
 * and experiments.  IFCM_ERR_INVALID for np outside 0..2 or chunks < 1. */
ifcm_status ifcm_stencil_force_plan(int32_t np, int32_t chunks);
/* Whole runs of small volumes in one launch (Alg 1 step 4 with Alg 2's loop
 * of steps 6-10 on the device).  When every volume of a batch fits one CTA's
 * shared memory -- x and two FP32 membership fields, (1 + 2c) x 4 bytes per
 * voxel, at most 225 KB (6400 voxels at c = 4, 3388 at c = 8) -- and the
 * batch stores FP32 memberships with V = 1, it runs as one launch of one CTA
 * per particle: the CTA keeps x, U^t and U^{t+1} in shared memory, sums
 * Eqs 1 and 3 (FP32 within a warp, FP64 or compensated FP32 across warps, as
 * `reduce` says) and takes the stop rule itself, instead of two launches per
 * iteration.  pifcm3d's FCM start (Alg 1 step 2) runs the same way.  The
 * arithmetic per voxel is the plain kernel's; results agree with the stencil
 * form up to FP32 rounding.  Mode 1 (default): on; 0: off, every batch takes
 * the stencil kernels.  A forced plan (ifcm_stencil_force_plan) also keeps
 * batches on the stencil kernels.  Process-wide. */
void ifcm_resident_enable(int32_t mode);
/* The plan a one-volume batch of P particles would use: *np, *tz.  Returns 1
 * when it comes from the tuning cache, 0 from the rule, -1 on bad input. */
int32_t ifcm_stencil_plan(ifcm_shape shape, int32_t c, int32_t P, int32_t* np, int32_t* tz);

/* ---------------------------------------------------------------------------
 * Algorithm 1 step 4 for many swarms at once: each volume brings its own
 * particles, start (u0, c0) and cluster count, and every (volume, particle)
 * fitness is evaluated in the same batched launches: volumes of the same c
 * share each stencil launch (up to 64 volumes and 4096 particles per launch).
 * Volumes are taken in order, grouped by c, and packed into waves that fit
 * ws_bytes; a wave runs to completion before the next reuses the workspace.
 * Each particle computes the same IFCM run as in pso_fitness_batch on its
 * volume alone; results agree to the order of the partial sums, which
 * depends on how the launch cuts the volume into work items (z-chunks,
 * particles or clusters per packed lane) and so on the whole batch.
 * vols: HOST array of n descriptors (pointers inside are device memory).
 * p: m, max_iter, eps_u, dist_floor and V are shared; p->c is ignored.
 */
typedef struct {
  const float* x;            /* device, normalised volume [nz][ny][pitch_x]   */
  ifcm_shape shape;
  int32_t c;                 /* clusters of this volume, 2..8                 */
  int32_t P;                 /* particles, >= 1                               */
  const double* lam_xi;      /* device, P*2 (lambda, xi)                      */
  const float* u0;           /* device [c][nz][ny][pitch_x]: shared start     */
  const double* c0;          /* device, c: shared start                       */
  double* fitness;           /* device, P                                     */
  int32_t* iters;            /* device, P (may be NULL)                       */
} ifcm_batch_volume;

/* Workspace to run every volume of a c in one wave (the largest such group). */
size_t pso_fitness_multi_workspace_bytes(const ifcm_batch_volume* vols, int32_t n,
                                         const ifcm_params* p);
/* Smallest workspace that still runs (one volume per wave). */
size_t pso_fitness_multi_min_workspace_bytes(const ifcm_batch_volume* vols, int32_t n,
                                             const ifcm_params* p);
/* Waves (batched launch sequences) a call with ws_bytes of workspace runs;
 * -1 on bad input or a workspace below the minimum. */
int32_t pso_fitness_multi_waves(const ifcm_batch_volume* vols, int32_t n, const ifcm_params* p,
                                size_t ws_bytes);
ifcm_status pso_fitness_multi(const ifcm_batch_volume* vols, int32_t n, const ifcm_params* p,
                              void* ws, size_t ws_bytes, void* stream);

/* The same call captured once into a CUDA graph: every replay re-runs it with
 * the values then in the buffers (the swarm's new lam_xi each generation)
 * and the same pointers, which must stay valid while the graph lives.  The
 * plan of each launch is fixed at capture (the cache, else the rule; no
 * timing).  Replays on one workspace must not overlap.  Checks as for
 * pso_fitness_multi; IFCM_ERR_CUDA when capture or instantiation fails. */
typedef struct ifcm_graph_t* ifcm_graph;
ifcm_status pso_fitness_multi_graph(const ifcm_batch_volume* vols, int32_t n,
                                    const ifcm_params* p, void* ws, size_t ws_bytes,
                                    ifcm_graph* out);
ifcm_status ifcm_graph_launch(ifcm_graph g, void* stream);
void ifcm_graph_destroy(ifcm_graph g);

/* ---------------------------------------------------------------------------
 * Algorithm 1 step 3: x ~ U[0,1)^2, v ~ U[-vmax, vmax)^2, pbest_x = x,
 * pbest_f = +inf, gen = 0.  Draws are Philox4x32-10 keyed by seed with
 * counter (generation, particle, dimension, stream).
 */
ifcm_status pso_init(const pso_state* s, void* stream);

/* Algorithm 1 steps 5-8 given fitness (device, P doubles) of the current
 * positions: strict personal-best update, best of the ring neighbours (ties to
 * the lowest index), v <- v + p1 (pbest - x) + p2 (lbest - x) clamped to
 * +-vmax, x <- clip(x + v, 0, 1), gen += 1.  Every operation is one rounded
 * FP64 operation (no fused multiply-add), so two runs fed the same fitness
 * values produce bit-identical swarms. */
ifcm_status pso_step(const pso_state* s, const double* fitness, void* stream);

/* ---------------------------------------------------------------------------
 * Algorithm 1 end to end on the device: normalise vol (device, unchanged),
 * optional slice, FCM start, `generations` x (fitness batch + swarm step),
 * final IFCM run at the best personal best.  u_out: device
 * [c][nz'][ny][pitch_x] (nz' = 1 with a slice; may be NULL).  result: device
 * pifcm_result.
 */
size_t pifcm3d_workspace_bytes(ifcm_shape shape, const ifcm_params* p, const pifcm_options* o);
ifcm_status pifcm3d(const float* vol, ifcm_shape shape, const ifcm_params* p,
                    const pifcm_options* o, float* u_out, pifcm_result* result,
                    void* ws, size_t ws_bytes, void* stream);

/* The same run captured once into a CUDA graph (the ifcm_graph type of
 * pso_fitness_multi_graph).  pifcm3d never waits on the host, so its ~3800
 * launches (181^3, 20 particles x 30 generations) become one graph; every
 * ifcm_graph_launch re-runs Algorithm 1 on what vol then holds, with the
 * same pointers, which must stay valid while the graph lives.  The stencil
 * plans are fixed at capture (the tuning cache, else the built-in rule).
 * Replays on one workspace must not overlap.  Checks as for pifcm3d;
 * IFCM_ERR_CUDA when capture or instantiation fails.  Replaying saves the
 * launch latency that bounds small images (about 8 ms of a 31 ms run at
 * 32 x 32). */
ifcm_status pifcm3d_graph(const float* vol, ifcm_shape shape, const ifcm_params* p,
                          const pifcm_options* o, float* u_out, pifcm_result* result, void* ws,
                          size_t ws_bytes, ifcm_graph* out);

/* The same with HOST input and outputs: copies vol_host in, runs pifcm3d and
 * copies the memberships and the result block back, then synchronises the
 * stream.  The workspace also holds the device copies of the volume, the
 * memberships and the result (size from pifcm3d_host_workspace_bytes()).
 * vol_host / u_out_host should be page-locked for full copy speed.
 * u_out_host may be NULL.  Returns the device status word's error, if any. */
size_t pifcm3d_host_workspace_bytes(ifcm_shape shape, const ifcm_params* p,
                                    const pifcm_options* o);
ifcm_status pifcm3d_host(const float* vol_host, ifcm_shape shape, const ifcm_params* p,
                         const pifcm_options* o, float* u_out_host,
                         pifcm_result* result_host,
                         void* ws, size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------------------
 * Derivative of the fitness with respect to (lambda, xi) (Eqs 1-8 by the chain
 * rule; the paper has no gradient).  The differentiated function is
 * L(lambda, xi) = J^{K-1}: the objective of the last of K IFCM iterations from
 * the fixed start (u0, c0), with no stop rule (the fitness of Algorithm 1 step
 * 4 with eps_u = 0 and max_iter = K).  The forward pass keeps every U^t
 * (checkpoints, K x c planes of the workspace) and a trace of C^{t+1},
 * sum_i u^m and J^t.  The reverse pass runs back through Eq 3, Eq 1, Eq 2,
 * Eq 4 (a clamp of reading R2 that is active passes no derivative) and the
 * transposed neighbourhood stencils of Eqs 5 and 7.
 * x: device, normalised volume.  lam_xi: device, 2 doubles.  u0: device
 * [c][nz][ny][pitch_x].  c0: device, c doubles (both required).  J_out:
 * device, 1 double (may be NULL).  grad_out: device, 2 doubles (dJ/dlambda,
 * dJ/dxi).  p->eps_u and p->max_iter are ignored (K iterations).  FP32
 * memberships only: IFCM_ERR_UNSUPPORTED for u_dtype = IFCM_U_BF16.
 */
size_t ifcm_grad_workspace_bytes(ifcm_shape shape, const ifcm_params* p, int32_t K);
ifcm_status ifcm_grad(const float* x, ifcm_shape shape, const ifcm_params* p, int32_t K,
                      const double* lam_xi, const float* u0, const double* c0, double* J_out,
                      double* grad_out, void* ws, size_t ws_bytes, void* stream);

/* Gradient polishing of a particle (e.g. the swarm's best): `steps` projected
 * descent steps of fixed length on [0,1]^2,
 *   (lambda, xi) <- clip((lambda, xi) - alpha_k g / |g|, 0, 1),
 *   alpha_k = step0 * decay^k,
 * with g = ifcm_grad at the current point.  Then J is evaluated at the last
 * point.  lam_xi (device, 2 doubles) is read as the start and overwritten
 * with the point of lowest J^{K-1} seen; J_out (device, 1 double, may be NULL)
 * receives that J.  Workspace as for ifcm_grad.  Stream-ordered: no host
 * synchronisation. */
ifcm_status ifcm_polish(const float* x, ifcm_shape shape, const ifcm_params* p, int32_t K,
                        int32_t steps, double step0, double decay, double* lam_xi,
                        const float* u0, const double* c0, double* J_out, void* ws,
                        size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------------------
 * ifcm_fit without a caller workspace.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory when they
 * run a segmentation (a graph being recorded under global capture mode, a
 * plugin whose host framework owns every allocation and hands it only its
 * input and output pointers, a loop that must not take the allocator's
 * implicit synchronisation).  Arguments and results are those of ifcm_fit;
 * the scratch is a static 64 MiB device array of the library.  The CUDA
 * runtime places it in a GPU's memory when it loads the library's module on
 * that GPU -- with lazy module loading (the default), at the first call of
 * this entry point there -- and it stays until the process exits; that first
 * call can therefore fail with IFCM_ERR_CUDA when the GPU has no room for it.
 * Calls whose ifcm_fit workspace would exceed 64 MiB (about 1.36 million
 * voxels at c = 4, e.g. 111^3) return IFCM_ERR_NOMEM with a message naming
 * both sizes.  The first call on each device looks up the array's device
 * address and keeps it for the process (a cudaDeviceReset makes it stale);
 * make that first call before any stream capture.  Every call on a device
 * shares the one array: calls that overlap on the GPU (other streams, other
 * threads) race and corrupt each other's results, so serialise them.  The
 * entry point calls no allocating routine; device-side failures of a call
 * (a bounded wait that ran out) go to the status word in the array, which
 * ifcm_fit_noalloc_status reports.
 */
ifcm_status ifcm_fit_noalloc(const float* x, ifcm_shape shape, const ifcm_params* p,
                             const double* lam_xi, const float* u_init, const double* c_init,
                             float* u_out, double* c_out, double* J_out, int32_t* iters_out,
                             void* stream);
/* The device status of the last ifcm_fit_noalloc call on the current device,
 * as ifcm_device_status reports it for a workspace: synchronises `stream`,
 * returns IFCM_OK or the condition the kernels recorded (IFCM_ERR_TIMEOUT for
 * a bounded wait that ran out).  The paper has no counterpart. */
ifcm_status ifcm_fit_noalloc_status(void* stream);

/* ---------------------------------------------------------------------------
 * Profiling counters (host side, per process): when enabled, the library
 * records CUDA events around every launch of the stencil-iteration kernel
 * and the updates it was launched for; ifcm_profile_read() synchronises the
 * recorded events and returns the summed kernel milliseconds, launches and
 * the voxel x particle updates processed (from the device counters).
 */
void ifcm_profile_enable(int32_t on);
ifcm_status ifcm_profile_read(double* kernel_ms, int64_t* launches);
/* The same for one kind of kernel: IFCM_PROF_STENCIL (what ifcm_profile_read
 * returns), IFCM_PROF_ADJOINT_POINT or IFCM_PROF_ADJOINT_GATHER (the two
 * kernels of each reverse iteration of ifcm_grad).  Reading a kind clears its
 * records.  IFCM_ERR_INVALID for another kind. */
#define IFCM_PROF_STENCIL 0
#define IFCM_PROF_ADJOINT_POINT 1
#define IFCM_PROF_ADJOINT_GATHER 2
/* IFCM_PROF_STENCIL3D: the stencil iterations of batches of 3D volumes that
 * run the float2-pair plane step alone (every iteration after the first of
 * an FP32 batch of two or more particles with m = 2, c <= 5); they are
 * counted in IFCM_PROF_STENCIL as well. */
#define IFCM_PROF_STENCIL3D 3
ifcm_status ifcm_profile_read_kind(int32_t kind, double* kernel_ms, int64_t* launches);

/* ---------------------------------------------------------------------------
 * Failure detection.  Every wait of a kernel on the arrival of its
 * shared-memory tiles (an mbarrier phase) is bounded: after ns nanoseconds
 * of the GPU's global timer without the phase completing, the kernel records
 * IFCM_ERR_TIMEOUT in the workspace's status word (ifcm_device_status), stops
 * issuing copies, waits (bounded, about a second) for the copies it already
 * issued, and returns; later launches of the call see the status and the
 * host entry points return normally.  The setting is process-wide and read
 * when a call builds its launches; 0 (the default) bounds each wait at about
 * one second.  A bound below 1000 ns gives up at the first unsuccessful
 * non-blocking test of a phase, which makes waits run out on purpose (for
 * tests of this path); they leave the GPU context usable. */
void ifcm_set_wait_limit_ns(uint64_t ns);

#ifdef __cplusplus
}
#endif
#endif /* PIFCM_H */
