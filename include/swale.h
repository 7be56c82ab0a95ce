/*
 * swale.h -- C ABI of the GB300 (sm_103a) solver for the one-dimensional well-balanced
 * finite-volume ALE-WENO hybrid scheme for the shallow water equations with bottom
 * topography of Zhang, Xia & Xu, "Structure-preserving finite volume arbitrary
 * Lagrangian-Eulerian WENO schemes for the shallow water equations" (arXiv 2208.06588).
 *
 * The calls follow the paper's problem statement: a mesh of N cells with nodes x_{j+1/2}
 * (Sec. 2.1), cell averages of the depth h, the discharge hu and the bottom b (Sec. 3.1,
 * Sec. 3.3), the gravitational constant g, the CFL number and the final time t_end
 * (Sec. 5). One step is the modified third-order SSP-RK method with the width recursion
 * (Eq. RK32D, Eq. Jacobi2D); each stage evaluates the well-balanced semi-discrete scheme
 * with hydrostatic reconstruction (Eq. hydro2D-HH2D) and the bottom scheme (Eq. bottomrk).
 *
 * Conventions
 *  - All floating-point data are IEEE double (FP64), contiguous, no padding.
 *  - Pointer arguments may be host or device memory (detected per pointer with
 *    cudaPointerGetAttributes); device pointers are used on the context's stream.
 *  - The caller owns every buffer it passes; the library copies inputs in and results out
 *    and keeps no reference to caller memory after a call returns.
 *  - Every call returns a swale_status. Nothing aborts, throws or traps; on an error the
 *    message is available from swale_last_error(ctx).
 *  - A context is not thread-safe; use one context per host thread / stream.
 */
#ifndef SWALE_H
#define SWALE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct swale_ctx swale_ctx;

typedef enum {
  SWALE_OK = 0,
  SWALE_EINVAL = -1,      /* invalid argument or state (message says which) */
  SWALE_ENOMEM = -2,      /* device allocation failed */
  SWALE_ECUDA = -3,       /* a CUDA runtime call failed */
  SWALE_EMESH = -4,       /* a cell width became <= 0 (mesh assumption A1 of Sec. 2.1) */
  SWALE_ENEGDEPTH = -5,   /* reserved: negative depth is reported as a warning bit */
  SWALE_ENONFINITE = -6,  /* a non-finite value appeared, or no finite dt (SWALE_BIT_NODT) */
  SWALE_ETIMEOUT = -7,    /* a bounded device wait gave up (SWALE_BIT_TIMEOUT); the step was not
                             committed (the state is that of the last good step) */
  SWALE_EWEIGHT = -8      /* a linear weight d_r <= 0 (Sec. 2.2: needs the Shi-Hu-Shu split) */
} swale_status;

/* Bits of the device status word returned by swale_get_status. */
#define SWALE_BIT_EWEIGHT 1u    /* linear weight <= 0 met in a stage */
#define SWALE_BIT_NEGDEPTH 2u   /* a cell-average depth below -eps_pp entered a stage (warning) */
#define SWALE_BIT_NONFINITE 4u  /* non-finite value */
#define SWALE_BIT_EMESH 8u      /* non-positive width */
#define SWALE_BIT_NODT 16u      /* zero wave speed, static mesh and t_end = 0: the CFL dt is not
                                   finite; no step is taken (the state is unchanged) */
#define SWALE_BIT_TIMEOUT 32u   /* a kernel's bounded wait for its bulk (TMA) copies gave up; the
                                   kernel returned early and the step was not committed */

typedef enum { SWALE_BC_PERIODIC = 0, SWALE_BC_TRANSMISSIVE = 1, SWALE_BC_REFLECTIVE = 2 } swale_bc;

typedef enum {
  SWALE_MESH_STATIC = 0,      /* w = 0 */
  SWALE_MESH_PROFILE = 1,     /* x_k(t) = x_k(0) + P_k sin(2 pi t / mesh_T); w_k is the secant
                                 speed over each step (Eq. w1D) */
  SWALE_MESH_FLUID_GAUSS = 2, /* w_k = Gaussian-smoothed (sigma = gauss_sigma cells, +-gauss_half
                                 nodes, renormalised) mean of the adjacent cell velocities;
                                 end nodes fixed */
  SWALE_MESH_LINEAR = 3       /* x_k(t) = x_k(0) + P_k t: constant node velocities w_k = P_k
                                 (Eq. velocity, Eq. meshspecial of Sec. 5.1, the graded mesh of
                                 the big-pulse example); the profile array holds the P_k */
} swale_mesh;

typedef enum {
  SWALE_SCHEME_HYDROSTATIC = 0, /* well-balanced scheme with hydrostatic reconstruction (Sec. 4.1):
                                   shared-indicator reconstruction of (eta, hu, b), modified flux */
  SWALE_SCHEME_NONWB = 1,       /* the ALE-WENO scheme of Eq. se2D / s2D: local characteristic
                                   reconstruction of (eta, hu), plain Lax-Friedrichs flux (not
                                   well-balanced; the paper's baseline) */
  SWALE_SCHEME_SPECIAL = 2      /* well-balanced scheme with the special source term (Sec. 4.2,
                                   Eq. special2D): the hydrostatic scheme's reconstruction, plain
                                   LF flux, source split as in Eq. source2 with a Gauss-Lobatto
                                   sum at reconstructed interior points (negative linear weights
                                   there treated by the split of Shi, Hu & Shu) */
} swale_scheme;

/* Scheme and run constants. Defaults used in the paper: g = 9.812, cfl = 0.6 (0.08 for
 * wet/dry problems), eps_weno = 1e-6 (Step 2 of Sec. 2.2), eps_pp = 1e-11 (Eq. modifiedhjn). */
typedef struct {
  double g;            /* gravitational constant */
  double cfl;          /* dt = cfl * min_j J_j / alpha_1 */
  double eps_weno;     /* epsilon of the smoothness detector and of the WENO-Z weights */
  double eps_pp;       /* floor of the bound-preserving limiter */
  double h_dry;        /* edge depths <= h_dry carry zero velocity (default 1e-6) */
  double mesh_T;       /* period of the prescribed motion (SWALE_MESH_PROFILE) */
  double gauss_sigma;  /* filter width in cells (SWALE_MESH_FLUID_GAUSS) */
  double t_end;        /* > 0: the last step is clipped to t_end and stepping stops there */
  double dt_fixed;     /* > 0: every step uses this dt instead of the CFL formula */
  int32_t bc;          /* swale_bc */
  int32_t mesh;        /* swale_mesh */
  int32_t gauss_half;  /* filter truncation half-width in nodes, <= 64 */
  int32_t beta_dx_global; /* 1: Delta x in the indicators is max_j J_j (Step 1); 0: local J_j */
  int32_t scheme;      /* swale_scheme */
  int32_t alpha_bound; /* 0 (default): the viscosity alpha of Eq. alpha2D as written, the largest
                          |u - w| + sqrt(g h) over the edge states, wherever the node velocities
                          w are known when the stage runs (every stage of the static, fluid-driven
                          and linear motions; stages 2 and 3 of the profile motion), and in stage
                          1 of the profile motion, whose secant w depends on dt, the bound
                          max |u| + sqrt(g h) + W with W >= max |w|; 1: that bound in every stage */
  int32_t limit_hu;    /* 0 (default): the bound-preserving limiter scales the depth's edge values
                          only, as Eq. modifiedhjn is written; 1: it scales the discharge's edge
                          values about their mean with the same theta as well */
} swale_config;

/* Creates a context bound to a CUDA stream (cudaStream_t; NULL = legacy default stream).
 * Checks the configuration; allocates nothing on the device yet.
 * Errors: SWALE_EINVAL (bad config, no CUDA device). */
swale_status swale_create(swale_ctx** out, const swale_config* cfg, void* cuda_stream);

/* Sets the problem (Sec. 2.1 mesh, Sec. 3 cell averages) and allocates the device state.
 *   N        number of cells, N >= 5
 *   x_nodes  N+1 node coordinates, strictly increasing
 *   q0       N cell averages of the depth h (q0_is_eta = 0) or of the surface eta = h + b
 *            (q0_is_eta = 1; lets a lake at rest be given exactly as eta = const)
 *   hu, b    N cell averages of the discharge and of the bottom
 *   profile  N+1 node amplitudes P_k of SWALE_MESH_PROFILE motion, or node velocities P_k of
 *            SWALE_MESH_LINEAR motion (ignored otherwise; may be NULL then)
 * The time is reset to 0. Errors: SWALE_EINVAL (sizes, non-finite data, negative depth,
 * non-increasing nodes), SWALE_ENOMEM, SWALE_ECUDA. */
swale_status swale_set_problem(swale_ctx* ctx, int64_t N, const double* x_nodes, const double* q0,
                               const double* hu, const double* b, const double* profile, int32_t q0_is_eta);

/* Sets a batch of B independent instances (offsets[B+1] cells, offsets[0] = 0, each instance
 * N_i = offsets[i+1] - offsets[i] >= 5 cells, total < 2^31). Arrays are concatenated over the
 * instances: cells of instance i at [offsets[i], offsets[i+1]), its N_i + 1 nodes (and profile
 * values) at [offsets[i] + i, offsets[i+1] + i + 1). cfl: B per-instance CFL numbers (NULL: the
 * configuration's). Every instance advances with its own dt (its own alpha, Eq. alpha2D) in the
 * same launches; the configuration (g, eps, boundary condition, mesh kind, T) is shared.
 * Errors as swale_set_problem. */
swale_status swale_batch_set_problem(swale_ctx* ctx, int64_t B, const int64_t* offsets, const double* x_nodes,
                                     const double* q0, const double* hu, const double* b, const double* profile,
                                     const double* cfl, int32_t q0_is_eta);

/* One SSP-RK3 step (three fused reconstruction + update stage pairs). If dt_out is not NULL
 * the call synchronises the stream and returns the step's dt. A step at t >= t_end (t_end > 0),
 * or after an error, does nothing. Errors: SWALE_EINVAL (no problem set), SWALE_ECUDA; the
 * status of the step itself is read with swale_get_status (or reported by swale_advance). */
swale_status swale_step(swale_ctx* ctx, double* dt_out);

/* Up to max_steps steps, replayed as CUDA graphs of fixed length; stops early at t_end (with
 * an end time the steps go out in chunks of 64 to 4096 steps, and the call returns once every
 * instance has reached t_end or stopped on an error). Synchronises at the end and reports the
 * steps actually taken in *steps_done (may be NULL).
 * Error contract: a step in which an error appears (a non-finite value, a non-positive width, a
 * non-positive linear weight, no finite dt, a bounded wait that gave up) is not committed: the
 * instance keeps the state, nodes, widths, time and step count of its last good step, and every
 * later step is a no-op for it (in a batch the other instances go on). The call then returns
 * SWALE_ENONFINITE / SWALE_EMESH / SWALE_EWEIGHT / SWALE_ETIMEOUT (the device status word has the
 * matching bit), and *steps_done counts the good steps of instance 0; else SWALE_OK. The
 * context stays usable: a new problem (swale_set_problem, swale_batch_set_problem) clears the
 * status. */
swale_status swale_advance(swale_ctx* ctx, int64_t max_steps, int64_t* steps_done);

/* Enqueues nsteps steps on the context's stream and returns without synchronising (steps at
 * t >= t_end are no-ops on the device). Errors: SWALE_EINVAL, SWALE_ECUDA. */
swale_status swale_enqueue(swale_ctx* ctx, int64_t nsteps);

/* Kernel timing. While enabled (enable != 0), every enqueued step records CUDA events on the
 * context's stream around each kernel and steps are not replayed as graphs. swale_get_timing
 * synchronises and returns, for the kernel families 0 = per-step prologue, 1 = mesh velocity,
 * 2 = reconstruction, 3 = update, the summed device time in ms (ms[4]) and the number of
 * launches (launches[4]) since timing was last enabled. Either pointer may be NULL. */
swale_status swale_set_timing(swale_ctx* ctx, int32_t enable);
swale_status swale_get_timing(swale_ctx* ctx, double* ms, int64_t* launches);

/* Copies the current state of a single instance out (a batch: swale_batch_get_state). Any
 * pointer may be NULL. h, hu, b, eta: N values; x_nodes: N+1 values; t: one value (host or
 * device). Synchronises the stream. */
swale_status swale_get_state(swale_ctx* ctx, double* h, double* hu, double* b, double* eta, double* x_nodes,
                             double* t);

/* State of a batch in the concatenated layout of swale_batch_set_problem; t and dt: B values
 * (the time and the last step of each instance). Any pointer may be NULL. Synchronises. */
swale_status swale_batch_get_state(swale_ctx* ctx, double* hu, double* b, double* eta, double* x_nodes, double* t,
                                   double* dt);

/* Launch shape: the tile (threads per block: 64, 128 or 256; a reconstruction tile is that many
 * cells, a forward update tile one cell fewer, so that its interfaces take one pass) of the
 * reconstruction and update kernels and their grid (0 = one block per tile; G > 0 = a persistent grid of G blocks
 * walking the (instance, tile) work list). tiles[4] = {recon_tile, update_tile, recon_grid,
 * update_grid}. Results do not depend on the launch shape (bitwise). */
swale_status swale_set_tiles(swale_ctx* ctx, int32_t recon_tile, int32_t update_tile, int32_t recon_grid,
                             int32_t update_grid);
swale_status swale_get_tiles(swale_ctx* ctx, int32_t* tiles);

/* Autotuner: times `steps` steps (after one untimed step, the best of three such timings) for
 * each tile size pair in {64, 128, 256}^2, each with one block per tile and with a persistent
 * grid, from a snapshot of the current state that is restored afterwards, and keeps the
 * fastest. With a cache_path, a
 * matching entry (key: SM count, B, log2 of the total cells, mesh kind) is used without timing,
 * and a new result is appended as one JSON object per line. tiles_out[4] (may be NULL) receives
 * the chosen shape. Allocates a temporary snapshot (5 doubles per cell). */
swale_status swale_autotune(swale_ctx* ctx, int32_t steps, const char* cache_path, int32_t* tiles_out);

/* Detector classes (0 smooth, 1 transition, 2 non-smooth; Step 2 of Sec. 2.2) of the first
 * stage of the last step, N bytes (a batch: all instances' cells in order). Synchronises. */
swale_status swale_get_flags(swale_ctx* ctx, uint8_t* flags);

/* Accumulated device status word (SWALE_BIT_*; OR over the instances of a batch), the step
 * count and the last dt (of instance 0). Any pointer may be NULL; host pointers. Synchronises. */
swale_status swale_get_status(swale_ctx* ctx, uint32_t* status_bits, int64_t* steps, double* last_dt);

/* One evaluation of the semi-discrete right-hand side (Eq. hydro2D with Eq. bottomrk) for
 * the given state, independent of the context's problem: E = eta, M = hu, B = b, J widths
 * (N values each), w node velocities (N+1), alpha > 0 the global viscosity (alpha <= 0: alpha
 * of Eq. alpha2D, the largest |u - w| + sqrt(g h) over the edge states; with alpha_bound = 1,
 * the largest |u| + sqrt(g h) plus max |w|). Outputs R_E, R_M, R_B (N), the largest edge wave
 * speed *A_out (relative to w unless alpha_bound), flags (N bytes, may be NULL) and the status
 * bits (may be NULL).
 * Allocates and frees its own device scratch. Synchronises. */
swale_status swale_rhs(swale_ctx* ctx, int64_t N, const double* E, const double* M, const double* B,
                       const double* J, const double* w, double alpha, double* RE, double* RM, double* RB,
                       double* A_out, uint8_t* flags, uint32_t* status_bits);

/* Allocation-free variant of swale_rhs, for callers that cannot call cudaMalloc: code running
 * inside another framework's memory pool, which owns the device memory and must see every
 * allocation, or work whose device memory must not grow while it runs. The paper has no
 * counterpart: this is a library-side addition.
 *   cfg, cuda_stream   configuration (its scheme and alpha_bound are honoured) and stream
 *                      (NULL = legacy default stream; a stream must belong to the current
 *                      device); no context
 *   N                  number of cells, 5 <= N <= 65536 (SWALE_NOALLOC_MAX_CELLS)
 *   E, M, B, J, w      device pointers: surface, discharge, bottom, widths (N), node velocities (N+1)
 *   alpha              the global viscosity, > 0 (it is not derived here)
 *   RE, RM, RB         device pointers, N values each: the right-hand side
 *   A_out              host pointer or NULL: the largest edge wave speed (relative to w unless
 *                      cfg->alpha_bound); when given, the call synchronises the stream,
 *                      otherwise it returns after enqueueing
 *   flags              N bytes (host or device) or NULL: detector classes
 * Scratch lives in one fixed array of about 6.3 MB per device, held from library load until
 * the process exits; the call allocates nothing and clears what it reuses. Every call shares
 * that array, so calls that overlap on the GPU (other streams, other host threads) race; run
 * them one after the other. The first call on a device looks up the array's device address;
 * make that first call before any stream capture.
 * Errors: SWALE_EINVAL (N out of range, alpha <= 0, null or host pointer where a device pointer
 * is required, a stream of another device, bad config), SWALE_ECUDA. */
#define SWALE_NOALLOC_MAX_CELLS 65536
swale_status swale_rhs_noalloc(const swale_config* cfg, void* cuda_stream, int64_t N, const double* E,
                               const double* M, const double* B, const double* J, const double* w, double alpha,
                               double* RE, double* RM, double* RB, double* A_out, uint8_t* flags);

/* Checkpoint / resume of a forward run. swale_save writes the context's state (configuration,
 * offsets, per-instance CFL numbers, the cell averages of eta, hu and b, the widths of the GCL
 * recursion, nodes, motion profile, per-instance scalars such as t and the step count, and
 * the L2-projection bottom if set) to a versioned binary file; swale_load reads such a file
 * into a context created with the same configuration (bitwise equal swale_config) and
 * replaces its problem. A resumed run recomputes the first step's mesh geometry from the
 * stored widths, so it agrees with the uninterrupted run to rounding. Host byte order.
 * Errors: SWALE_EINVAL (no problem, file not readable / writable, wrong format, version or
 * configuration), SWALE_ENOMEM, SWALE_ECUDA. */
swale_status swale_save(swale_ctx* ctx, const char* path);
swale_status swale_load(swale_ctx* ctx, const char* path);

/* Bottom by L2 projection (Eq. baverage, Sec. 3.3) instead of its evolution by Eq. bottomrk:
 * b(x) is the piecewise polynomial with npieces pieces on breaks[npieces + 1] (increasing,
 * covering every instance's domain), piece p being sum_{k<=degree} coef[p (degree+1) + k]
 * (x - breaks[p])^k (degree <= 8; host or device arrays, copied). The bottom average of every
 * cell is then the exact average of b over the cell on each stage mesh (t_n, t_{n+1},
 * t_{n+1/2}) and after every step; the bottom averages passed to swale_set_problem should be
 * that projection at t = 0. All instances of a batch share b. npieces = 0 returns to Eq.
 * bottomrk; a new problem also does. Needs a problem set; not available with swale_adjoint.
 * Errors: SWALE_EINVAL (sizes, order, coverage, non-finite values), SWALE_ENOMEM, SWALE_ECUDA. */
swale_status swale_set_bottom_function(swale_ctx* ctx, int32_t npieces, int32_t degree, const double* breaks,
                                       const double* coef);

/* Stage viscosities alpha (Eq. alpha2D) of the next nsteps steps, 3 per step and instance, in
 * a log the context owns: mode 1 records them, mode 2 replays `log` (nsteps * B * 3 values,
 * host or device) instead of computing them, mode 0 turns the log off. Rows count from the
 * context's step counter at the call. Replay is the convention under which the discrete
 * adjoint differentiates (alpha held fixed), e.g. for finite-difference checks. */
swale_status swale_alpha_log(swale_ctx* ctx, int32_t mode, int64_t nsteps, const double* log);
swale_status swale_get_alpha_log(swale_ctx* ctx, double* log);

/* Discrete adjoint of a gauge misfit over the next nsteps steps from the current state, for
 * every instance i of the context:
 *   J_i = sum_{n=1..nsteps} dt_n sum_{g<G} (h_g(q^n) - h_obs[n-1][i][g])^2,
 * where h_g is the depth average of the cell that contains gauges_x[i*G + g] on the mesh at t_n.
 * Outputs (host or device, any may be NULL): J[B], and the gradients of J with respect to the
 * initial cell averages of eta, hu and b (Ntot values each; b varied with eta fixed).
 * The gradient is that of the discrete scheme under the replay convention: dt and the stage
 * viscosities alpha are those of the forward run, detector classes, limiter branches, dry-edge
 * tests and max/min selections are frozen (a tie follows the first argument); if a replay log
 * is active (swale_alpha_log mode 2) the forward run replays it instead. Checkpoints of
 * the state every ckpt_every steps; each segment but the last is recomputed once with per-step
 * snapshots (by a further set of state arrays on a low-priority stream, one segment ahead of the
 * reverse sweep; the forward run keeps the last segment's snapshots, and in tape mode its stage
 * data, itself) and each step once more before its reverse sweep (on a third stream, alternating
 * between the context's arrays and one more set, one step ahead of the reverse sweep, which
 * runs on the context's stream). These forward runs compute the mesh geometry in every stage
 * (no reuse of the previous step's), so the trajectory, and the gradient up to the order of
 * atomic additions, does not depend on ckpt_every. Device memory beyond the context's own: about
 * 5 (ceil(nsteps/C) + b C + 3) + 117 doubles per cell with C = min(ckpt_every, nsteps) and b = 2
 * segment buffers (1 when C = nsteps), taken as one block of exactly swale_adjoint_bytes bytes
 * (a single cudaMalloc); the block and the two streams are freed before the call returns. With ckpt_every >= nsteps every step runs
 * twice (once in tape mode). The mesh must be prescribed (static, profile or linear motion) and
 * t_end = 0. On return the context holds the state after the nsteps steps.
 * Errors: SWALE_EINVAL, SWALE_ENOMEM, SWALE_ECUDA, and the status errors of swale_advance. */
swale_status swale_adjoint(swale_ctx* ctx, int64_t nsteps, int64_t ckpt_every, int32_t G, const double* gauges_x,
                           const double* h_obs, double* J, double* dJ_deta0, double* dJ_dhu0, double* dJ_db0);

/* Device bytes swale_adjoint allocates for B instances with Ntot cells in total, without
 * (tape = 0) or with (tape = 1) the tape of swale_set_adjoint_tape (host-only arithmetic; needs
 * no device). Lets a caller pick ckpt_every for the memory it has: the checkpoints grow as
 * nsteps / ckpt_every, the per-segment snapshots (and the tape: about 39 doubles per cell and
 * step, for two segments, one when ckpt_every >= nsteps) as ckpt_every.
 * Errors: SWALE_EINVAL (a size < 1, tape not 0 or 1, or a NULL bytes pointer). */
swale_status swale_adjoint_bytes(int64_t B, int64_t Ntot, int64_t nsteps, int64_t ckpt_every, int32_t G,
                                 int32_t tape, uint64_t* bytes);

/* How swale_adjoint gets each step's stage data (the edge values of the three stages, q^(1),
 * q^(2) and their widths) for the reverse sweep. enable = 0 (the default): each step is
 * recomputed from its snapshot before its reverse sweep, so every step is run three times (twice
 * in the last segment). enable = 1: the recompute of a segment (for the last segment, the
 * forward run) keeps every step's stage data (a tape of about 39 doubles per cell and step, for
 * two segments), and the reverse sweep reads it: every step is run twice (once in the last
 * segment: with ckpt_every >= nsteps the forward run is the only one). The gradient is the same
 * up to the order of atomic additions. This
 * is a trade of memory for arithmetic that the paper does not discuss (it has no adjoint).
 * Errors: SWALE_EINVAL. */
swale_status swale_set_adjoint_tape(swale_ctx* ctx, int32_t enable);

/* Test hook for the bounded waits of the bulk (TMA) copies that stage the reconstruction's
 * tiles (the paper has no counterpart). With pad_bytes > 0, each tile of the next steps, after
 * its real copies have landed, also waits on a second barrier that expects pad_bytes which
 * never arrive, for `tries` polls (0: the default, about a million), so that wait runs out: the
 * kernel then sets SWALE_BIT_TIMEOUT and returns, the step is not committed and reports
 * SWALE_ETIMEOUT, and the context stays usable (reset the hook with 0, 0; the instance keeps the
 * state of its last good step, a new problem clears the status). A block never returns while a
 * copy of its own may still write its shared memory. Nothing faults or hangs.
 * Errors: SWALE_EINVAL, SWALE_ECUDA. */
swale_status swale_set_wait_test(swale_ctx* ctx, int32_t tries, uint32_t pad_bytes);

/* Check of the reciprocal that every kernel here uses in place of a division (the paper has
 * no counterpart): y[i] = the kernels' 1 / x[i] for i < n, on the given stream (NULL: the
 * legacy default stream; it must belong to the current device), asynchronous. x and y are
 * arrays of n doubles on the current device (they may be the same array). The reciprocal is
 * the hardware approximation refined by one third-order Newton-Raphson (Householder) step; for
 * normal, finite, non-zero x it is within one unit in the last place of the correctly rounded
 * 1 / x. Zero, infinite and subnormal x give NaN.
 * Errors: SWALE_EINVAL (n < 0, a NULL array, or one not on the current device), SWALE_ECUDA
 * (launch). */
swale_status swale_check_recip(void* cuda_stream, int64_t n, const double* x, double* y);

/* Message of the last error of this context ("" if none). Never NULL. */
const char* swale_last_error(const swale_ctx* ctx);

/* Frees the context and its device memory. NULL is ignored. */
void swale_destroy(swale_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* SWALE_H */
