/*
 * gmaf.h - C ABI of the GB300 piston-gap library (GMAF hot path).
 *
 * The library computes, for a joint batch of working conditions of an axial
 * piston pump's piston/bore oil film (arXiv 2511.06824):
 *   (a) the FVM-discretised Reynolds equation of the unwrapped gap
 *       (Sec. 2.1, Eq. 2.1-2.7) with film thickness from Eq. 2.3 plus
 *       dimple texture,
 *   (b) the solution of all conditions as one joint system (Eq. 3.7-3.8) by
 *       ASSOR-II (Eq. 3.3-3.6) or Jacobi (Eq. 2.8) preconditioned conjugate
 *       gradient (Table 1) under the synchronized criterion (Eq. 3.9),
 *   (c) force and moment integration from normal pressure and viscous shear
 *       (Sec. 2.4-III),
 *   and, around them, one double-Jacobian Picard iteration (Eq. 2.12-2.19).
 *
 * Conventions shared by every entry point:
 *   - All functions are `extern "C"`, return an int status (GMAF_OK = 0 or a
 *     negative code below), never abort and never print.
 *   - Device arrays are owned by the caller (e.g. torch tensors); the library
 *     owns only the opaque context and the workspace it allocates inside the
 *     context's HBM budget.  Host arrays are plain C arrays owned by the
 *     caller.
 *   - Grid layout: n_theta x n_z cells, theta (circumferential, periodic) is
 *     the fastest index; cell (i, j) of condition k is element
 *     i + n_theta * (j + n_z * k) of a joint array (system-major, Eq. 3.8).
 *   - Work is issued on the context's CUDA stream.  Calls that return host
 *     results (iteration counts, residuals, loads of the Picard step)
 *     synchronise that stream before returning; gmaf_assemble and
 *     gmaf_integrate_loads are asynchronous.
 *   - A context is not thread-safe: one host thread at a time per context.
 */
#ifndef GMAF_H
#define GMAF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define GMAF_OK              0
#define GMAF_INVALID_ARG    -1  /* null pointer, n_theta < 3, n_z < 2, c <= 0, mu <= 0,
                                   omega not in (0,2), eps <= 0, ...            */
#define GMAF_CONTACT        -2  /* some film thickness h <= 0 (piston touches the bore) */
#define GMAF_NOT_CONVERGED  -3  /* iteration budget exhausted; outputs still written   */
#define GMAF_NONFINITE      -4  /* NaN/Inf met in a reduction (or a non-positive u.Au) */
#define GMAF_OUT_OF_MEMORY  -5  /* workspace would exceed the context's HBM budget    */
#define GMAF_CUDA_ERROR     -6  /* CUDA runtime error; destroy the context            */
#define GMAF_TIMEOUT        -7  /* a device-side bounded loop gave up                 */
#define GMAF_CANCELLED      -8  /* a served request was cancelled before it finished  */

/* ---- problem description (Sec. 2.1, Eq. 2.3, Table 8) ---------------- */

/* Cells of the unwrapped gap: n_theta >= 3 around (periodic), n_z >= 2 along. */
typedef struct { int32_t n_theta, n_z; } gmaf_grid;

/* R_k piston radius [m]; L gap (coupling) length [m]; c radial clearance [m]
 * (bore radius R_c = R_k + c); mu dynamic viscosity [Pa s]; v_slide axial speed
 * of the piston relative to the bore, + from chamber (z = 0) to case (z = L)
 * [m/s]; p_chamber, p_case Dirichlet pressures at z = 0 and z = L [Pa]. */
typedef struct {
    double R_k, L, c;
    double mu;
    double v_slide;
    double p_chamber, p_case;
} gmaf_physics;

/* kind 0: smooth piston.  kind 1: flat-bottom circular dimples of `radius` and
 * `depth` on a hexagonal lattice with the given area density; the lattice has
 * a whole number of columns around the piston and is shifted by
 * (offset_theta, offset_z) metres on the unwrapped surface (h_Text of Eq. 2.3). */
typedef struct {
    int32_t kind;
    double radius, depth, area_density, offset_theta, offset_z;
} gmaf_texture;

/* Eccentricities e1, e2 at z = 0 and e3, e4 at z = L [m] and their rates [m/s] (Eq. 2.3). */
typedef struct { double e[4], edot[4]; } gmaf_state;

/* precond: 0 Jacobi (Eq. 2.8), 1 ASSOR-II (Eq. 3.4), 2 ASSOR-I (Eq. 3.2, the
 *   diagonal w (2 - w) / {(D + w L) D^-1 (D + w L)^T}_ii).  omega in (0, 2).
 * eps: tolerance of the convergence criterion below.
 * max_iter: PCG iteration budget (inner iterations in mixed precision).
 * precision: 0 FP64 throughout; 1 mixed - FP32 stencil, preconditioner and
 *   vector updates with dot products accumulated to FP64 accuracy, inside an
 *   FP64 iterative-refinement loop whose residual and stopping test are FP64.
 *   By default the inner FP32 PCG is not restarted at a refinement: after every
 *   tenfold reduction its residual is replaced by the FP64 residual and the
 *   recurrence continues with its search direction (environment variables
 *   GMAF_RELIABLE_DELTA for the reduction, GMAF_MIXED_RESTART=1 to restart
 *   instead; both read when the context is created).
 * zero_init: 1 start from p = 0 (Table 1 step 1); 0 use the contents of p. */
typedef struct {
    int32_t precond;
    double omega, eps;
    int32_t max_iter;
    int32_t precision;
    int32_t zero_init;
    int32_t criterion;  /* 0 synchronized (Sec. 3.3, Eq. 3.9): one PCG on the joint
                           system with global scalars, stopped when
                           ||A_G p_G - S_G||_2 / ||S_G||_2 <= eps.
                           1 asynchronized (Eq. 3.10): every condition k is its own
                           PCG with its own scalars, stopped when
                           ||A_k p_k - S_k||_2 / ||S_k||_2 <= eps; converged
                           conditions drop out on the device.  FP64 only
                           (precision 0); GMAF_INVALID_ARG otherwise. */
} gmaf_solver_opts;

/* Details of the last solve on a context (filled by gmaf_solve_joint and
 * gmaf_picard_step). */
typedef struct {
    int32_t iterations;        /* PCG iterations (inner iterations summed in mixed mode) */
    int32_t outer_iterations;  /* FP64 refinements (mixed), 1 in FP64                   */
    int32_t restarts;          /* restarts after a true-residual check failed            */
    int32_t status;
    double rel_residual;       /* recurrence relative residual at exit (FP64 mode)       */
    double true_rel_residual;  /* ||S - A p|| / ||S|| at exit, in FP64                   */
    int32_t kernel_variant;    /* PCG kernels used: 1000 VEC + 10 TY + MINB (columns per
                                  lane, rows per task, blocks per SM), + 100000 DB when
                                  phase B stages its rows DB ahead through shared memory,
                                  + 200000 DA when phase A does, + 2000000 when phase B
                                  is filled by bulk copies, + 10000000 when phase A
                                  rebuilds the diagonal from the couplings, + 100000000 W
                                  for blocks of W warps; 1000000 + 1000 VEC + MINB for the
                                  static schedule; 3000000 + 10000 RPW + 1000 NS + TB for
                                  the block-marched phase B with TMA tiles.  Chosen per
                                  problem shape by the autotuner on the first solve of
                                  that shape */
    int32_t tasks;             /* strip x row-block x condition tasks per PCG phase       */
    int32_t iterations_sum;    /* PCG iterations summed over the conditions: n_cond x
                                  iterations under the synchronized criterion, the sum of
                                  the per-condition counts under the asynchronized one
                                  (iterations is then the largest of them)              */
    int32_t p_update_period;   /* PCG iterations between two updates of p in phase A: 1,
                                  or 2 when the staged FP32 phase A pairs them           */
} gmaf_solve_info;

typedef struct gmaf_ctx gmaf_ctx;

/* Create a context on the current CUDA device.  hbm_budget_bytes caps the
 * workspace the library may allocate (0 = no cap).  cuda_stream is a
 * cudaStream_t (NULL = legacy default stream).  *out receives the context. */
int gmaf_create(gmaf_ctx **out, size_t hbm_budget_bytes, void *cuda_stream);

/* Synchronise the context's stream and free the context and its workspace. */
int gmaf_destroy(gmaf_ctx *ctx);

/* Change the stream subsequent calls are issued on. */
int gmaf_set_stream(gmaf_ctx *ctx, void *cuda_stream);

/* Bytes of device workspace currently held by the context. */
int gmaf_workspace_bytes(const gmaf_ctx *ctx, size_t *bytes_out);

/* Details of the last solve. */
int gmaf_last_solve_info(const gmaf_ctx *ctx, gmaf_solve_info *info_out);

/* FVM assembly of the Reynolds equation (Sec. 2.1, Eq. 2.1-2.7; Sec. 2.4-I).
 * conds: host array of n_cond states.  D, aE, aN, S: device arrays of
 * n_cond * n_z * n_theta doubles, written.  Row P of condition k reads
 *   D p_P - aE[P] p_E - aE[W] p_W - aN[P] p_N - aN[S] p_S = S[P]
 * (aE couples i to i+1 with periodic wrap, aN couples j to j+1 and is 0 in
 * the last row; the half-cell Dirichlet terms are inside D and S).
 * Returns GMAF_CONTACT (arrays still written) when some h <= 0.  Synchronises
 * the stream only to read the contact flag. */
int gmaf_assemble(gmaf_ctx *ctx, const gmaf_grid *grid, const gmaf_physics *phys,
                  const gmaf_texture *tex, const gmaf_state *conds, int32_t n_cond,
                  double *D, double *aE, double *aN, double *S);

/* Joint PCG on the block-diagonal system of n_cond conditions (Table 1,
 * Eq. 3.7-3.9) with one set of scalars for the whole joint system.
 * D, aE, aN, S: device arrays as written by gmaf_assemble.  p: device array
 * (n_cond * n), initial guess unless opts->zero_init, overwritten with the
 * solution.  iters_out, rel_res_out: host outputs (may be NULL); rel_res_out
 * receives the true relative residual ||S - A p|| / ||S|| in FP64.
 * Synchronises the stream.  GMAF_NOT_CONVERGED leaves the last iterate in p. */
int gmaf_solve_joint(gmaf_ctx *ctx, const gmaf_grid *grid, int32_t n_cond,
                     const double *D, const double *aE, const double *aN, const double *S,
                     double *p, const gmaf_solver_opts *opts, int32_t *iters_out,
                     double *rel_res_out);

/* Loads from the pressure fields (Sec. 2.4-III): per condition, force and
 * moment (Fx, Fy, Fz, Mx, My, Mz) from normal pressure and from viscous shear,
 * integrated on the elements bounded by cell centres and the two boundary
 * lines, moments about the bore axis at z = 0.  conds: host array (for the
 * film thickness in the shear stress).  p: device array (n_cond * n).
 * loads: device array of n_cond * 12 doubles, written as
 * [k][0..5] pressure part, [k][6..11] shear part.  Asynchronous. */
int gmaf_integrate_loads(gmaf_ctx *ctx, const gmaf_grid *grid, const gmaf_physics *phys,
                         const gmaf_texture *tex, const gmaf_state *conds, int32_t n_cond,
                         const double *p, double *loads);

/* One general (double-Jacobian) Picard iteration (Eq. 2.12-2.19), all on the
 * device: fan-out into the 9 conditions (base, e_j + d_e, edot_j + d_edot),
 * assembly, joint solve, loads, the 6 x 8 Jacobian of the total (pressure +
 * shear) loads by forward differences (Eq. 2.13-2.14), the generalized force
 *   G = (Fx - My/L, Fy + Mx/L, My/L, -Mx/L) + F_ext
 * and the update of (e, edot) from (J_edot + dt J_e) delta = -G - J_e (e_prev
 * + dt edot - e), edot += delta, e = e_prev + dt edot.
 * All arguments are host memory.  opts->zero_init = 1 starts the joint solve
 * from p = 0 (Table 1 step 1); 0 starts it from the 9 pressure fields the
 * previous gmaf_picard_step call on this context left behind when that call
 * had the same grid (the usual case inside a Picard loop or a time march),
 * else from 0.  state is updated in place only when the solve converged.  loads_out[12]: loads of the base condition; J_out[48]:
 * row-major 6 x 8 Jacobian (columns e1..e4, edot1..edot4); G_out[4]: G before
 * the update.  Synchronises the stream. */
int gmaf_picard_step(gmaf_ctx *ctx, const gmaf_grid *grid, const gmaf_physics *phys,
                     const gmaf_texture *tex, gmaf_state *state, const double e_prev[4],
                     double dt, const double F_ext[4], double d_e, double d_edot,
                     const gmaf_solver_opts *opts, double loads_out[12], double J_out[48],
                     double G_out[4], int32_t *iters_out);

/* One conventional (simplified) Picard iteration, Eq. 2.20-2.22, for comparison
 * with the general scheme: the Jacobian F_,e is dropped, so only the base
 * condition and the 4 rate perturbations edot_j + d_edot are assembled and
 * solved (one joint system of 5 conditions sharing one coefficient set), then
 *   edot_new = edot - [F_,edot]^-1 G                    (Eq. 2.21)
 *   e_new    = e + dt (edot_new - edot)                  (Eq. 2.22)
 * with G the generalized force of the base loads plus F_ext.  Arguments,
 * outputs and errors as gmaf_picard_step (no e_prev, no d_e); J_out's e-columns
 * are 0 (not formed).  Synchronises the stream. */
int gmaf_picard_step_simplified(gmaf_ctx *ctx, const gmaf_grid *grid, const gmaf_physics *phys,
                                const gmaf_texture *tex, gmaf_state *state, double dt,
                                const double F_ext[4], double d_edot,
                                const gmaf_solver_opts *opts, double loads_out[12],
                                double J_out[48], double G_out[4], int32_t *iters_out);

/* Per-phase kernel timing (tracing).  When enabled (on != 0), the PCG loop of
 * later solves is driven in host chunks instead of the graph WHILE node, with a
 * CUDA event pair around every phase launch on the context's stream; results
 * are bitwise the same.  gmaf_phase_timing returns, per kernel kind
 * [0] phase A (u update + stencil), [1] phase B (residual update + ASSOR-II),
 * [2] initial preconditioner pass, [3] FP64 residual, the summed event time in
 * milliseconds and the number of launches since timing was enabled.  Enabling
 * resets the sums. */
int gmaf_set_phase_timing(gmaf_ctx *ctx, int on);
int gmaf_phase_timing(const gmaf_ctx *ctx, double ms_out[4], int64_t launches_out[4]);

/* Allocation-free joint solve.  The paper has no counterpart: this entry point
 * exists for callers that may not allocate device memory while they run, for
 * example a solver plug-in inside a host program whose own pool allocator owns
 * all of the GPU's memory and offers plug-ins no allocation hook, or a
 * real-time co-simulation loop that cannot accept the latency, or the possible
 * failure, of an allocation in the middle of a time step.  It computes what
 * gmaf_solve_joint computes in FP64 mode with the synchronized criterion
 * (opts->precision and opts->criterion must be 0), with the
 * same arguments minus the context and plus the stream, and allocates nothing:
 * its scratch is a fixed array of GMAF_NOALLOC_SCRATCH_BYTES inside the
 * library.  The array sits in a code module of its own, which CUDA loads on a
 * device at the first call of this entry point there (lazy module loading, the
 * default; under CUDA_MODULE_LOADING=EAGER at context creation): that is when
 * the array's device memory is committed, and the device holds it until the
 * process exits.  Loading the module can itself fail for lack of memory, so a
 * caller whose pool allocator later takes the GPU's memory should make one
 * warm-up call on each device first (it may be a small problem), and make it
 * before any stream capture: the first call on a device also looks up the
 * array's device address with that device current.  The array lies outside
 * every context's hbm_budget_bytes and gmaf_workspace_bytes and outside the
 * server's footprint admission; the other entry points never load it.
 * A problem needs 1048576 + 7 * ceil256(8 * n_cond * n_theta * n_z)
 * bytes of it, so at most 1,778,816 joint unknowns (the 9-condition
 * 512 x 256 batch fits);
 * larger problems return GMAF_OUT_OF_MEMORY before any work is issued.  Every
 * call uses the same array and leaves its contents behind, so calls whose GPU
 * work overlaps (different streams, threads or processes sharing the library on
 * one device) race on it: serialise them.  Synchronises the stream, also when it
 * returns an error after issuing work, so a failed call leaves nothing running
 * on the array. */
#define GMAF_NOALLOC_SCRATCH_BYTES (96u * 1024u * 1024u)
int gmaf_solve_joint_noalloc(const gmaf_grid *grid, int32_t n_cond, const double *D,
                             const double *aE, const double *aN, const double *S, double *p,
                             const gmaf_solver_opts *opts, void *cuda_stream, int32_t *iters_out,
                             double *rel_res_out);

/* ---- continuous-batching server ---------------------------------------
 * Requests are single Picard iterations (as gmaf_picard_step, always in the
 * mixed-precision mode, ASSOR-II) of a 9-condition joint batch on their own
 * grid (n_theta must be a multiple of 4).  gmaf_server_submit queues a request;
 * gmaf_server_run admits queued requests first-come first-served while their
 * device footprint (gmaf_request_footprint) fits in the server's arena of
 * hbm_budget_bytes (allocated once at creation on the context's device and
 * stream), advances all admitted requests together by `iterations` batched PCG
 * iterations (one persistent kernel per CG phase over every request's tasks),
 * then takes the FP64 refinement step of every request whose inner solve ended
 * and either restarts it or finishes it (loads, Jacobian, update) and frees its
 * memory.  Finished results are collected with gmaf_server_poll in completion
 * order.  Each request keeps its own scalars and convergence test
 * (Eq. 3.9 per request), so its result does not depend on which other
 * requests share the GPU.  Not thread-safe.
 * Tiling: every request's tasks span 128 columns and a number of rows chosen
 * per grid by an autotuner: the first request of a grid on a device times one
 * batched PCG iteration on its own data for each candidate (16, 32, 64 rows) and
 * the fastest is kept for that grid for the life of the process (so a request's
 * decomposition, hence its result, depends only on its grid).  Rounds are CUDA
 * graphs of `iterations` phase pairs, re-instantiated only when the round
 * length or the kernels change and updated in place when the launch grid does.
 * Environment (read when a server is created): GMAF_SV_GRAPH=0 drives rounds
 * from the host instead, GMAF_SV_TUNE=0 keeps 32 rows for every grid. */
typedef struct gmaf_server gmaf_server;

typedef struct {
    gmaf_grid grid;
    gmaf_physics phys;
    gmaf_texture tex;
    gmaf_state state;          /* state at which the step is evaluated */
    double e_prev[4];          /* eccentricity at the previous time point */
    double dt;
    double F_ext[4];           /* generalized external force */
    double d_e, d_edot;        /* forward-difference steps */
    double omega, eps;         /* ASSOR relaxation, Eq. 3.9 tolerance (FP64 residual) */
    int32_t max_iter;          /* inner PCG iteration budget */
} gmaf_request;

typedef struct {
    int64_t id;
    int32_t status;            /* GMAF_OK, GMAF_NOT_CONVERGED, GMAF_CONTACT, ... */
    int32_t iterations;        /* inner PCG iterations */
    int32_t outer_iterations;  /* refinement sweeps */
    double true_rel_residual;
    gmaf_state state;          /* updated state (input state unless GMAF_OK) */
    double loads[12];          /* base-condition loads: pressure then shear */
    double J[48];              /* 6 x 8 Jacobian, row-major */
    double G[4];               /* generalized force before the update */
    int32_t tile_rows;         /* rows per task of its batched PCG tasks (tuned per grid) */
} gmaf_result;

/* Device bytes one request of this grid occupies in a server's arena. */
int gmaf_request_footprint(const gmaf_grid *grid, size_t *bytes_out);
int gmaf_server_create(gmaf_ctx *ctx, size_t hbm_budget_bytes, gmaf_server **out);
int gmaf_server_destroy(gmaf_server *server);
/* Queue a request; *id_out receives its id.  GMAF_OUT_OF_MEMORY if it can never fit. */
int gmaf_server_submit(gmaf_server *server, const gmaf_request *request, int64_t *id_out);
/* Admit, advance by `iterations` batched PCG iterations, refine/finish; synchronises. */
int gmaf_server_run(gmaf_server *server, int32_t iterations, int32_t *active_out,
                    int32_t *queued_out);
/* Move up to max_results finished results to out; *n_out receives the count. */
int gmaf_server_poll(gmaf_server *server, gmaf_result *out, int32_t max_results, int32_t *n_out);
/* Free bytes left in the server's arena. */
int gmaf_server_free_bytes(const gmaf_server *server, size_t *bytes_out);
/* Cancel request `id`, queued or admitted: it leaves the queue or the batched set,
 * its arena block is released at once (after the server's stream has finished
 * the work already issued for it), and gmaf_server_poll later returns one result
 * for it with status GMAF_CANCELLED and its input state.  GMAF_INVALID_ARG if
 * no queued or active request has this id (e.g. it already finished).
 * Synchronises the server's stream when the request was admitted. */
int gmaf_server_cancel(gmaf_server *server, int64_t id);

/* Copy the pressure fields of the last Picard step on this context
 * (condition-major, device memory p_out of 9 * n_z * n_theta doubles): the 9
 * conditions of gmaf_picard_step, or the 5 of gmaf_picard_step_simplified (base,
 * then edot_1..4 + d_edot; the rest of p_out is left alone), for a step of the
 * given grid; GMAF_INVALID_ARG if the last step had another grid.  Asynchronous. */
int gmaf_last_fields(gmaf_ctx *ctx, const gmaf_grid *grid, double *p_out);

/* Static description of a status code. */
const char *gmaf_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* GMAF_H */
