/*
 * rmhd.h -- C ABI of the GB300 (sm_103a) library for one SSP2(222) IMEX time
 * step of resistive special-relativistic MHD, single-fluid and two-fluid,
 * after Wright & Hawke, "Resistive and multi-fluid RMHD on graphics
 * processing units" (arXiv:1808.09721).
 *
 * Conventions
 *   - Every call returns an int status: RMHD_OK (0) or a negative RMHD_ERR_*.
 *     rmhd_last_error() gives a message owned by the context, valid until the
 *     next call on that context.
 *   - Arrays are structure-of-arrays FP64, variable-major, x fastest:
 *     a[v][j][i] at a[(v * ny + j) * nx + i], interior cells only (no ghosts).
 *   - `where` selects RMHD_HOST (pageable or pinned host memory) or
 *     RMHD_DEVICE (memory of the context's GPU). The caller keeps ownership of
 *     every array it passes; the library never keeps the pointer. The state
 *     and primitive calls (set/get prims, cons, state) read and write device
 *     arrays and page-locked host arrays (cudaHostAlloc, cudaHostRegister,
 *     pinned torch tensors) in place from their kernels, host arrays over the
 *     host-GPU link; pageable host arrays go through a staging copy. A
 *     RMHD_DEVICE pointer that is not device memory of the context's device
 *     fails with RMHD_ERR_INVALID.
 *   - All device work is issued on the CUDA stream given to rmhd_create. Calls
 *     marked "async" return after enqueueing; the calls that read results back
 *     synchronise that stream first.
 *
 * Variables (Sec. 2.1.1 and Sec. 2.1.2 of the paper)
 *   one fluid, 14 conserved: D, S_x, S_y, S_z, tau, B_x, B_y, B_z, E_x, E_y, E_z, varrho, psi, phi
 *   one fluid, 11 primitives: rho, v_x, v_y, v_z, p, B_x, B_y, B_z, E_x, E_y, E_z
 *   two fluids, 18 conserved: D, S_xyz, tau, Dbar, Sbar_xyz, taubar, B_xyz, E_xyz, psi, phi
 *   two fluids, 16 primitives: rho_e, v_e(3), p_e, rho_p, v_p(3), p_p, B(3), E(3)
 */
#ifndef RMHD_H
#define RMHD_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define RMHD_OK 0
#define RMHD_ERR_INVALID (-1)  /* bad argument, or inadmissible primitive state (v >= 1, rho <= 0, p <= 0, NaN) */
#define RMHD_ERR_CUDA (-2)     /* a CUDA runtime call failed */
#define RMHD_ERR_NEWTON (-3)   /* an implicit-stage solve did not converge in some cell */
#define RMHD_ERR_C2P (-4)      /* primitive recovery failed in some cell */
#define RMHD_ERR_STATE (-5)    /* call out of order (e.g. step before set_prims) */
#define RMHD_ERR_NOMEM (-6)    /* workspace too small or allocation failed */

/* models */
#define RMHD_RESISTIVE 0 /* single-fluid resistive SRMHD, Eq. (resistive RMHD), N_c = 14 */
#define RMHD_TWO_FLUID 1 /* two-fluid resistive SRMHD, Eq. (twoFluid cons) + Appendix A, N_c = 18 */

/* boundary conditions */
#define RMHD_OUTFLOW 0  /* ghost cells copy the nearest interior cell */
#define RMHD_PERIODIC 1 /* ghost cells wrap around */

/* flux arithmetic */
#define RMHD_FP64 0  /* everything in FP64 */
#define RMHD_MIXED 1 /* WENO3/flux arithmetic in FP32 with FP64 accumulation of the update;
                        the implicit source solve, primitive recovery and current J stay FP64 */
#define RMHD_FLOATFLOAT 2 /* WENO3/flux arithmetic in float-float (pairs of FP32 numbers, ~48
                             significant bits, on the FP32 pipes), the rest as RMHD_MIXED; both
                             models on single grids (1-D, 2-D, 3-D), not batches. Differs from
                             RMHD_FP64 by ~1e-13 relative per step (unstable flows amplify it like
                             any round-off) while the state stays inside FP32's range */

/* memory kinds for `where` */
#define RMHD_HOST 0
#define RMHD_DEVICE 1

/* IMEX integrators of Sec. 2.2.1: SSP2(222) (Table 1; 2 implicit stages and
 * 2 flux passes per step) and SSP3(332) (Table 2; 3 + 3), gamma = 1 - 1/sqrt(2). */
#define RMHD_SSP2 0
#define RMHD_SSP3 1

typedef struct rmhd_config {
    int model;        /* RMHD_RESISTIVE or RMHD_TWO_FLUID */
    int nx, ny;       /* interior cells; ny = 1 is a 1-D run along x */
    double xmin, xmax, ymin, ymax;
    double gamma;     /* Gamma-law EOS p = rho e (Gamma - 1), Sec. 2.1; 1 < Gamma <= 2 */
    double sigma;     /* conductivity (one fluid, Ohm's law of Sec. 2.1.1); eta = 1/sigma for two fluids */
    double mu_e, mu_p;/* charge-to-mass ratios (two fluids only), mu_e != mu_p */
    double kappa;     /* divergence-cleaning rate, 1 in the paper (Sec. 2.1.1) */
    double cfl;       /* dt = cfl * min(dx, dy, dz) when rmhd_imex_step gets dt <= 0 */
    int bc_x, bc_y;   /* RMHD_OUTFLOW or RMHD_PERIODIC */
    int precision;    /* RMHD_FP64, RMHD_MIXED or RMHD_FLOATFLOAT */
    int scheme;       /* RMHD_SSP2 (0, Table 1) or RMHD_SSP3 (1, Table 2); batches: RMHD_SSP2 */
    int nz;           /* cells along z; 0 or 1: a 1-D or 2-D grid. nz > 1 (3-D) needs ny > 1 and a
                         single grid (not a batch); arrays are then [n_var][nz][ny][nx] */
    int bc_z;         /* RMHD_OUTFLOW or RMHD_PERIODIC along z (3-D only) */
    double zlen;      /* extent of the grid along z (3-D only), dz = zlen / nz */
} rmhd_config;

typedef struct rmhd_ctx rmhd_ctx;

/* Bytes of device workspace a context with this configuration needs.
 * Errors: RMHD_ERR_INVALID for a bad configuration: any field out of range,
 * nx*ny*nz above 2^31 - 1 cells, or above the flux kernel's launch grid
 * (ny > 524280 in 2-D; nz or ny > 65535 in 3-D). */
int rmhd_workspace_bytes(const rmhd_config *cfg, size_t *bytes);

/* Create a context on the device of `cuda_stream` (a cudaStream_t; NULL means
 * the legacy default stream of the current device). If `workspace` is not
 * NULL it must be device memory of at least rmhd_workspace_bytes() bytes,
 * 256-byte aligned, owned by the caller and kept alive until rmhd_destroy;
 * otherwise the library allocates (and later frees) its own.
 * Errors: RMHD_ERR_INVALID, RMHD_ERR_NOMEM, RMHD_ERR_CUDA. On error *out is NULL. */
int rmhd_create(rmhd_ctx **out, const rmhd_config *cfg, void *cuda_stream,
                void *workspace, size_t workspace_bytes);

/* Release the context (synchronises its stream). NULL is accepted. */
void rmhd_destroy(rmhd_ctx *ctx);

/* Message for the last failing call on this context (never NULL). */
const char *rmhd_last_error(const rmhd_ctx *ctx);

/* Set the state from primitives [n_prim][ny][nx] (11 or 16 variables, see
 * above). psi = phi = 0 (Sec. 2.1.1). For one fluid the charge density is
 * initialised from Gauss's law varrho = div E by second-order central
 * differences with the boundary conditions (Sec. 2.1.1). Conserved variables
 * follow Eq. (resistive prims) / Eq. (twoFluid cons). Synchronous.
 * Errors: RMHD_ERR_INVALID (inadmissible state; message names the first cell). */
int rmhd_set_prims(rmhd_ctx *ctx, const double *prims, int where);

/* Primitives of the current state in the same layout. After a step they are
 * recovered from the conserved state (Sec. 2.1.3) in the same pass that
 * writes the output. Synchronous. Errors: RMHD_ERR_STATE (no state),
 * RMHD_ERR_C2P (some cell has no primitives; message names the first one;
 * the contents of `prims` are then unspecified), RMHD_ERR_INVALID, RMHD_ERR_CUDA. */
int rmhd_get_prims(rmhd_ctx *ctx, double *prims, int where);

/* Conserved state [N_c][ny][nx]; set_cons recovers the primitives
 * (Sec. 2.1.3) and fails with RMHD_ERR_C2P if some cell has none. Synchronous. */
int rmhd_get_cons(rmhd_ctx *ctx, double *cons, int where);
int rmhd_set_cons(rmhd_ctx *ctx, const double *cons, int where);

/* Full-state checkpoint for bitwise restarts: the conserved state and the
 * primitives the next stage solve starts from, [N_c + N_w][ny][nx] (N_w = 5,
 * one fluid: v_x, v_y, v_z, p, W; N_w = 10, two fluids: v, p, rho h W^2 per
 * species, electrons first). A context restored with rmhd_set_state (same
 * configuration) continues bit for bit as the saved one would have;
 * rmhd_set_cons restores the same conserved state but recovers fresh
 * primitives, so a continued run agrees only to round-off. The simulation
 * time is not part of the state. rmhd_state_doubles gives the array length.
 * Synchronous. Errors: RMHD_ERR_INVALID, RMHD_ERR_STATE (get before any
 * state), RMHD_ERR_CUDA. */
int rmhd_state_doubles(const rmhd_ctx *ctx, size_t *n);
int rmhd_get_state(rmhd_ctx *ctx, double *state, int where);
int rmhd_set_state(rmhd_ctx *ctx, const double *state, int where);

/* Advance `nsteps` IMEX steps of the configured scheme (SSP2(222), Table 1,
 * or SSP3(332), Table 2; Sec. 2.2.1) with fluxes from Lax-Friedrichs
 * splitting + WENO3 (Sec. 2.2.2). dt <= 0 selects dt = cfl * min(dx, dy, dz)
 * over the grid's directions (batches: each run's own cfl * dx). Steps of one
 * dt are replayed from one captured CUDA graph. Async: enqueued on the
 * context's stream. A failed
 * implicit solve or recovery is recorded on the device and reported by the
 * next synchronous call (or rmhd_check). If t_out is not NULL it receives the
 * simulation time after the steps (host bookkeeping, no synchronisation). */
int rmhd_imex_step(rmhd_ctx *ctx, double dt, int nsteps, double *t_out);

/* Synchronise the stream and report any failure recorded on the device since
 * the last check: RMHD_ERR_NEWTON or RMHD_ERR_C2P with the first failing cell
 * in rmhd_last_error. */
int rmhd_check(rmhd_ctx *ctx);

/* Solver statistics (tracing; off by default). While enabled, every stage
 * solve adds one count to three device histograms: by the number of FP32
 * Newton iterations it took (hist[k], k = 1..30; hist[31]: 31 or more), by
 * the number of FP64 refinement passes (hist[32 + k - 1], k = 1..8), and by
 * the start that converged (hist[40]: the explicit part's E; hist[41]: the
 * ideal-MHD limit E = -v x B after the first start failed; hist[42]: the
 * continuation in a dt after both failed; hist[43]: no start converged --
 * the cell is then reported as RMHD_ERR_NEWTON; two-fluid solves count 40
 * or 43). Counting uses device atomics and slows the stage kernels: it is for
 * diagnostics, not for timed runs. rmhd_set_solver_stats(ctx, 1) clears the
 * histograms and starts counting, 0 stops it; rmhd_solver_stats copies the
 * 44 counts into the caller's host array `hist` and clears them.
 * Synchronous. Errors: RMHD_ERR_INVALID, RMHD_ERR_CUDA. */
int rmhd_set_solver_stats(rmhd_ctx *ctx, int enable);
int rmhd_solver_stats(rmhd_ctx *ctx, unsigned long long *hist);

/* Fault injection for tests of the error path, with no GPU fault involved:
 * caps the FP64 refinement passes of every stage solve at `passes` (1..8;
 * 0 restores the default, 8). A solve needs at least two passes to confirm
 * convergence, so with a cap of 1 the next step records RMHD_ERR_NEWTON with
 * the first failing cell (reported by rmhd_check), and the context stays
 * usable. Errors: RMHD_ERR_INVALID (passes outside 0..8). */
int rmhd_set_refinement_cap(rmhd_ctx *ctx, int passes);

/* Test control of the stage-solve restarts (single fluid). Every implicit
 * stage solve (Sec. 2.2.1, Eq. implicit stage) tries up to three starts: 0,
 * the explicit part's E; 1, the ideal-MHD limit E = -v x B (Sec. 2.1.1); 2,
 * a continuation in a dt; a cell whose start fails goes on to the next. The
 * root is the same whichever start converges. rmhd_set_first_start(ctx, s)
 * makes every solve begin at start s (1 or 2; 0, the default, restores all
 * starts), which exercises the restart path on any state; all cells must fit
 * the restart list (2^18 cells). Errors: RMHD_ERR_INVALID (s outside 0..2,
 * grid too large), RMHD_ERR_STATE (two-fluid context). */
int rmhd_set_first_start(rmhd_ctx *ctx, int start);

/* Diagnostics of the current state (Sec. 2.1 invariants), written to out[8]:
 * sum D, sum tau, sum S_x, sum B_x, sum varrho (Dbar for two fluids)
 * (cell sums times the cell volume), max |v|, number of non-finite conserved
 * values, and the CFL time step cfl * min(dx, dy, dz) over the grid's
 * directions. Synchronous. */
int rmhd_diagnostics(rmhd_ctx *ctx, double *out);

/* Discrete adjoint of the IMEX step, SSP2(222) or SSP3(332) (either model,
 * FP64, 1-D, 2-D or 3-D single grid with at least 3 cells per direction): gradients
 * of a functional of the final
 * conserved state with respect to the initial primitives and sigma.
 *   rmhd_record arms recording of the next `nsteps` steps; it must follow
 *   rmhd_set_prims directly (the gradient is w.r.t. those primitives, with
 *   psi = phi = 0 and, for one fluid, varrho = div E as rmhd_set_prims
 *   builds them; for two fluids the charge Dbar follows from the species
 *   densities). While
 *   armed, rmhd_imex_step stores a checkpoint every `ckpt_every` steps and
 *   all recorded steps must use one dt. `workspace` (device, 256-byte
 *   aligned, >= rmhd_recording_bytes) may be NULL: the library allocates.
 *   Arming again drops the earlier recording (and frees the library's own
 *   workspace) first; if the new arming fails, the context is left unarmed.
 *   rmhd_adjoint_step reverses every recorded step: from dJ/dq at the final
 *   state ([N_c][ny][nx], N_c = 14 or 18) it writes dJ/d(prims) ([n_prim][ny][nx],
 *   n_prim = 11 or 16 in the layout of rmhd_set_prims, may be NULL) and
 *   dJ/dsigma (may be NULL). Two fluids: the stiff unknowns of a stage are
 *   (Sbar, taubar, E), whose transposed 7 x 7 system is solved per cell, and
 *   the primitives come from the species split and one pressure root per
 *   species (Sec. 2.1.3), both differentiated by the implicit-function theorem. Each segment of ckpt_every steps is recomputed from its
 *   checkpoint (same kernels, same results), the implicit stage solves and
 *   the primitive recovery are differentiated by the implicit-function
 *   theorem, and the WENO3/LF flux divergence is transposed face by face.
 *   The final state is restored afterwards; the recording stays valid for
 *   further adjoint calls. Synchronous.
 * (The paper has no adjoint; this serves gradient-based use of the method.)
 * Errors: RMHD_ERR_STATE (unsupported context, not armed, too many steps),
 * RMHD_ERR_INVALID, RMHD_ERR_NOMEM, RMHD_ERR_CUDA. */
int rmhd_recording_bytes(rmhd_ctx *ctx, int nsteps, int ckpt_every, size_t *bytes);
int rmhd_record(rmhd_ctx *ctx, int nsteps, int ckpt_every, void *workspace, size_t workspace_bytes);
int rmhd_adjoint_step(rmhd_ctx *ctx, const double *dJ_dcons, int where_in, double *dJ_dprims0, int where_out,
                      double *dJ_dsigma);

/* Phase-by-phase stepping (the building block of domain decomposition). One
 * IMEX step of the configured scheme is 4 phases (SSP2(222), Table 1) or 6
 * (SSP3(332), Table 2), run in order 0, 1, ...: an even phase 2k is the
 * implicit stage solve of stage k + 1 (Sec. 2.2.1, Eq. implicit stage), an odd
 * phase 2k + 1 the flux pass that follows it (WENO3/LF divergence of the
 * stage state, Sec. 2.2.2, fused with the stage combinations of the tableau).
 * dt <= 0 in phase 0 selects the CFL step; later phases take the same dt (pass
 * it again or pass 0). The phases of a step give exactly the results of
 * rmhd_imex_step. Async (enqueued on the context's stream, no CUDA graph).
 * If t_out is not NULL it receives the simulation time (advanced after the
 * last phase). rmhd_imex_step is refused while a step is half done.
 * Errors: RMHD_ERR_STATE (no state, batch, armed recording, phase out of
 * order), RMHD_ERR_INVALID, RMHD_ERR_CUDA. */
int rmhd_step_phase(rmhd_ctx *ctx, double dt, int phase, double *t_out);

/* Domain decomposition along y (the paper names multi-GPU runs as future
 * work, Sec. 3.1 and Sec. 5). A slab context holds rows [j0, j0 + ny_local)
 * of the 2-D grid described by `global` (ny_local >= 2; 1-D and 3-D grids
 * are not decomposed); its arrays are [n_var][ny_local][nx]. A side of the
 * slab is a halo side unless it is a global boundary with RMHD_OUTFLOW (a
 * periodic global grid has halo sides everywhere, also a single slab that
 * covers it all, which is then its own neighbour).
 *   Before every flux pass (odd phase of rmhd_step_phase) each halo side needs
 *   the neighbour's two rows next to it, of the neighbour's current stage
 *   state: after the even phase, rmhd_halo_pack writes a slab's first two rows
 *   (lo) and last two rows (hi) of all N_c conserved and N_w internal
 *   primitive variables to caller device buffers [N_c + N_w][2][nx]
 *   (rmhd_halo_doubles gives the length); the caller moves them (a device copy
 *   on one GPU, NCCL or peer copies across GPUs): slab s receives into its lo
 *   side the hi rows of slab s - 1 and into its hi side the lo rows of slab
 *   s + 1 (periodic: cyclically); rmhd_halo_unpack copies them into the slab
 *   (a NULL pointer, or a side without a neighbour, is skipped). pack and
 *   unpack are async on the context's stream; the caller orders the stream of
 *   a neighbour's pack before its own unpack. With exchanged halos every phase
 *   gives bit for bit the rows of the undecomposed run.
 *   A slab with a halo side is stepped only through rmhd_step_phase, takes its
 *   state from rmhd_set_cons or rmhd_set_state (rmhd_set_prims is refused:
 *   Gauss's law at its edge needs the neighbour's field) and has no adjoint.
 *   Diagnostics sum over the slab's own cells.
 * Errors: RMHD_ERR_INVALID (bad configuration or rows), RMHD_ERR_STATE (pack,
 * unpack or halo_doubles on a context that is not a slab), RMHD_ERR_NOMEM,
 * RMHD_ERR_CUDA. */
int rmhd_slab_workspace_bytes(const rmhd_config *global, int j0, int ny_local, size_t *bytes);
int rmhd_create_slab(rmhd_ctx **out, const rmhd_config *global, int j0, int ny_local, void *cuda_stream,
                     void *workspace, size_t workspace_bytes);
int rmhd_halo_doubles(const rmhd_ctx *ctx, size_t *n);
int rmhd_halo_pack(rmhd_ctx *ctx, double *lo, double *hi);
int rmhd_halo_unpack(rmhd_ctx *ctx, const double *lo, const double *hi);

/* Batched ensemble of independent 1-D runs (many tests of Sec. 4.1 at once).
 * All runs share `base` (model, x-range, Gamma, kappa, cfl, boundary
 * conditions, precision; base->ny is ignored and taken as 1); run r has
 * nx[r] cells and conductivity sigma[r] (sigma == NULL: base->sigma for all).
 * The runs are packed one after another: every array of the other calls
 * (prims, cons) has the layout [n_var][sum_r nx[r]] with run r at offset
 * sum_{s<r} nx[s]. rmhd_imex_step with dt <= 0 advances every run by its own
 * dt_r = cfl * dx_r (t_out reports run 0's time); dt > 0 uses dt for all.
 * The step runs as one CUDA graph of persistent kernels walking a work list of
 * (run, tile) pairs. rmhd_diagnostics on a batch sums over all cells without
 * a cell-volume factor. Errors as for rmhd_create. */
int rmhd_batch_workspace_bytes(const rmhd_config *base, int nruns, const int *nx, size_t *bytes);
int rmhd_create_batch(rmhd_ctx **out, const rmhd_config *base, int nruns, const int *nx, const double *sigma,
                      void *cuda_stream, void *workspace, size_t workspace_bytes);

/* Autotuner for a batched context (needs a state): times the flux tile width
 * (64, 128, 256 cells), the number of persistent CTAs and the stage-kernel
 * block size on the current state -- which it saves and restores -- keeps
 * the fastest, and writes (tile width, CTAs, stage threads) to choice[3].
 * Synchronous. Errors: RMHD_ERR_STATE for a single-grid context. */
int rmhd_autotune(rmhd_ctx *ctx, int *choice);

/* Per-kernel timing for roofline measurements (no counterpart in the paper,
 * which times whole main-loop iterations). While enabled, rmhd_imex_step
 * launches its kernels without a CUDA graph and brackets each launch with
 * CUDA events on the context's stream. rmhd_kernel_times synchronises the
 * stream, writes the summed milliseconds and launch counts per kernel kind
 * (RMHD_K_STAGE, RMHD_K_FLUX1, RMHD_K_FLUX2) into ms[3] and counts[3], and
 * clears the record. Enabling twice or disabling while off is harmless. */
#define RMHD_K_STAGE 0 /* implicit-stage solve (both stages) */
#define RMHD_K_FLUX1 1 /* flux pass after stage 1 (+ stage-2 right-hand side) */
#define RMHD_K_FLUX2 2 /* flux pass after stage 2 (+ combine + recovery) */
int rmhd_set_profiling(rmhd_ctx *ctx, int enable);
int rmhd_kernel_times(rmhd_ctx *ctx, double *ms, int *counts);

/* Measured FP64 fused multiply-add rate of the current device (no
 * counterpart in the paper; the peak against which the FP64-bound kernels of
 * the step are judged). Launches, on `cuda_stream`, independent FMA chains on
 * every SM (8 blocks of 256 threads per SM, 8 chains per thread), times them
 * with CUDA events and writes the best of three timed launches to
 * *fma_per_s (lane FMAs per second; x2 for FLOP/s) and the number of SMs to
 * *sm_count (may be NULL). Allocates no device memory. Synchronous, about
 * 0.1 s. Errors: RMHD_ERR_INVALID (fma_per_s NULL), RMHD_ERR_CUDA (a CUDA
 * error was pending on entry, or a launch or event call failed). */
int rmhd_fp64_fma_rate(void *cuda_stream, double *fma_per_s, int *sm_count);

/* Elementwise evaluation of the device arithmetic helpers the kernels use
 * (tests of their error bounds; no counterpart in the paper). For i < n,
 * out[i] = (device arrays, async on cuda_stream)
 *   RMHD_MATH_RCP    1/x[i]: approximate reciprocal refined by the series
 *                    y0 (1 + e + e^2), e = 1 - x y0; relative error ~2^-57
 *                    plus the last rounding, for 2^-1022 <= |x| <= 2^1021
 *                    (the approximation flushes subnormal inputs and results);
 *   RMHD_MATH_RSQRT  1/sqrt(x[i]): y0 (1 + e/2 + 3 e^2/8), e = 1 - x y0^2;
 *                    same accuracy, 2^-1022 <= x < 2^1024;
 *   RMHD_MATH_DIV1   a[i]/x[i] with one Newton step, t (1 + e), t = a y0:
 *                    relative error ~2^-38 (used only for WENO3 weights);
 *   RMHD_MATH_F32    x[i] rounded to FP32 on the integer pipes (nearest,
 *                    ties away from zero; FP32 subnormals included), as double;
 *   RMHD_MATH_F64    x[i] (an FP32 value held in a double) converted back by
 *                    the integer-pipe conversion (exact).
 * Errors: RMHD_ERR_INVALID (bad which, n < 0, NULL array), RMHD_ERR_CUDA. */
#define RMHD_MATH_RCP 0
#define RMHD_MATH_RSQRT 1
#define RMHD_MATH_DIV1 2
#define RMHD_MATH_F32 3
#define RMHD_MATH_F64 4
int rmhd_eval_math(int which, long long n, const double *x, const double *a, double *out, void *cuda_stream);

/* Diagnostics without any allocation (the paper has no counterpart). For
 * callers that cannot call cudaMalloc -- e.g. code running while a memory
 * pool or arena owns the device, or a framework that forbids allocation after
 * start-up -- this computes the same 7 numbers as out[0..6] of
 * rmhd_diagnostics from caller-owned device arrays, with no context:
 *   cons  [N_c][nz][ny][nx] and prims [n_prim][nz][ny][nx] (dense, device,
 *         FP64; nz = 1 for 1-D and 2-D grids, ny = 1 for 1-D),
 *   dx, dy, dz  cell widths (dy is used when ny > 1, dz when nz > 1; the
 *         sums are multiplied by the cell volume dx [dy] [dz]),
 *   out   7 doubles in device memory (written asynchronously on cuda_stream).
 * Partial sums live in a file-scope device array of 512 KiB that every GPU
 * loading the library keeps until exit; it limits inputs to 16,777,216 cells.
 * The first call on a device looks up that array's address with
 * cudaGetSymbolAddress (once per device, that device current) and caches it
 * for the life of the process; make that first call before any stream
 * capture, and do not use this call on a device after cudaDeviceReset. Calls
 * share the array: two calls whose kernels overlap on the GPU race. Calls no
 * cudaMalloc/cudaFree.
 * Errors: RMHD_ERR_INVALID (bad argument; nz > 1 needs ny > 1),
 * RMHD_ERR_NOMEM (more cells than the static array holds), RMHD_ERR_CUDA (a
 * CUDA error was already pending on entry -- it is left pending and nothing
 * is launched -- or one of this call's launches failed). */
int rmhd_diagnostics_noalloc(int model, int nx, int ny, int nz, double dx, double dy, double dz,
                             const double *cons, const double *prims, double *out, void *cuda_stream);

/* Library version string. */
const char *rmhd_version(void);

#ifdef __cplusplus
}
#endif
#endif /* RMHD_H */
