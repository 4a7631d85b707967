/*
 * libstokes: GPU solve of the pressure-stress system of one backward-Euler
 * Stokes step on a staggered grid with embedded free surfaces and solids.
 *
 * The method is the variational finite-difference discretization of
 * "A Simple Finite Difference Method for Time-Dependent, Variable
 * Coefficient Stokes Flow on Irregular Domains": velocity is eliminated from
 * the indefinite system eq. (stokesmixedsystem) to give the sparse
 * symmetric positive-definite system eq. (stokesmixedsystemspd) in the
 * deviatoric stress tau and the pressure p,
 *
 *     A x = b,  A = C + B K B^T,  B = [W_L^tau D ; W_L^p G^T],
 *     K = dt P^-1 (W_L^u)^-1 W_F^u,
 *
 * which this library builds from level sets and coefficient fields, applies
 * matrix-free, and solves with preconditioned conjugate gradients.  Units
 * are SI (Appendix A).  All entry points are plain C; all array arguments
 * are caller-owned memory of the kind stated (device = CUDA device memory on
 * the context's device, host = ordinary host memory).
 *
 * Threading and streams: a context is bound to one device and one CUDA
 * stream.  Calls on one context must not overlap from several host threads.
 * Work is enqueued on the context's stream; calls return after enqueueing
 * unless stated otherwise.
 *
 * Errors: every call returns a stokes_status; on failure the context (or,
 * for stokes_create, a thread-local slot) keeps a message readable with
 * stokes_last_error().  Arguments are validated on the host before any work
 * is enqueued; an argument error leaves the context unchanged.
 */
#ifndef STOKES_H
#define STOKES_H

#include <stdint.h>
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    STOKES_OK = 0,
    STOKES_ERR_ARG = -1,            /* invalid argument (null, size, range)   */
    STOKES_ERR_CUDA = -2,           /* a CUDA runtime call failed             */
    STOKES_ERR_NOT_CONVERGED = -3,  /* iteration cap reached above tolerance  */
    STOKES_ERR_BREAKDOWN = -4,      /* p.Ap <= 0 or r.z <= 0 in CG            */
    STOKES_ERR_TIMEOUT = -5,        /* a bounded device-side wait gave up     */
    /* -6 is not used */
    STOKES_ERR_NONFINITE = -7,      /* NaN/Inf found in an input or residual  */
    STOKES_ERR_STATE = -8           /* call out of order (e.g. no weights)    */
} stokes_status;

/* Precision of a stencil apply or of the inner solve. */
enum {
    STOKES_FP64 = 0,   /* FP64 vectors and coefficients                         */
    STOKES_FP32 = 1,   /* FP32 vectors and coefficients, FP32 arithmetic        */
    STOKES_BF16 = 2    /* FP32 vectors, BF16-stored coefficients, FP32 arithmetic */
};

/* Uniform grid of nx x ny (x nz) cells of side h, lower corner at origin.
 * dim = 2 ignores nz and origin[2].  The grid boundary is a static wall. */
typedef struct {
    int dim;
    int nx, ny, nz;
    double h;
    double dt;
    double origin[3];
} stokes_grid;

typedef struct stokes_ctx_s* stokes_ctx;

/*
 * Field layouts (caller side, "field layout"): C order, x fastest.
 *   2D: u (ny, nx+1)   v (ny+1, nx)   cells (ny, nx)   nodes (ny+1, nx+1)
 *   3D: u (nz, ny, nx+1)  v (nz, ny+1, nx)  w (nz+1, ny, nx)
 *       cells (nz, ny, nx)  tau_xy on z-edges (nz, ny+1, nx+1)
 *       tau_xz on y-edges (nz+1, ny, nx+1)  tau_yz on x-edges (nz+1, ny+1, nx)
 * Level sets live on the half lattice of spacing h/2, padded by h/2:
 *   2D (2ny+3, 2nx+3), 3D (2nz+3, 2ny+3, 2nx+3); point (a, b, c) sits at
 *   origin + ((a-1) h/2, (b-1) h/2, (c-1) h/2).
 * phi_liquid < 0 in the liquid (extended into solids); phi_solid < 0 in solids.
 */

/* Create a context for one grid on the current CUDA device.  ``stream`` is a
 * cudaStream_t; NULL makes the context create its own blocking stream, which
 * is ordered with the legacy default stream both ways (the legacy stream
 * itself cannot be captured into the solver's CUDA graphs).  Allocates all device work
 * space for the grid.  Returns STOKES_ERR_ARG for dim not in {2,3},
 * non-positive sizes, h <= 0 or dt <= 0. */
stokes_status stokes_create(stokes_ctx* out, const stokes_grid* grid, void* stream);

/* Free every resource of the context.  NULL is accepted. */
stokes_status stokes_destroy(stokes_ctx ctx);

/* Message of the last failure on this context (ctx may be NULL for the
 * calling thread's last stokes_create failure).  Never NULL. */
const char* stokes_last_error(stokes_ctx ctx);

/*
 * Weights, coefficients and validity masks (Section 5, volume fractions;
 * Section 8, null-space elimination) from device arrays in field layout:
 *   phi_liquid, phi_solid : half-lattice level sets (FP64, device)
 *   rho[d]                : density at faces of kind d = u, v(, w)  (device)
 *   mu[s]                 : viscosity at stress sites, 2D {cells, nodes},
 *                           3D {cells, z-edges, y-edges, x-edges}   (device)
 *   u_bc[d]               : prescribed solid velocity per face kind (device)
 * Every fraction, coefficient and mask is computed on the device.  rho and
 * mu must be positive where used.  The arrays are read during this call's
 * kernels only; u_bc is copied.  Enqueued on the context's stream.
 */
stokes_status stokes_build_weights(stokes_ctx ctx, const double* phi_liquid, const double* phi_solid,
                                   const double* const* rho, const double* const* mu,
                                   const double* const* u_bc);

/*
 * Floor eps (0 <= eps <= 1, default 0) of the liquid fraction of live faces
 * where it is the face's mass: from the next stokes_build_weights on, K =
 * dt W_F / (rho max(W_L, eps)) and the velocity recovery and traction use
 * the same floored fraction.  The paper (Section 5) is silent on slivers; a
 * face holding a rounding-level amount of liquid otherwise makes K and the
 * condition number arbitrarily large.  eps = 0 is the paper's system.
 * STOKES_ERR_ARG outside [0, 1].
 */
stokes_status stokes_set_min_face_liquid(stokes_ctx ctx, double eps);

/*
 * Unknown vectors use the context's internal "slot layout": every unknown
 * kind is stored on a padded copy of the (nx+1)(ny+1)(nz+1) vertex lattice,
 * one field after another (2D: tau_xx, tau_xy, p; 3D: tau_xx, tau_yy,
 * tau_xy, tau_xz, tau_yz, p).  stokes_vector_layout() returns, for element
 * size 1, the number of elements of one field (``field_stride``, guard
 * included), the pitch P, rows R, planes Q and the offset of the first
 * stored element ``base``; the sample (i, j[, k]) of field f sits at
 *     f * field_stride + base + ((k + 1) * R + (j + 1)) * P + (i + 1)   (3D)
 *     f * field_stride + base + (j + 1) * P + (i + 1)                   (2D)
 * and every other element is padding that must be zero on input.
 * ``total`` = nfields * field_stride elements per vector.
 */
typedef struct {
    int nfields;
    int64_t field_stride;
    int64_t base;
    int pitch, rows, planes;
    int64_t total;
} stokes_layout;

stokes_status stokes_vector_layout(stokes_ctx ctx, stokes_layout* out);

/*
 * y = A x, matrix-free (eq. stokesmixedsystemspd in the factored form of
 * Section 7: face values z = K B^T x, then y = B z + C x).  x, y are device
 * vectors in slot layout of element type double (STOKES_FP64) or float
 * (STOKES_FP32, STOKES_BF16).  Inactive unknowns act as the identity.
 * Requires stokes_build_weights.  x and y must not alias.  Any element
 * alignment is accepted; in 2D, float vectors that both start on a 16-byte
 * boundary are read and written 16 bytes at a time (the faster kernel).
 */
stokes_status stokes_apply(stokes_ctx ctx, const void* x, void* y, int precision);

/* Right-hand side b (FP64 slot layout, device) of eq. stokesmixedsystemspd
 * with the prescribed-velocity terms of Section 6.2, for input velocity
 * u_star[d] (device, field layout). */
stokes_status stokes_rhs(stokes_ctx ctx, const double* const* u_star, double* b);

/* Velocity recovery (first block row of eq. stokesmixedsystem) from a
 * solution x (FP64 slot layout, device) into u_out[d] (device, field
 * layout): live faces u* - dt/(rho W_L) (B^T x); faces with zero effective
 * fluid weight u_BC; fluid faces without liquid u*. */
stokes_status stokes_recover(stokes_ctx ctx, const double* const* u_star, const double* x,
                             double* const* u_out);

typedef struct {
    int mode;          /* STOKES_FP64: FP64 PCG; STOKES_FP32 / STOKES_BF16:
                          inner PCG in that precision inside FP64 iterative
                          refinement                                         */
    double tol;        /* target true relative residual ||b-Ax||/||b||       */
    int max_iter;      /* cap on total (inner) CG iterations                */
    double inner_tol;  /* relative tolerance of each inner solve (mixed)    */
    int max_outer;     /* cap on refinement steps (mixed)                    */
    int check_every;   /* iterations between host convergence checks        */
    int precond;       /* 0 = Jacobi (point diagonal); 1 = learned network
                          (flexible CG, see stokes_set_learned_preconditioner);
                          2 = additive Schwarz, 2D: overlapping patches of
                          4x4 slots plus a one-slot ring, exact local solves
                          (inverse factors stored in FP16 with a FP32 scale
                          per row, FP32 inner CG)                             */
    int use_graph;     /* 1: CG loop in a device-side CUDA graph (conditional
                          while node); 0: host-driven chunks of check_every
                          iterations launched one kernel at a time (for
                          profilers that cannot enter conditional graphs)   */
    int wait_test;     /* test hook for the bounded device-side waits, 0 in
                          normal use.  1 (precond = 2, mixed mode): the
                          Schwarz local solves wait for a factor copy that is
                          never issued, giving up after 1,024 polls, so the
                          call returns STOKES_ERR_TIMEOUT and the context
                          stays usable.                                     */
} stokes_options;

typedef struct {
    int status;              /* stokes_status of the solve                  */
    int iterations;          /* total CG iterations (inner ones if mixed)   */
    int outer;               /* refinement steps (mixed), 1 for FP64 PCG    */
    double rel_residual;     /* final true relative residual in FP64        */
    double ms_rhs, ms_solve, ms_recover;  /* device time per phase          */
    int precision_used;      /* inner precision of the last refinement step:
                                a refinement step that does not reduce the
                                FP64 residual is undone and the inner solve
                                moves up one precision (BF16 -> FP32 -> FP64) */
} stokes_stats;

/* Fill ``o`` with defaults: FP64 mode, tol 1e-8, max_iter 200000,
 * inner_tol 1e-4, max_outer 40, check_every 64, Jacobi, wait_test 0. */
void stokes_default_options(stokes_options* o);

/*
 * Prescribed surface pressure p_BC and deviatoric stress tau_BC (Section 6.1,
 * a traction boundary such as surface tension): writes to u_star_out[d] the
 * u* to pass to stokes_solve_step.  The section's force enters the first
 * block row of eq. stokesmixedsystem weighted like the mass term, so on live
 * faces u*_out = u* + dt/(rho W_L^u) f with
 *   f = W_A^u (M^T x_BC) - M^T (W_A x_BC),  M^T = [D^T | G],
 * W_A = 1 - W_L the air fraction of each sample (1 for eliminated unknowns),
 * x_BC = (tau_BC, p_BC); elsewhere u*_out = u*.  The sign is the opposite of
 * the one printed: with it a uniform p_BC = P0 on liquid at rest gives the
 * liquid pressure P0 (the printed sign gives -P0).  tau_bc[s] (stress kinds
 * in slot-field order) and p_bc use the layout of stokes_solve_step's
 * tau_out and p_out; all device arrays; u_star_out may be u_star.  Uses the
 * solver's work vectors (do not overlap with a solve on this context).
 */
stokes_status stokes_traction_u_star(stokes_ctx ctx, const double* const* tau_bc, const double* p_bc,
                                     const double* const* u_star, double* const* u_star_out);

/*
 * Transport stage of the fractional-step Navier-Stokes routine around the
 * implicit Stokes step (Section "Application to Viscous Jet Buckling"), 2D
 * only: from u^n build u* = (first-order semi-Lagrangian advection of u^n
 * with bilinear interpolation) + dt * gravity, and advect the liquid level
 * set with the same velocity (basic semi-Lagrangian level set).
 *   u_in[d], u_out[d] : u^n and u* per face kind, FP64 device, field layout;
 *                       u_out may equal u_in (the velocity is staged)
 *   phi_in, phi_out   : liquid level set on the half lattice (FP64 device);
 *                       phi_in NULL skips the level set; phi_out must not
 *                       overlap phi_in
 *   gravity[2]        : body acceleration (host), added as dt * gravity
 *   ext_passes        : Jacobi sweeps extending the velocity into faces that
 *                       are not valid: each sweep gives such a face the mean
 *                       of its valid 4-neighbours of the same component (left,
 *                       right, below, above) and makes it valid
 *   valid             : one byte per face (u then v, field layout, nonzero =
 *                       valid), or NULL: valid faces are then those that are
 *                       not fluid-without-liquid in the weights last built on
 *                       this context (live faces and faces holding u_BC)
 *   phi_union         : NULL, or a half-lattice level set of a source region
 *                       (an inflow): phi_out = min(advected phi, phi_union)
 * Positions are in grid units: u face (i, j) at (i, j + 1/2), v face (i, j)
 * at (i + 1/2, j), lattice point (a, b) at ((a - 1)/2, (b - 1)/2); a
 * departure point X - (dt/h) u(X) outside a field's samples is clamped onto
 * them.  dt and h are the context's.  Enqueued on the context's stream; the
 * first call allocates (nu + nv) * 18 bytes of scratch on the context.
 * Errors: STOKES_ERR_ARG (3D, nx or ny < 2, null or aliased arrays),
 * STOKES_ERR_STATE (valid NULL before any weight build), STOKES_ERR_CUDA.
 */
stokes_status stokes_advect(stokes_ctx ctx, const double* const* u_in, const double* phi_in, const double* gravity,
                            int ext_passes, const uint8_t* valid, const double* phi_union, double* const* u_out,
                            double* phi_out);

/*
 * One implicit step (the hot path): b from u*, solve A x = b to the
 * requested true relative residual, recover u.  Inputs u_star[d] and outputs
 * u_out[d], tau_out[s] (stress kinds in slot-field order without p) and
 * p_out are device arrays in field layout; inactive unknowns come out 0.
 * Synchronises the context's stream once at the end to fill ``stats``
 * (may be NULL).  Returns STOKES_ERR_NOT_CONVERGED with the best x found if
 * the caps are reached first.  A grid with no active unknown (no liquid)
 * has an empty system: the call returns STOKES_OK after 0 iterations with
 * x = 0 (u = u_BC on solid faces, u* elsewhere).
 */
stokes_status stokes_solve_step(stokes_ctx ctx, const double* const* u_star, double* const* u_out,
                                double* const* tau_out, double* p_out, const stokes_options* opt,
                                stokes_stats* stats);

/* Solve A x = b for a given right-hand side (FP64 slot layout, device);
 * x (same layout) is overwritten.  Same options and statistics. */
stokes_status stokes_solve_system(stokes_ctx ctx, const double* b, double* x, const stokes_options* opt,
                                  stokes_stats* stats);

/*
 * Export of the weights for checking: ``what`` selects
 *   0: W_L per sample kind, 1: W_F per sample kind (FP64, kinds in the order
 *      2D {cell, node, u, v}, 3D {cell, u, v, w, exy, exz, eyz}, each in field
 *      layout, concatenated);
 *   2: face flags (one byte per face, field layout, u then v (then w)):
 *      bit0 live, bit1 bad, bit2 invalid (solid side), bit3 on the wall;
 *   3: unknown activity (one byte per unknown, stress kinds then p, field
 *      layout).
 * ``out`` is a device buffer of at least stokes_export_size() bytes.
 */
stokes_status stokes_export(stokes_ctx ctx, int what, void* out);
int64_t stokes_export_size(stokes_ctx ctx, int what);

/* Copy an unknown vector between slot layout (FP64) and field layout
 * (concatenation of the stress fields then p, FP64).  Device pointers. */
stokes_status stokes_slots_to_fields(stokes_ctx ctx, const double* slots, double* fields);
stokes_status stokes_fields_to_slots(stokes_ctx ctx, const double* fields, double* slots);

/* Device time (ms) of the last stokes_apply call, measured with CUDA events
 * on the context's stream (synchronises).  Returns -1 if none. */
double stokes_last_apply_ms(stokes_ctx ctx);

/* Measurement support: run ``launches`` real CG iterations (right-hand side
 * = the last one stokes_solve_step built, Jacobi, inner precision
 * ``precision``) launch by launch, outside any graph, with CUDA events
 * around each kernel on the context's stream; return the mean device time
 * (ms) of the CG-mode apply kernel (direction update, A p and p.Ap fused)
 * and of the vector-update kernel.  Overwrites the solver's work vectors.
 * Synchronises. */
/* Measurement support for the Schwarz path (2D): ``launches`` times the two
 * preconditioner kernels of an FP32 Schwarz-CG iteration (right-hand side =
 * the last one stokes_solve_step built), CUDA events around each on the
 * context's stream; mean device ms of the local patch solves and of the
 * gather (z, r.z, r.r); *bytes_local = algorithmic bytes of one local-solve
 * launch (every active patch's stored factor X = L^-1, its residual gather,
 * scaling, local map and results).  Builds the patch factors if needed.
 * Overwrites the solver's work vectors.  Synchronises. */
stokes_status stokes_bench_schwarz_kernels(stokes_ctx ctx, int launches, double* ms_local, double* ms_gather,
                                           double* bytes_local);
stokes_status stokes_bench_cg_kernels(stokes_ctx ctx, int precision, int launches, double* ms_apply,
                                      double* ms_update);

/*
 * Batched solve of many independent 2D systems of uneven size (one context
 * per instance, weights already built) in one persistent cooperative kernel
 * replayed from a CUDA graph: right-hand sides, FP64 Jacobi-PCG of every
 * instance with its own scalars and stopping test (true relative residual
 * <= opt->tol, verified in FP64 before an instance retires), recovery and
 * output unpacking.  All device waits inside the kernel are bounded; a wait
 * that gives up returns STOKES_ERR_TIMEOUT.
 *
 * stokes_batch_create plans the batch (per-instance tile lists) and picks
 * the tile height (4, 8 or 16 rows of 32 slots) and CTAs per SM by timing
 * every candidate (an autotuner), caching the choice in a text file (path
 * ``tune_cache``, else $STOKES_AUTOTUNE_CACHE, else
 * $HOME/.cache/libstokes_autotune.txt) keyed by instance count, problem
 * size class and GPU name.  The contexts must stay alive and unchanged
 * (no new stokes_build_weights) for the life of the batch.
 * stokes_batch_solve enqueues on the batch's own stream and synchronises;
 * ``stats`` (n entries, may be NULL) receive per-instance results and
 * ``ms`` (may be NULL) the device time of the whole batched step.
 * The graph is re-captured when the io pointers change.
 */
typedef struct {
    const double* u_star[3];   /* device, field layout (2D: u, v)          */
    double* u_out[3];          /* device, field layout                     */
    double* tau_out[5];        /* device, field layout (2D: tau_xx, tau_xy) */
    double* p_out;             /* device, cells                             */
} stokes_batch_io;

typedef struct stokes_batch_s* stokes_batch;

stokes_status stokes_batch_create(stokes_batch* out, int n, const stokes_ctx* ctxs, const stokes_options* opt,
                                  const char* tune_cache);
stokes_status stokes_batch_solve(stokes_batch b, const stokes_batch_io* io, stokes_stats* stats, double* ms);
stokes_status stokes_batch_destroy(stokes_batch b);
/* Tuning picked for the batch: tile rows, CTAs per SM, time per iteration
 * (us) measured by the tuner, and whether the step runs from a captured
 * graph (1) or from direct launches (0). */
stokes_status stokes_batch_tuning(stokes_batch b, int* tile_rows, int* ctas_per_sm, double* us_per_iter,
                                  int* graph_captured);
/* One-shot convenience: create, solve once, destroy. */
stokes_status stokes_solve_batched(int n, const stokes_ctx* ctxs, const stokes_batch_io* io,
                                   const stokes_options* opt, stokes_stats* stats);

/*
 * Learned preconditioner network (not in the paper: a data-driven
 * preconditioner for the CG solve).  A three-level U-Net on the slot lattice
 * (convolutions 3x3 in 2D, 3x3x3 in 3D, widths 8/16/32, ReLU, 2x average
 * pooling, nearest upsampling, skip concatenation, 1x1 output).  Activations
 * are BF16, accumulation and master weights FP32.  Tensors passed in are FP32
 * device arrays, channel-last (B, D, H, W, C) with D = 1 in 2D, H and W
 * multiples of 4 (D too in 3D); ``cin`` and ``cout`` must be one of 4, 8,
 * 12, 16.  The convolutions run on the tensor cores with BF16 operands
 * (activations, weights, and output gradients in the backward pass) and
 * FP32 accumulation; a gradient is bit-reproducible.  The flat parameter vector holds, per convolution in
 * the order enc0a enc0b enc1a enc1b enc2a enc2b dec1a dec1b dec0a dec0b out,
 * the weights W[tap][cin][cout] then the bias (stokes_net_layer gives the
 * offsets).  All calls run on the network's own stream and synchronise.
 */
typedef struct stokes_net_s* stokes_net;

stokes_status stokes_net_create(stokes_net* out, int dim, int cin, int cout, int64_t max_voxels);
stokes_status stokes_net_destroy(stokes_net net);
int64_t stokes_net_param_count(stokes_net net);
stokes_status stokes_net_layer(stokes_net net, int i, int* cin, int* cout, int* ksize, int64_t* w_off,
                               int64_t* b_off);
stokes_status stokes_net_set_params(stokes_net net, const float* host_params);
stokes_status stokes_net_get_params(stokes_net net, float* host_params);
stokes_status stokes_net_forward(stokes_net net, int B, int D, int H, int W, const float* x, float* y);
/* loss = mean over the batch of ||N(x_b) - y_b||^2 / ||y_b||^2 (a sample with
 * y_b = 0 contributes 0), and its gradient with respect to the parameters
 * (copied to grad_host if given). */
stokes_status stokes_net_gradient(stokes_net net, int B, int D, int H, int W, const float* x, const float* y,
                                  double* loss, float* grad_host);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on that loss. */
stokes_status stokes_net_train_step(stokes_net net, int B, int D, int H, int W, const float* x, const float* y,
                                    float lr, double* loss);

/*
 * Learned preconditioner for a context.  The network sees, per slot (i, j[, k])
 * at voxel (k, j, i) of a grid padded to multiples of 4 (stokes_learned_grid),
 * the Jacobi-scaled residual sqrt(m_f) r_f normalised to unit RMS over the
 * active unknowns, and log(m_f)/16 (m = inverse diagonal of A), one channel
 * per unknown field each, zero-padded to cin = 8 (2D) or 12 (3D); its output
 * channels (cout = 4 or 8) correct the Jacobi step:
 * z_f = m_f r_f + sqrt(m_f) out_f rms on active unknowns (z = r on inactive
 * ones), so a zero network is plain Jacobi.  With options.precond = 1
 * (mode FP32 or BF16) the inner solve is flexible CG (Polak-Ribiere beta)
 * with this preconditioner, falling back to the Jacobi direction for a step
 * whose network direction fails r.z > 0, and to plain Jacobi-PCG for the rest
 * of an inner solve whose residual norm does not halve within 100 iterations,
 * inside the same FP64 refinement loop.  Re-attach after every
 * stokes_build_weights.
 */
stokes_status stokes_set_learned_preconditioner(stokes_ctx ctx, stokes_net net);
stokes_status stokes_learned_grid(stokes_ctx ctx, int* D, int* H, int* W, int* cin, int* cout);
/* Network input for an FP64 slot-layout residual r (device) into x (device,
 * FP32, D*H*W*cin); *rms receives the normalisation used. */
stokes_status stokes_learned_features(stokes_ctx ctx, const double* r, float* x, double* rms);
/* Training target for an FP64 slot-layout vector e with the rms of its
 * residual: y_f = e_f / (sqrt(m_f) rms) on active unknowns, 0 elsewhere.
 * For the preconditioner above, pass e = err - M_J A err (the part of the
 * error err that the Jacobi step misses). */
stokes_status stokes_learned_targets(stokes_ctx ctx, const double* e, double rms, float* y);
/* Steps at which the flexible CG fell back to the Jacobi direction. */
long stokes_learned_jacobi_steps(stokes_ctx ctx);

/* z = M^-1 r for FP32 slot-layout device vectors: which = 0 Jacobi
 * (z = r / diag A, z = r on inactive unknowns), 2 additive Schwarz (2D):
 * z = sum_p R_p^T A_p^-1 R_p r over overlapping patches (4x4-slot core plus a
 * one-slot ring, the patch's active unknowns), inactive unknowns z = r.  The
 * Schwarz patch inverses are built on first use after each weight build
 * (stokes_schwarz_setup_ms reports the device time of that build, -1 if
 * none). */
stokes_status stokes_apply_preconditioner(stokes_ctx ctx, int which, const float* r, float* z);
double stokes_schwarz_setup_ms(stokes_ctx ctx);
/* Allocation-free form of stokes_apply_preconditioner(ctx, 2, r, z); the
 * paper has no counterpart (it is an interface for callers that cannot
 * allocate device memory while they run: a process whose device memory is
 * reserved up front by its own pool, or a real-time loop that cannot accept
 * the device-wide synchronisation of cudaMalloc/cudaFree).  Same arguments,
 * layout and result; it allocates nothing, host or device: its scratch is a
 * fixed 8 MiB device array inside the library, which bounds 2D grids to
 * 555^2 (larger grids: STOKES_ERR_ARG with the sizes in stokes_last_error).
 * The context's Schwarz plan must already exist (an earlier
 * stokes_apply_preconditioner(ctx, 2, ...) or a solve with precond = 2 after
 * the last weight build), else STOKES_ERR_STATE.  The context's device must
 * be the current device (else STOKES_ERR_ARG): the array's address is looked
 * up on the first call on each device, with that device current.  Each call
 * reads a status word back and synchronises the context's stream.  Calls
 * share the array: calls that overlap on the GPU race.  The result z is
 * bit-identical to stokes_apply_preconditioner(ctx, 2, r, z). */
stokes_status stokes_apply_schwarz_noalloc(stokes_ctx ctx, const float* r, float* z);

/* Number of tiles holding an active unknown (2D tiles are 32 x 8 slots,
 * 3D tiles 32 x 4 x 4); every CG kernel launches one CTA per such tile. */
int stokes_active_tiles(stokes_ctx ctx);

#ifdef __cplusplus
}
#endif
#endif /* STOKES_H */
