/*
 * tsfem.h -- C ABI of the GB300 two-scale finite element library.
 *
 * The library advances, one implicit Euler step at a time, the coupled
 * macro/micro system of Lakkis, Muntean, Richardson and Venkataraman
 * ("Parallel two-scale finite element implementation of a system with varying
 * microstructure"): a macroscopic field u on Omega = [0,1]^2 and one
 * microscopic field v_i per macroscopic node x_i (Sec. 3.3: one micro system
 * per macro degree of freedom, located at its support point).  Every micro
 * problem lives on the shared reference cell Z = [0,1]^2 and sees the
 * geometry of its own cell Y_{x_i} = chi(x_i, Z) only through pulled-back
 * coefficients (Sec. 3.1, Eqs. (13)-(16)):
 *
 *   J = det F,  C = J F^{-1} D F^{-T},  s = |cof(F) nu|,   F = D_yhat chi.
 *
 * One step solves (u-v part of the model system Eq. (5), with a time
 * derivative added to both equations; discrete form Eq. (17)):
 *
 *   (M_i/dt + A_i + kappa R_i) v_i - kappa r_i u_i = M_i (v_i^n/dt + fv_i) + R_i g_i
 *   (M_H/dt + Du K_H + kappa L Gam) u - kappa L rho(v) = M_H (u^n/dt + fu) - L G
 *
 * with Q1 elements on uniform square meshes, 2x2 Gauss quadrature, the Robin
 * (inflow) edge yhat_1 = 1 of Z, homogeneous Neumann data on the other micro
 * edges, r_i = R_i 1, |Gam_i| = 1^T r_i, L = diag(row sums of M_H),
 * rho(v)_i = r_i^T v_i and G_i = r_i^T g_i.  The coupled step is solved by
 * the partitioned fixed-point iteration of Sec. 3.3 (all micro problems with
 * the current u, then the macro problem with the new micro fluxes) until the
 * relative change of u is below a tolerance.
 *
 * Node numbering (both meshes): node (p, q) of an N x N cell mesh has index
 * p + (N+1) q and sits at (p, q)/N.  Micro fields are stored instance-major:
 * v[i * nm + j], nm = (Nm+1)^2.
 *
 * Conventions for every entry point:
 *  - Pointers flagged "on_device" are CUDA device pointers of the current
 *    device, otherwise host pointers.  The library copies what it reads and
 *    never keeps a caller pointer after the call returns (except a workspace
 *    bound with tsf_bind_workspace, which the caller keeps alive).
 *  - All work is enqueued on the stream given in tsf_options.cuda_stream
 *    (NULL = a stream the library creates).  Setters and tsf_step return
 *    once the work is enqueued; getters synchronise that stream.
 *  - Every function returns a tsf_status and never aborts the process; on an
 *    error tsf_last_error() describes it.  Device-side outcomes of tsf_step
 *    (a solve that did not converge, a NaN) are reported by
 *    tsf_synchronize() and tsf_get_stats().
 */
#ifndef TSFEM_H
#define TSFEM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tsf_ctx tsf_ctx;

typedef enum tsf_status {
    TSF_OK = 0,
    TSF_E_ARG = 1,           /* invalid argument (sizes, family, NULL pointer, ...) */
    TSF_E_STATE = 2,         /* call out of order (e.g. step before meshes were set) */
    TSF_E_BAD_JACOBIAN = 3,  /* det F <= 0 at a quadrature point (Eq. (3) requires det F > 0) */
    TSF_E_NOT_CONVERGED = 4, /* a CG solve or the coupling iteration hit its iteration cap */
    TSF_E_NAN = 5,           /* a non-finite value appeared in a solve */
    TSF_E_CUDA = 6,          /* a CUDA runtime call failed */
    TSF_E_OOM = 7,           /* device memory allocation failed or workspace too small */
    TSF_E_BREAKDOWN = 8,     /* p^T A p <= 0 in a CG solve (operator not SPD) */
    TSF_E_TIMEOUT = 9        /* a device-side wait (an asynchronous copy into shared memory) did not
                                complete within its bound; the results of that step are not valid */
} tsf_status;

/* arithmetic of the micro solves */
enum {
    TSF_FP64 = 0,  /* Jacobi-PCG in FP64 */
    TSF_MIXED = 1  /* FP32 Jacobi-PCG inner solves inside iterative refinement with an
                      FP64-accurate residual.  The column-strip variants keep that residual
                      in float-float arithmetic (pairs of FP32 numbers, about 2^-44) and
                      scale their FP32 norms per micro problem by a power of two, so the
                      relative tolerance has no FP32 range limit; under the pipelined
                      elimination their state is held in FP32 pairs, which represent values
                      down to about 1e-37 (a micro problem whose right-hand side is smaller
                      is solved to that absolute level). */
};

/* deformation families chi(x_i, .) : Z -> Y_{x_i} (Sec. 2, Eqs. (2)-(3)) and their
 * per-node parameters */
enum {
    TSF_FAMILY_IDENTITY = 0,    /* chi = yhat;                                     0 params */
    TSF_FAMILY_BUMP = 1,        /* chi = yhat + a (sin pi y1 sin pi y2, 0);        1: a */
    TSF_FAMILY_SHEAR_BUMP = 2,  /* chi = (y1 + s y2 + b sin pi y1 sin pi y2, y2);  2: s, b */
    TSF_FAMILY_AFFINE = 3,      /* chi = A yhat + c;   6: A11, A12, A21, A22, c1, c2 */
    TSF_FAMILY_AFFINE_BUMP = 4  /* chi = A yhat + b (sin pi y1 sin pi y2, 0); 5: A11, A12, A21, A22, b */
};

/* macroscopic boundary condition */
enum { TSF_BC_NEUMANN = 0, TSF_BC_DIRICHLET = 1 };

typedef struct tsf_options {
    int precision;           /* TSF_FP64 or TSF_MIXED */
    double cg_tol;           /* micro solves: stop when ||b - A v||_2 <= cg_tol ||b||_2 (FP64 residual) */
    double inner_tol;        /* TSF_MIXED: relative tolerance of each FP32 inner solve */
    double macro_tol;        /* macro solve: relative residual tolerance */
    double coupling_tol;     /* stop the coupling iteration when ||u_new - u||_2 <= coupling_tol ||u_new||_2 */
    int cg_maxit;            /* cap on CG iterations per micro solve (inner iterations summed over sweeps) */
    int max_sweeps;          /* TSF_MIXED: cap on refinement sweeps per micro solve */
    int macro_maxit;         /* cap on macro CG iterations */
    int coupling_maxit;      /* cap on coupling iterations per step */
    int tiling;              /* -1: library choice; >= 0 fixed micro-kernel variant (see tsf_stats.tiling) */
    int use_graph;           /* 1: each step is one CUDA graph launch with a device-controlled
                                coupling loop; 0: kernels launched one by one */
    void *cuda_stream;       /* cudaStream_t to enqueue on, NULL = library-owned stream */
    int profile;             /* 1 (with use_graph = 0): time every micro and macro kernel launch
                                with CUDA events on the stream; totals in tsf_stats */
    int coupling;            /* how a step reaches the coupled fixed point:
                                TSF_COUPLING_PARTITIONED: the partitioned iteration of Sec. 3.3
                                  (micro solves with the current u, macro solve with the new
                                  fluxes, until coupling_tol);
                                TSF_COUPLING_ELIMINATION: exact elimination.  Given u_i the micro
                                  solution is affine in u_i, v_i = v0_i + u_i phi_i with
                                  S_i phi_i = kappa r_i independent of the state, so the fluxes
                                  are rho_i = r_i^T v0_i + u_i r_i^T phi_i and one macro solve with
                                  the diagonal kappa m_i (|Gam_i| - r_i^T phi_i) gives u; one micro
                                  solve per step (phi is solved once per geometry and dt, to
                                  1e-3 cg_tol, at least 1e-13).  Same discrete solution, without
                                  the coupling tolerance; coupling_tol and coupling_maxit unused. */
} tsf_options;

enum { TSF_COUPLING_PARTITIONED = 0, TSF_COUPLING_ELIMINATION = 1 };

typedef struct tsf_stats {
    int64_t inner_iters;        /* CG iterations summed over micro instances, solves and steps */
    int64_t dof_cg_iters;       /* inner_iters * nm: micro DOF-CG-iterations */
    int64_t refine_sweeps;      /* FP64 residual evaluations of the micro problems (summed over instances) */
    int64_t micro_solves;       /* micro solves (instances x coupling iterations) */
    int64_t macro_iters;        /* macro CG iterations */
    int coupling_iters_last;    /* coupling iterations of the last step */
    int coupling_iters_total;
    int max_inner_iters;        /* largest inner-iteration count of a single micro solve */
    int steps;                  /* steps taken since the last tsf_reset_stats */
    int status;                 /* first device-side error (tsf_status), TSF_OK if none */
    int tiling;                 /* micro-kernel variant in use: 0..3 shared-memory stencil with
                                   1, 2, 4, 8 nodes per thread (FP64 or mixed); 4..6 column strips
                                   of 3, 5, 7 nodes with the stencil in registers (mixed); 7..9
                                   column strips of 9, 11, 13 nodes with the stencil in shared
                                   memory (mixed); 10 is the three-field direct solve
                                   (tsfem3.h); 11..14 one micro problem per thread-block cluster
                                   of G CTAs with column strips of R nodes, (R, G) = (5, 2),
                                   (5, 4) stencil in registers, (9, 4), (9, 8) stencil in shared
                                   memory (mixed); 15, 16 one warp per micro problem with
                                   strips of 3, 5 nodes, for micro meshes whose strips fit 32
                                   threads (mixed) */
    double coupling_change;     /* final ||du|| / ||u|| of the last step */
    int64_t micro_launches;     /* profiled micro-solve kernel launches */
    int64_t macro_launches;     /* profiled macro-solve kernel launches */
    double micro_kernel_ms;     /* summed CUDA-event time of the profiled micro-solve launches */
    double macro_kernel_ms;     /* summed CUDA-event time of the profiled macro-solve launches */
} tsf_stats;

/* Fill *opt with defaults: TSF_MIXED, cg_tol 1e-8, inner_tol 1e-5, macro_tol 1e-12,
 * coupling_tol 1e-10, cg_maxit 5000, max_sweeps 20, macro_maxit 500, coupling_maxit 50,
 * tiling -1, use_graph 1, cuda_stream NULL, profile 0, coupling TSF_COUPLING_PARTITIONED. */
void tsf_default_options(tsf_options *opt);

/* Create a context.  opt may be NULL (defaults).  *out receives the handle.
 * Errors: TSF_E_ARG (out NULL, bad option), TSF_E_CUDA (no device / stream). */
tsf_status tsf_create(tsf_ctx **out, const tsf_options *opt);

/* Replace the options of an existing context (stream excluded). */
tsf_status tsf_set_options(tsf_ctx *ctx, const tsf_options *opt);

/* Reference micro mesh on Z = [0,1]^2 (Sec. 3.1: one mesh of the reference
 * domain, shared by all micro problems).  nx = ny = Nm cells per side,
 * 1 <= Nm <= 128.  Up to 64 cells a micro problem is solved by one thread
 * block; the mixed-precision cluster variants (tiling 11..14) spread one
 * micro problem over a thread-block cluster and are the only variants beyond
 * 64 cells (TSF_FP64 takes at most 64).  robin_edge must be 0 (the edge
 * yhat_1 = 1).  Errors: TSF_E_ARG. */
tsf_status tsf_set_micro_mesh(tsf_ctx *ctx, int nx, int ny, int robin_edge);

/* Macro mesh on Omega = [0,1]^2 with nx = ny = NM cells per side
 * (1 <= NM <= 1023), hence nM = (NM+1)^2 micro problems.  bc: TSF_BC_NEUMANN
 * (homogeneous, whole boundary) or TSF_BC_DIRICHLET (whole boundary);
 * dirichlet_vals: host array of nM values read on boundary nodes, NULL keeps
 * the current state there.  Errors: TSF_E_ARG. */
tsf_status tsf_set_macro_mesh(tsf_ctx *ctx, int nx, int ny, int bc, const double *dirichlet_vals);

/* Micro diffusion D = [[D11, D12], [D12, D22]] (symmetric positive definite),
 * Robin transfer coefficient kappa >= 0 (kappa_1 = kappa_2 = kappa in Eq. (5)),
 * macro diffusion macro_diff > 0.  Errors: TSF_E_ARG. */
tsf_status tsf_set_physics(tsf_ctx *ctx, const double D[3], double kappa, double macro_diff);

/* Per-node deformation parameters params[i * nparam + k], i < nM, for the
 * given family (nparam must match it).  Computes the pulled-back Q1 operators
 * of every micro problem on the device and validates det F > 0 at every
 * quadrature point (TSF_E_BAD_JACOBIAN otherwise).  Requires both meshes. */
tsf_status tsf_set_deformation(tsf_ctx *ctx, int family, int nparam, const double *params, int params_on_device);

/* State: u[nM] and v[nM * nm] (NULL = zero micro field). */
tsf_status tsf_set_state(tsf_ctx *ctx, const double *u, const double *v, int on_device);

/* Nodal source data used by the following steps (each may be NULL = zero):
 *   fv[nM * nm]        micro volume source at the micro nodes,
 *   g[nM * (Nm+1)]     Robin data at the Robin-edge nodes yhat = (1, q/Nm),
 *   fu[nM]             macro volume source,
 *   ud[nM]             Dirichlet values (read on boundary nodes when bc = Dirichlet).
 * Load vectors are mass (resp. boundary-mass) matrices times nodal values. */
tsf_status tsf_set_sources(tsf_ctx *ctx, const double *fv, const double *g, const double *fu, const double *ud,
                           int on_device);

/* Advance nsteps implicit Euler steps of size dt > 0.  Enqueued on the stream;
 * returns TSF_OK once enqueued.  Requires meshes, deformation and state. */
tsf_status tsf_step(tsf_ctx *ctx, double dt, int nsteps);

/* Wait for the stream; returns the first device-side error of the steps
 * since the last tsf_reset_stats (TSF_OK if none). */
tsf_status tsf_synchronize(tsf_ctx *ctx);

/* Getters (synchronise the stream): macro field u[nM]; micro averages
 * vbar_i = int_{Y_x_i} v / |Y_x_i| = 1^T M_i v_i / vol_i; micro fields
 * v[nM * nm]; boundary fluxes F_i = kappa (|Gam_i| u_i - r_i^T v_i) + G_i;
 * geometry |Gam_i| and |Y_x_i|. */
tsf_status tsf_get_macro(tsf_ctx *ctx, double *u_out, int on_device);
tsf_status tsf_get_micro_averages(tsf_ctx *ctx, double *vbar_out, int on_device);
tsf_status tsf_get_micro_field(tsf_ctx *ctx, double *v_out, int on_device);
tsf_status tsf_get_flux(tsf_ctx *ctx, double *flux_out, int on_device);
/* Coupling moments rho_i = r_i^T v_i of the current micro fields (the Robin
 * boundary integral of v_i that enters the macro equation, Eq. (17) and
 * Sec. 3.3), rho_out[nM], summed with compensated (TwoSum) FP64 arithmetic.
 * tsf_get_flux returns kappa (|Gam_i| u_i - rho_i) + G_i from the same sum;
 * rho itself does not cancel, so it is the quantity to compare at tight
 * tolerances.  Synchronises the stream.  Errors: TSF_E_ARG, TSF_E_STATE. */
tsf_status tsf_get_rho(tsf_ctx *ctx, double *rho_out, int on_device);
tsf_status tsf_get_geometry(tsf_ctx *ctx, double *gamma_out, double *vol_out, int on_device);

/* Asynchronous variants of tsf_get_macro and tsf_get_micro_averages for
 * streaming results out while the next steps run: the copy is enqueued on
 * the context's stream behind the work already there, and the call returns
 * without synchronising.  The destination holds the values once the stream
 * reaches the copy (after tsf_synchronize, or an event recorded behind it);
 * a host destination must be page-locked memory for the copy to be
 * asynchronous and must stay valid until then. */
tsf_status tsf_get_macro_async(tsf_ctx *ctx, double *u_out, int on_device);
tsf_status tsf_get_micro_averages_async(tsf_ctx *ctx, double *vbar_out, int on_device);

/* Push-forward of the micro fields for visualisation (Sec. 3.6: every micro
 * solution is mapped from the reference cell Z to its physical cell Y_x and
 * translated to its macroscopic location, scaled so that the cells can be
 * told apart).  Micro node j of the micro problem at macro node i (reference
 * point yhat_j = (p, q)/Nm, macro point x_i on [0,1]^2) goes to
 *     X = x_i + scale (chi(x_i, yhat_j) - (1/2, 1/2)),
 * chi the deformation map of tsf_set_deformation (shift of the affine family
 * included).  out[(i nm + j) 3 + {0, 1, 2}] = (X1, X2, v_i(yhat_j)): nM x nm
 * x 3 floats (FP32, for pictures), host (on_device = 0) or device.  scale > 0
 * (for instance 0.8 / NM).  With a host buffer the call allocates and frees a
 * device buffer of the same size.  Synchronises the stream.  Errors:
 * TSF_E_ARG, TSF_E_STATE (no deformation), TSF_E_OOM, TSF_E_CUDA. */
tsf_status tsf_get_pushforward(tsf_ctx *ctx, float scale, float *out, int on_device);

tsf_status tsf_get_stats(tsf_ctx *ctx, tsf_stats *out);
tsf_status tsf_reset_stats(tsf_ctx *ctx);

/* Gradient of the mean macro concentration after a march, by a discrete
 * adjoint of the implicit two-scale steps (the Eq. (17) step operator
 * differentiated through the pull-back factors of Eqs. (13)-(16)).
 *   J = int_Omega u(t_N) dx = sum_k m_k u_k^N   (Omega = [0,1]^2, m = row sums of M_H)
 * after nsteps steps of size dt from the current state, and dJ/dp for every
 * per-node deformation parameter of the family given to tsf_set_deformation
 * (grad_out[i * nparam + k]; parameters that do not change F, such as the
 * shift of the affine family, get 0).  The forward states are kept at
 * checkpoints every ckpt_every steps and recomputed segment by segment for
 * the backward march.  The gradient is that of the discrete march as solved
 * (use FP64 and tight tolerances when comparing with finite differences).
 * Requires the Neumann macro boundary and no sources (TSF_E_ARG otherwise).
 * J_out, grad_out: host (on_device = 0) or device pointers, may be NULL.  On
 * return the state is the state after the nsteps steps (as after tsf_step)
 * and the call has synchronised the stream.  The call allocates its own
 * checkpoint buffers (about (nsteps/ckpt_every + ckpt_every + 3) states) and
 * frees them before returning; TSF_E_OOM if that fails. */
tsf_status tsf_adjoint_mean_u(tsf_ctx *ctx, double dt, int nsteps, int ckpt_every, double *J_out, double *grad_out,
                              int on_device);

/* Device memory: bytes of the workspace the current meshes need, and binding
 * of a caller-owned device buffer of at least that size (256-byte aligned)
 * that the library then uses for all its arrays (e.g. memory from PyTorch's
 * caching allocator).  Without a bound workspace the library allocates its
 * own on first use.  Rebinding or changing a mesh invalidates the state. */
tsf_status tsf_workspace_bytes(tsf_ctx *ctx, size_t *bytes);
tsf_status tsf_bind_workspace(tsf_ctx *ctx, void *device_ptr, size_t bytes);

/* Text of the last error of this context ("" if none); never NULL. */
const char *tsf_last_error(const tsf_ctx *ctx);

/* Release everything the context owns (not a bound workspace).  NULL is a no-op. */
void tsf_destroy(tsf_ctx *ctx);

/* Library version as MAJOR*10000 + MINOR*100 + PATCH. */
int tsf_version(void);

/* -------------------------------------------------------------------------
 * Batches of independent two-scale problems (library addition; the paper
 * solves one problem at a time).  Each instance is an ordinary context: get
 * it with tsf_batch_instance and configure it with the tsf_set_* calls (its
 * own micro and macro meshes, physics, deformation, state, sources), read it
 * with the tsf_get_* calls.  All instances enqueue on the batch's stream.
 * tsf_batch_step advances every instance by nsteps steps of size dt; with
 * use_graph = 1 each batch step is ONE CUDA graph launch holding one
 * independent branch per instance (its prologues and its own device-side
 * coupling loop), so the instances run concurrently.  The graph is captured
 * on the first step and again whenever an instance's operators, variant,
 * workspace or dt change.  Each instance chooses its own micro-solve variant
 * (timed on its own problem when options.tiling = -1).
 * ------------------------------------------------------------------------- */
typedef struct tsf_batch tsf_batch;
#define TSF_BATCH_MAX 4096

/* Create a batch of ninst (1..TSF_BATCH_MAX) empty instances with options
 * opt (NULL = defaults; opt->cuda_stream NULL = a stream owned by the batch).
 * Errors: TSF_E_ARG, TSF_E_CUDA, TSF_E_OOM. */
tsf_status tsf_batch_create(tsf_batch **out, int ninst, const tsf_options *opt);

/* Borrowed handle of instance inst (0-based); it lives as long as the batch
 * and must not be passed to tsf_destroy.  Calling tsf_step on it steps that
 * instance alone. */
tsf_status tsf_batch_instance(tsf_batch *b, int inst, tsf_ctx **out);

/* Advance every instance by nsteps implicit Euler steps of size dt
 * (asynchronous on the batch stream; device-side errors are reported by
 * tsf_batch_synchronize).  TSF_E_STATE if an instance lacks meshes,
 * deformation or state; instance errors name the instance. */
tsf_status tsf_batch_step(tsf_batch *b, double dt, int nsteps);

/* Persistent batch steps (on = 1; default 0).  Each batch step is then ONE
 * CUDA graph launch: per instance, on its own branch, the macro prologue and
 * the macro solve; after the prologues, the micro solves of every micro
 * problem of every instance in persistent kernel launches, one per class of
 * micro mesh (strip height, threads a block, bulk-copy staging), side by side,
 * each of as many blocks as fit the GPU at once.  Every block solves one micro
 * problem at a time and takes work items from its class's global atomic
 * queue, ordered largest micro mesh first.  Requires mixed precision and
 * coupling by elimination without volume or Robin sources for every instance
 * (tsf_batch_step then returns TSF_E_ARG otherwise), micro meshes of at most
 * 49 cells per side and at most 64 instances, and switches
 * every instance to the column-strip variant whose arithmetic the batch
 * kernel runs: strips of 3 rows (tiling 4) up to 32 micro cells per side, of 5
 * rows (tiling 5) beyond.  Errors: TSF_E_ARG. */
tsf_status tsf_batch_set_persistent(tsf_batch *b, int on);

/* *out = the persistent micro-solve launches of one batch step (one per
 * class of micro mesh), as captured by the last persistent batch step; 0 if
 * no persistent batch step has been captured.
 * Errors: TSF_E_ARG (NULL pointer). */
tsf_status tsf_batch_persistent_launches(const tsf_batch *b, int *out);
tsf_status tsf_batch_synchronize(tsf_batch *b);

/* Statistics summed over the instances (coupling_iters_last, max_inner_iters
 * and coupling_change are maxima; steps counts batch steps; tiling = -1). */
tsf_status tsf_batch_get_stats(tsf_batch *b, tsf_stats *out);
tsf_status tsf_batch_reset_stats(tsf_batch *b);
const char *tsf_batch_last_error(const tsf_batch *b);
void tsf_batch_destroy(tsf_batch *b);

/* ---------------------------------------------------------------------------
 * Macro solve that allocates no device memory.  The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc when they
 * need a solve -- for example an application that gives all device memory to
 * its own pool allocator at start-up, or a latency-critical loop in which a
 * device-synchronising allocation is not acceptable.
 *
 * It runs the macro-solve kernel of tsf_step once, on caller-owned device
 * arrays, solving on the NM x NM macro mesh
 *     (M_H/dt + Du K_H + kappa L Gam) u = cH + kappa L rho
 * with L = diag(row sums of M_H), Gam = diag(gam), and u = u0 on the whole
 * boundary when bc = TSF_BC_DIRICHLET; FP64 flexible PCG started from u0
 * until ||residual||_2 <= tol ||rhs||_2, at most maxit iterations.
 * Arguments: NM cells per side (1 <= NM <= TSF_NOALLOC_MAX_NM); bc, dt > 0,
 * macro_diff (Du) > 0, kappa >= 0; gam, cH, rho, u0: device arrays of
 * nM = (NM+1)^2 doubles, node (p,q) at index p + (NM+1) q, read only;
 * u_out: device array of nM doubles that receives u (it may be u0 itself);
 * cuda_stream: cudaStream_t to run on (NULL = legacy default stream);
 * iters_out: optional host int receiving the PCG iteration count.
 *
 * Its scratch (six vectors of the PCG and a control block) is one fixed
 * device array of the library, sized for TSF_NOALLOC_MAX_NM (about 0.8 MB);
 * every GPU that loads the library holds it until the process exits.  The
 * first call on a device looks up that array's device address and sets the
 * kernel's shared-memory limit (and keeps both for the later calls).  All
 * calls on a device share the array (it keeps the last call's contents; the
 * call clears what must start from zero): calls that overlap on the GPU, e.g.
 * on two streams at once, race and must not be issued.  The call blocks: it
 * reads the solve's status back and waits for cuda_stream before returning.
 * Errors: TSF_E_ARG (NM outside 1..TSF_NOALLOC_MAX_NM, bad
 * scalar, NULL array), TSF_E_CUDA (runtime failure), TSF_E_NOT_CONVERGED or
 * TSF_E_NAN from the solve; there is no context, so tsf_last_error does not
 * apply.
 * ------------------------------------------------------------------------- */
#define TSF_NOALLOC_MAX_NM 128
tsf_status tsf_macro_solve_noalloc(int NM, int bc, double dt, double macro_diff, double kappa, const double *gam,
                                   const double *cH, const double *rho, const double *u0, double *u_out,
                                   double tol, int maxit, void *cuda_stream, int *iters_out);

#ifdef __cplusplus
}
#endif

#endif /* TSFEM_H */
