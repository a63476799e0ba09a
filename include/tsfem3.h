/* tsfem3.h -- C ABI of the stationary three-field two-scale system on one GB300.
 *
 * The full model of Lakkis, Muntean, Richardson, Venkataraman (arXiv
 * 2103.17040), Eq. (5): a macro nutrient u, one micro field v per macro node
 * and a macro product w, in the pulled-back discrete form of Eq. (17):
 *
 *   -Lap u           = f^u - int_{Gamma_I} (kappa_1 u - kappa_2 v + g_1)    in Omega,
 *   u = u_D on the Dirichlet edges,  grad u . n = g^u on the others,
 *   -div(D grad v)   = f^v                                                  in Y_x,
 *   D grad v . n     = kappa_1 u - kappa_2 v + g_1   on Gamma_I,
 *                      kappa_3 w - kappa_4 v + g_2   on Gamma_O,
 *                      g_3                           on Gamma_N,
 *   -D^w Lap w       = f^w - int_{Gamma_O} (kappa_3 w - kappa_4 v + g_2)    in Omega,
 *   D^w grad w . n   = g^w                                                  on the boundary,
 *
 * with the sources and data g of the manufactured system, Eq. (18) (all zero
 * for the model itself).  Omega = [x0, x0 + L]^2 carries an NM x NM Q1 mesh.
 * Every macro node x_i has one micro problem on the reference cell
 * [0,1]^2 (Nm x Nm Q1 cells), mapped to its cell Y_x by the per-node
 * deformation of tsfem.h's families.  Gamma_I is the reference edge
 * yhat_1 = 0, Gamma_O is yhat_1 = 1, and Gamma_N is yhat_2 = 0 and
 * yhat_2 = 1 (Fig. 1).  The discretisation readings are those of the
 * two-field library:
 * - collocation in x (one micro system per macro node, Sec. 3.3);
 * - coupling integrals lumped at the node with the row sums m of M_H;
 * - boundary measure |cof(F) nu| (Eq. (16));
 * - 2x2 Gauss points in cells, 2 on edges;
 * - data given as nodal values and integrated as Q1 interpolants.
 *
 * Solution method (exact elimination of the micro unknowns; the paper
 * iterates instead):
 *   v_i = v0_i + u_i phi_I,i + w_i phi_O,i,   S_i = A_i + kappa_2 R_I,i + kappa_4 R_O,i,
 *   S_i phi_I = kappa_1 r_I,  S_i phi_O = kappa_3 r_O,  S_i v0 = (micro sources);
 * three batched micro solves (phi_I and phi_O once per geometry and physics).
 * One coupled, symmetric positive definite macro solve in (u, w) follows.
 *
 * Conventions (as tsfem.h): the caller owns every buffer it passes; pointers
 * are host or device memory as the on_device flag says; the library copies
 * inputs and never keeps caller pointers; every call returns a status and
 * tsf3_last_error() describes the last failure; nothing aborts.  Calls are
 * asynchronous on the context's stream; tsf3_solve and the getters with
 * on_device = 0 synchronise it.
 */
#ifndef TSFEM3_H
#define TSFEM3_H

#include "tsfem.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tsf3_ctx tsf3_ctx;

enum { TSF3_TILING_DIRECT = 10 };

/* Dirichlet edges of u (bit set = Dirichlet), also the order of the per-edge data */
enum { TSF3_EDGE_BOTTOM = 1, TSF3_EDGE_RIGHT = 2, TSF3_EDGE_TOP = 4, TSF3_EDGE_LEFT = 8 };

typedef struct {
    int64_t inner_iters;     /* inner CG iterations of the micro solves, summed over instances */
    int64_t dof_cg_iters;    /* sum over instances of (micro DoFs x inner iterations) */
    int64_t refine_sweeps;   /* FP64 residual evaluations of micro problems */
    int64_t micro_solves;    /* micro problems solved (3 per node with a new geometry, else 1) */
    int64_t macro_iters;     /* CG iterations of the coupled macro solve */
    int status;              /* device status of the last solve (tsf_status) */
    int tiling;              /* micro-solve variant in use (0..9 and 11..14 as tsf_stats.tiling, or TSF3_TILING_DIRECT) */
    double micro_ms;         /* device time of the micro solves of the last tsf3_solve */
    double macro_ms;         /* device time of the macro solve */
    double total_ms;         /* device time of the whole last tsf3_solve */
    double factor_ms;        /* direct solve: device time of the band factorisation in the last solve (0 if kept) */
    double band_solve_ms;    /* direct solve: device time of the triangular-solve launches of the last solve */
    int band_launches;       /* direct solve: triangular-solve launches (refinement sweeps) of the last solve */
    int band_rhs;            /* direct solve: right-hand sides per launch in the last solve (1 or 3) */
} tsf3_stats;

/* Uses from tsf_options: precision, cg_tol (micro relative residual),
 * inner_tol, cg_maxit, max_sweeps, macro_tol, macro_maxit, tiling,
 * cuda_stream (NULL = own stream).  tiling: 0..9 and 11..14 the iterative
 * micro-solve variants of tsf_stats.tiling; TSF3_TILING_DIRECT (mixed precision only): a
 * banded Cholesky factor of every micro operator in FP32, kept while the
 * geometry and physics stay the same, with FP64 iterative refinement to
 * cg_tol (at most max(max_sweeps, 30) sweeps); -1: the direct solve in
 * mixed precision when its factor (nM nm (Nm+3) 4 bytes) fits in half the
 * free device memory, else the fastest iterative variant, timed on the first
 * solve. */
tsf_status tsf3_create(tsf3_ctx** out, const tsf_options* opt);

/* Nm x Nm micro cells (1..64), NM x NM macro cells (1..256) on
 * [x0, x0 + L]^2 (L > 0); dir_mask: Dirichlet edges of u (TSF3_EDGE_*), at
 * least one (Sec. 2.2: without one the constant equilibrium state is a null
 * vector of the stationary system), else TSF_E_ARG.
 * Allocates the device state; forgets geometry, sources and solution. */
tsf_status tsf3_set_meshes(tsf3_ctx* ctx, int Nm, int NM, double x0, double L, int dir_mask);

/* D = D^v as (D11, D12, D22), symmetric positive definite; Dw = D^w > 0;
 * kappa[0..3] = kappa_1..kappa_4, all > 0 (Sec. 2.2). */
tsf_status tsf3_set_physics(tsf3_ctx* ctx, const double D[3], double Dw, const double kappa[4]);

/* Per-node deformation, as tsf_set_deformation: family TSF_FAMILY_*,
 * params [nM][nparam] row-major.  TSF_E_BAD_JACOBIAN from tsf3_solve if
 * det F <= 0 at a quadrature point. */
tsf_status tsf3_set_deformation(tsf3_ctx* ctx, int family, int nparam, const double* params, int on_device);

/* Sources and data (each NULL = zero):
 *   fu, fw [nM]      nodal f^u, f^w;
 *   ud [nM]          Dirichlet values of u (read on Dirichlet nodes only);
 *   gu, gw [4][NM+1] Neumann data of u (ignored on Dirichlet edges) and w per
 *                    macro edge: bottom (by p), right (by q), top (by p), left (by q);
 *   fv [nM][nm]      nodal f^v of every micro problem (nm = (Nm+1)^2);
 *   gI, gO [nM][Nm+1] g_1 on Gamma_I and g_2 on Gamma_O, by q;
 *   gN [nM][2][Nm+1]  g_3 on yhat_2 = 0 and on yhat_2 = 1, by p. */
tsf_status tsf3_set_sources(tsf3_ctx* ctx, const double* fu, const double* fw, const double* ud, const double* gu,
                            const double* gw, const double* fv, const double* gI, const double* gO,
                            const double* gN, int on_device);

/* Solves the stationary system; returns the device status (TSF_E_NOT_CONVERGED,
 * TSF_E_NAN, ...) after synchronising the stream. */
tsf_status tsf3_solve(tsf3_ctx* ctx);

/* Copies of the solution (each NULL = skip): u, w [nM], v [nM][nm],
 * vbar [nM] (micro averages 1^T M_i v_i / |Y_x_i|). */
tsf_status tsf3_get_fields(tsf3_ctx* ctx, double* u, double* w, double* v, double* vbar, int on_device);

/* Push-forward of the micro fields for visualisation (Sec. 3.6): micro node j
 * of node i at X = x_i + scale (chi(x_i, yhat_j) - chi(x_i, (1/2, 1/2))), each
 * cell centred on its macro node; out = [nM][nm][3] FP32 (X1, X2, v).  The
 * same buffer layout as tsf_get_pushforward; TSF_E_STATE before a solve. */
tsf_status tsf3_get_pushforward(tsf3_ctx* ctx, float scale, float* out, int on_device);

tsf_status tsf3_get_stats(tsf3_ctx* ctx, tsf3_stats* out);
const char* tsf3_last_error(const tsf3_ctx* ctx);
void tsf3_destroy(tsf3_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* TSFEM3_H */
