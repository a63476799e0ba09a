/*
 * tsf_oracle.c -- plain FP64 CPU oracle of the two-scale finite element time
 * step (Lakkis, Muntean, Richardson, Venkataraman, "Parallel two-scale finite
 * element implementation of a system with varying microstructure").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header, table or constant with the
 * CUDA path.
 *
 * What it computes (the u-v part of the model system, Eq. (5), made parabolic
 * with implicit Euler; one micro problem per macro node, Sec. 3.3):
 *
 *   micro i:  (M_i/dt + A_i + kappa R_i) v_i - kappa r_i u_i
 *                 = M_i v_i^n/dt + M_i fv_i + R_i g_i
 *   macro:    (M_H/dt + Du K_H + kappa L Gam) u - kappa L rho(v)
 *                 = M_H u^n/dt + M_H fu - L G
 *
 *   M_i = int_Z J eta_j eta_l,  A_i = int_Z C grad eta_j . grad eta_l,
 *   C = J F^{-1} D F^{-T},      R_i = int_Gamma |cof(F) nu| eta_j eta_l,
 *   r_i = R_i 1, |Gam_i| = 1^T r_i, L = diag(row sums of M_H),
 *   rho(v)_i = r_i^T v_i, G_i = r_i^T g_i.
 *
 * The pull-back factors follow Eqs. (13), (14) and (16) of Sec. 3.1; the
 * bilinear forms follow the discrete weak form Eq. (17) with the boundary
 * measure read as |cof(F) nu| (Eq. (16)) and the macro coupling term lumped
 * at the collocation node (Sec. 3.3: one micro system per macro degree of
 * freedom, located at its support point).  The coupled system is solved by
 * the partitioned fixed-point iteration of Sec. 3.3 (micro solves with the
 * current u, then the macro solve with the new micro fluxes) with
 * Jacobi-preconditioned CG for every system (Sec. 3.5, last paragraph),
 * micro systems distributed over the host threads with OpenMP.
 *
 * Meshes: Z = [0,1]^2 with Nm x Nm square Q1 cells, Omega = [0,1]^2 with
 * NM x NM cells; node (p,q) has index p + (N+1) q and sits at (p,q)/N.
 * Quadrature: 2x2 Gauss per cell, 2-point Gauss per edge.  The Robin
 * (inflow) edge of the reference cell is yhat_1 = 1 with normal nu = (1,0);
 * the other three edges carry homogeneous Neumann data.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_E_ARG 1
#define OR_E_BAD_JACOBIAN 3
#define OR_E_NOT_CONVERGED 4
#define OR_E_BREAKDOWN 5
#define OR_E_OOM 7

#define OR_PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* Deformation families chi(x_i, .) : Z -> Y_x (Sec. 2, Eqs. (2)-(3)).       */
/* F is the Jacobian D_yhat chi, row-major {F11, F12, F21, F22}.             */
/*   0 identity        chi = yhat                                            */
/*   1 bump (a)        chi = yhat + a (sin pi y1 sin pi y2, 0)               */
/*   2 shear+bump (s,b) chi = (y1 + s y2 + b sin pi y1 sin pi y2, y2)        */
/*   3 affine (A11,A12,A21,A22,c1,c2)  chi = A yhat + c                      */
/*   4 affine+bump (A11,A12,A21,A22,b) chi = A yhat + b (sin sin, 0)         */
/* ------------------------------------------------------------------------ */
int or_family_nparam(int family)
{
    switch (family) {
    case 0: return 0;
    case 1: return 1;
    case 2: return 2;
    case 3: return 6;
    case 4: return 5;
    default: return -1;
    }
}

int or_chi(int family, const double *prm, double y1, double y2, double chi[2], double F[4])
{
    double s1 = sin(OR_PI * y1), c1 = cos(OR_PI * y1);
    double s2 = sin(OR_PI * y2), c2 = cos(OR_PI * y2);
    switch (family) {
    case 0:
        chi[0] = y1; chi[1] = y2;
        F[0] = 1.0; F[1] = 0.0; F[2] = 0.0; F[3] = 1.0;
        return OR_OK;
    case 1: {
        double a = prm[0];
        chi[0] = y1 + a * s1 * s2; chi[1] = y2;
        F[0] = 1.0 + a * OR_PI * c1 * s2; F[1] = a * OR_PI * s1 * c2;
        F[2] = 0.0; F[3] = 1.0;
        return OR_OK;
    }
    case 2: {
        double s = prm[0], b = prm[1];
        chi[0] = y1 + s * y2 + b * s1 * s2; chi[1] = y2;
        F[0] = 1.0 + b * OR_PI * c1 * s2; F[1] = s + b * OR_PI * s1 * c2;
        F[2] = 0.0; F[3] = 1.0;
        return OR_OK;
    }
    case 3:
        chi[0] = prm[0] * y1 + prm[1] * y2 + prm[4];
        chi[1] = prm[2] * y1 + prm[3] * y2 + prm[5];
        F[0] = prm[0]; F[1] = prm[1]; F[2] = prm[2]; F[3] = prm[3];
        return OR_OK;
    case 4: {
        double b = prm[4];
        chi[0] = prm[0] * y1 + prm[1] * y2 + b * s1 * s2;
        chi[1] = prm[2] * y1 + prm[3] * y2;
        F[0] = prm[0] + b * OR_PI * c1 * s2; F[1] = prm[1] + b * OR_PI * s1 * c2;
        F[2] = prm[2]; F[3] = prm[3];
        return OR_OK;
    }
    default:
        return OR_E_ARG;
    }
}

/* chi and F at many points of one deformation (vectorised helper for the
 * error norms of the manufactured-solution check) */
int or_chi_many(int family, const double *prm, int n, const double *y1, const double *y2,
                double *chi_out, double *F_out)
{
    for (int k = 0; k < n; ++k) {
        int e = or_chi(family, prm, y1[k], y2[k], chi_out + 2 * k, F_out + 4 * k);
        if (e) return e;
    }
    return OR_OK;
}

/* Pull-back factors at one point (Sec. 3.1, Eqs. (13), (14), (16)):
 *   J = det F,  K = F^{-1},  C = J K D K^T  (diffusion tensor on Z, with the
 *   micro diffusion D inserted between K and K^T),
 *   cof(F) = J F^{-T},  s = |cof(F) nu|  (surface-measure factor for the
 *   reference normal nu).
 * D is symmetric, given as {D11, D12, D22}; C is returned the same way. */
void or_pullback(const double F[4], const double D[3], const double nu[2],
                 double *J, double C[3], double *s)
{
    double det = F[0] * F[3] - F[1] * F[2];
    /* K = F^{-1} */
    double K11 = F[3] / det, K12 = -F[1] / det, K21 = -F[2] / det, K22 = F[0] / det;
    /* K D K^T */
    double KD11 = K11 * D[0] + K12 * D[1], KD12 = K11 * D[1] + K12 * D[2];
    double KD21 = K21 * D[0] + K22 * D[1], KD22 = K21 * D[1] + K22 * D[2];
    C[0] = det * (KD11 * K11 + KD12 * K12);
    C[1] = det * (KD11 * K21 + KD12 * K22);
    C[2] = det * (KD21 * K21 + KD22 * K22);
    /* cof(F) = det * K^T */
    double c11 = det * K11, c12 = det * K21, c21 = det * K12, c22 = det * K22;
    double w1 = c11 * nu[0] + c12 * nu[1];
    double w2 = c21 * nu[0] + c22 * nu[1];
    *J = det;
    *s = sqrt(w1 * w1 + w2 * w2);
}

/* unit outward normal of Y_x on the image of a reference edge with normal nu:
 * cof(F) nu / |cof(F) nu| (Nanson's relation behind Eq. (16)) */
void or_unit_normal(const double F[4], const double nu[2], double n_out[2])
{
    double c11 = F[3], c12 = -F[2], c21 = -F[1], c22 = F[0];
    double w1 = c11 * nu[0] + c12 * nu[1];
    double w2 = c21 * nu[0] + c22 * nu[1];
    double l = sqrt(w1 * w1 + w2 * w2);
    n_out[0] = w1 / l;
    n_out[1] = w2 / l;
}

/* ------------------------------------------------------------------------ */
/* Q1 element on the unit reference square, local nodes                     */
/*   0:(0,0) 1:(1,0) 2:(0,1) 3:(1,1);  phi_k(s,t) bilinear.                  */
/* ------------------------------------------------------------------------ */
static void q1_shape(double s, double t, double phi[4], double ds[4], double dt[4])
{
    phi[0] = (1 - s) * (1 - t); phi[1] = s * (1 - t); phi[2] = (1 - s) * t; phi[3] = s * t;
    ds[0] = -(1 - t); ds[1] = (1 - t); ds[2] = -t; ds[3] = t;
    dt[0] = -(1 - s); dt[1] = -s; dt[2] = (1 - s); dt[3] = s;
}

static double gauss_pt(int k) { return 0.5 + (k ? 0.5 : -0.5) / sqrt(3.0); }

/* CSR pattern of a Q1 mesh with N x N cells: row = node, columns = the (up to
 * nine) nodes sharing a cell with it, ascending. Returns nnz. */
int or_q1_pattern(int N, int *rowptr, int *col)
{
    int n1 = N + 1, nnz = 0;
    for (int q = 0; q < n1; ++q)
        for (int p = 0; p < n1; ++p) {
            rowptr[p + n1 * q] = nnz;
            for (int dq = -1; dq <= 1; ++dq)
                for (int dp = -1; dp <= 1; ++dp) {
                    int pp = p + dp, qq = q + dq;
                    if (pp < 0 || qq < 0 || pp >= n1 || qq >= n1) continue;
                    col[nnz++] = pp + n1 * qq;
                }
        }
    rowptr[n1 * n1] = nnz;
    return nnz;
}

int or_q1_nnz(int N)
{
    int n1 = N + 1;
    /* interior rows 9, edge rows 6, corner rows 4 */
    return 9 * (n1 - 2) * (n1 - 2) + 4 * 6 * (n1 - 2) + 4 * 4;
}

static int csr_pos(const int *rowptr, const int *col, int row, int c)
{
    for (int k = rowptr[row]; k < rowptr[row + 1]; ++k)
        if (col[k] == c) return k;
    return -1;
}

/* Assemble M = int J eta eta, A = int C grad eta . grad eta on the reference
 * mesh of Z (Nm cells per side) for one deformation (Eq. (17) micro block;
 * Sec. 3.4: J and J K K^T evaluated at every quadrature point), and the Robin
 * boundary mass R = int_{yhat1=1} |cof(F) e1| eta eta.  Any of the outputs may
 * be NULL.  Returns OR_E_BAD_JACOBIAN if J <= 0 at a quadrature point
 * (Eq. (3) requires 0 < c_* <= det). */
int or_assemble_q1(int N, int family, const double *prm, const double D[3],
                   const int *rowptr, const int *col,
                   double *M, double *A, double *R)
{
    int n1 = N + 1, nnz = rowptr[n1 * n1];
    double h = 1.0 / N;
    const double e1[2] = {1.0, 0.0};
    if (M) memset(M, 0, sizeof(double) * nnz);
    if (A) memset(A, 0, sizeof(double) * nnz);
    if (R) memset(R, 0, sizeof(double) * nnz);
    for (int b = 0; b < N; ++b)
        for (int a = 0; a < N; ++a) {
            int gl[4] = {a + n1 * b, a + 1 + n1 * b, a + n1 * (b + 1), a + 1 + n1 * (b + 1)};
            double Me[4][4] = {{0}}, Ae[4][4] = {{0}};
            for (int qt = 0; qt < 2; ++qt)
                for (int qs = 0; qs < 2; ++qs) {
                    double s = gauss_pt(qs), t = gauss_pt(qt);
                    double chi[2], F[4], J, C[3], sg;
                    or_chi(family, prm, (a + s) * h, (b + t) * h, chi, F);
                    or_pullback(F, D, e1, &J, C, &sg);
                    if (!(J > 0.0)) return OR_E_BAD_JACOBIAN;
                    double phi[4], ds[4], dt[4];
                    q1_shape(s, t, phi, ds, dt);
                    /* weight 1/4 per point on the unit square; dy = h^2 d(s,t),
                       grad_yhat = grad_(s,t) / h, so A picks up h^2/h^2 = 1 */
                    for (int i = 0; i < 4; ++i)
                        for (int j = 0; j < 4; ++j) {
                            Me[i][j] += 0.25 * h * h * J * phi[i] * phi[j];
                            Ae[i][j] += 0.25 * (ds[i] * (C[0] * ds[j] + C[1] * dt[j]) +
                                                dt[i] * (C[1] * ds[j] + C[2] * dt[j]));
                        }
                }
            for (int i = 0; i < 4; ++i)
                for (int j = 0; j < 4; ++j) {
                    int k = csr_pos(rowptr, col, gl[i], gl[j]);
                    if (M) M[k] += Me[i][j];
                    if (A) A[k] += Ae[i][j];
                }
        }
    if (R) {
        /* Robin edge yhat1 = 1: cells (N-1, b), local nodes 1 (t=0) and 3 (t=1) */
        for (int b = 0; b < N; ++b) {
            int g1 = N + n1 * b, g3 = N + n1 * (b + 1);
            double Re[2][2] = {{0}};
            for (int qt = 0; qt < 2; ++qt) {
                double t = gauss_pt(qt);
                double chi[2], F[4], J, C[3], sg;
                or_chi(family, prm, 1.0, (b + t) * h, chi, F);
                or_pullback(F, D, e1, &J, C, &sg);
                double ph[2] = {1 - t, t};
                for (int i = 0; i < 2; ++i)
                    for (int j = 0; j < 2; ++j) Re[i][j] += 0.5 * h * sg * ph[i] * ph[j];
            }
            int gg[2] = {g1, g3};
            for (int i = 0; i < 2; ++i)
                for (int j = 0; j < 2; ++j) R[csr_pos(rowptr, col, gg[i], gg[j])] += Re[i][j];
        }
    }
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Parameter derivatives of the pulled-back operators (for the discrete      */
/* adjoint of the two-scale march).                                          */
/* ------------------------------------------------------------------------ */
/* dF/dp_k of the deformation families at one point, row-major.  Returns
 * OR_E_ARG for k outside the family's parameters. */
int or_dchi(int family, int k, double y1, double y2, double dF[4])
{
    double s1 = sin(OR_PI * y1), c1 = cos(OR_PI * y1);
    double s2 = sin(OR_PI * y2), c2 = cos(OR_PI * y2);
    dF[0] = dF[1] = dF[2] = dF[3] = 0.0;
    if (k < 0 || k >= or_family_nparam(family)) return OR_E_ARG;
    int bump = (family == 1 && k == 0) || (family == 2 && k == 1) || (family == 4 && k == 4);
    if (bump) {
        dF[0] = OR_PI * c1 * s2;
        dF[1] = OR_PI * s1 * c2;
        return OR_OK;
    }
    if (family == 2 && k == 0) { dF[1] = 1.0; return OR_OK; } /* shear s */
    if ((family == 3 || family == 4) && k < 4) { dF[k] = 1.0; return OR_OK; } /* A entries */
    return OR_OK;                                                           /* affine shift c */
}

/* Derivatives at one point, obtained by differentiating the formulas of
 * or_pullback: J = det F, C = adj(F) D adj(F)^T / J, s = |adj(F)^T nu|. */
static void dpullback(const double F[4], const double dF[4], const double D[3], const double nu[2],
                      double *dJ, double dC[3], double *ds)
{
    double J = F[0] * F[3] - F[1] * F[2];
    double G[4] = {F[3], -F[1], -F[2], F[0]};        /* adj(F) */
    double dG[4] = {dF[3], -dF[1], -dF[2], dF[0]};   /* adj is linear */
    double Dm[4] = {D[0], D[1], D[1], D[2]};
    *dJ = dF[0] * F[3] + F[0] * dF[3] - dF[1] * F[2] - F[1] * dF[2];
    /* P = G D G^T, dP = dG D G^T + G D dG^T */
    double GD[4], dGD[4];
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            GD[2 * a + b] = G[2 * a] * Dm[b] + G[2 * a + 1] * Dm[2 + b];
            dGD[2 * a + b] = dG[2 * a] * Dm[b] + dG[2 * a + 1] * Dm[2 + b];
        }
    double P[4], dP[4];
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            P[2 * a + b] = GD[2 * a] * G[2 * b] + GD[2 * a + 1] * G[2 * b + 1];
            dP[2 * a + b] = dGD[2 * a] * G[2 * b] + dGD[2 * a + 1] * G[2 * b + 1] +
                            GD[2 * a] * dG[2 * b] + GD[2 * a + 1] * dG[2 * b + 1];
        }
    /* C = P / J  ->  dC = dP / J - P dJ / J^2 */
    dC[0] = dP[0] / J - P[0] * *dJ / (J * J);
    dC[1] = dP[1] / J - P[1] * *dJ / (J * J);
    dC[2] = dP[3] / J - P[3] * *dJ / (J * J);
    /* w = G^T nu, s = |w|, ds = w . dw / s */
    double w0 = G[0] * nu[0] + G[2] * nu[1], w1 = G[1] * nu[0] + G[3] * nu[1];
    double dw0 = dG[0] * nu[0] + dG[2] * nu[1], dw1 = dG[1] * nu[0] + dG[3] * nu[1];
    *ds = (w0 * dw0 + w1 * dw1) / sqrt(w0 * w0 + w1 * w1);
}

/* dM, dA, dR: derivatives of the micro matrices of or_assemble_q1 with respect
 * to parameter k of the deformation (same quadrature, same pattern). */
int or_assemble_q1_dparam(int N, int family, const double *prm, int k, const double D[3],
                          const int *rowptr, const int *col, double *dM, double *dA, double *dR)
{
    int n1 = N + 1, nnz = rowptr[n1 * n1];
    double h = 1.0 / N;
    const double e1[2] = {1.0, 0.0};
    memset(dM, 0, sizeof(double) * nnz);
    memset(dA, 0, sizeof(double) * nnz);
    memset(dR, 0, sizeof(double) * nnz);
    if (k < 0 || k >= or_family_nparam(family)) return OR_E_ARG;
    for (int b = 0; b < N; ++b)
        for (int a = 0; a < N; ++a) {
            int gl[4] = {a + n1 * b, a + 1 + n1 * b, a + n1 * (b + 1), a + 1 + n1 * (b + 1)};
            double Me[4][4] = {{0}}, Ae[4][4] = {{0}};
            for (int qt = 0; qt < 2; ++qt)
                for (int qs = 0; qs < 2; ++qs) {
                    double s = gauss_pt(qs), t = gauss_pt(qt);
                    double chi[2], F[4], dF[4], dJ, dC[3], dsg;
                    or_chi(family, prm, (a + s) * h, (b + t) * h, chi, F);
                    or_dchi(family, k, (a + s) * h, (b + t) * h, dF);
                    dpullback(F, dF, D, e1, &dJ, dC, &dsg);
                    double phi[4], ds[4], dt[4];
                    q1_shape(s, t, phi, ds, dt);
                    for (int i = 0; i < 4; ++i)
                        for (int j = 0; j < 4; ++j) {
                            Me[i][j] += 0.25 * h * h * dJ * phi[i] * phi[j];
                            Ae[i][j] += 0.25 * (ds[i] * (dC[0] * ds[j] + dC[1] * dt[j]) +
                                                dt[i] * (dC[1] * ds[j] + dC[2] * dt[j]));
                        }
                }
            for (int i = 0; i < 4; ++i)
                for (int j = 0; j < 4; ++j) {
                    int kk = csr_pos(rowptr, col, gl[i], gl[j]);
                    dM[kk] += Me[i][j];
                    dA[kk] += Ae[i][j];
                }
        }
    for (int b = 0; b < N; ++b) {
        int gg[2] = {N + n1 * b, N + n1 * (b + 1)};
        double Re[2][2] = {{0}};
        for (int qt = 0; qt < 2; ++qt) {
            double t = gauss_pt(qt);
            double chi[2], F[4], dF[4], dJ, dC[3], dsg;
            or_chi(family, prm, 1.0, (b + t) * h, chi, F);
            or_dchi(family, k, 1.0, (b + t) * h, dF);
            dpullback(F, dF, D, e1, &dJ, dC, &dsg);
            double ph[2] = {1 - t, t};
            for (int i = 0; i < 2; ++i)
                for (int j = 0; j < 2; ++j) Re[i][j] += 0.5 * h * dsg * ph[i] * ph[j];
        }
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j) dR[csr_pos(rowptr, col, gg[i], gg[j])] += Re[i][j];
    }
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Sparse kernels and Jacobi-preconditioned CG (Sec. 3.5, last paragraph).   */
/* ------------------------------------------------------------------------ */
void or_csr_matvec(int n, const int *rowptr, const int *col, const double *val,
                   const double *x, double *y)
{
    for (int i = 0; i < n; ++i) {
        double acc = 0.0;
        for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) acc += val[k] * x[col[k]];
        y[i] = acc;
    }
}

static double dot(int n, const double *a, const double *b)
{
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/* Solve A x = b, A symmetric positive definite in CSR, x holds the initial
 * guess on entry.  Stops when ||b - A x||_2 <= tol ||b||_2 (recursive
 * residual), or after maxit iterations.  work: 4 n doubles.
 * Returns OR_OK, OR_E_NOT_CONVERGED or OR_E_BREAKDOWN (p^T A p <= 0). */
int or_pcg(int n, const int *rowptr, const int *col, const double *val,
           const double *b, double *x, double tol, int maxit, double *work,
           int *iters, double *relres)
{
    double *r = work, *z = work + n, *p = work + 2 * n, *q = work + 3 * n;
    double bn = sqrt(dot(n, b, b));
    *iters = 0;
    if (bn == 0.0) {
        for (int i = 0; i < n; ++i) x[i] = 0.0;
        *relres = 0.0;
        return OR_OK;
    }
    or_csr_matvec(n, rowptr, col, val, x, q);
    for (int i = 0; i < n; ++i) r[i] = b[i] - q[i];
    double rn = sqrt(dot(n, r, r));
    if (rn <= tol * bn) { *relres = rn / bn; return OR_OK; }
    for (int i = 0; i < n; ++i) {
        double d = val[csr_pos(rowptr, col, i, i)];
        z[i] = r[i] / d;
        p[i] = z[i];
    }
    double rz = dot(n, r, z);
    for (int it = 1; it <= maxit; ++it) {
        or_csr_matvec(n, rowptr, col, val, p, q);
        double pq = dot(n, p, q);
        if (!(pq > 0.0)) { *iters = it; *relres = rn / bn; return OR_E_BREAKDOWN; }
        double alpha = rz / pq;
        for (int i = 0; i < n; ++i) { x[i] += alpha * p[i]; r[i] -= alpha * q[i]; }
        rn = sqrt(dot(n, r, r));
        if (rn <= tol * bn) { *iters = it; *relres = rn / bn; return OR_OK; }
        for (int i = 0; i < n; ++i) z[i] = r[i] / val[csr_pos(rowptr, col, i, i)];
        double rz1 = dot(n, r, z), beta = rz1 / rz;
        rz = rz1;
        for (int i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
    }
    *iters = maxit;
    *relres = rn / bn;
    return OR_E_NOT_CONVERGED;
}

/* ------------------------------------------------------------------------ */
/* Two-scale problem                                                        */
/* ------------------------------------------------------------------------ */
typedef struct or_stats {
    int64_t inner_iters;      /* sum over instances, coupling iterations and steps of CG iterations */
    int64_t micro_solves;     /* number of micro CG solves */
    int64_t macro_iters;      /* macro CG iterations */
    int coupling_iters_last;  /* coupling iterations in the last step */
    int coupling_iters_total;
    int max_inner_iters;      /* largest single micro solve */
    int status;               /* OR_OK or first error */
    double coupling_change;   /* final ||du||/||u|| of the last step */
    double paper_residual;    /* macro relative residual + mean micro relative residual */
} or_stats;

typedef struct or_problem {
    int Nm, NM, nm, nM, nnz_m, nnz_M;
    int bc;                   /* 0: homogeneous Neumann on dOmega, 1: Dirichlet on all of dOmega */
    int family, nparam;
    double D[3], kappa, Du;
    double *prm;              /* [nM][nparam] */
    int *rp, *ci;             /* micro CSR pattern, shared by all instances (Sec. 3.3) */
    int *rpH, *ciH;           /* macro CSR pattern */
    double *Mv, *Av, *Rv;     /* [nM][nnz_m] micro matrices */
    double *Sv;               /* [nM][nnz_m] micro system M/dt + A + kappa R for Sdt */
    double Sdt;
    double *MH, *KH;          /* macro mass and stiffness */
    double *r, *gam, *vol, *mH; /* r_i = R_i 1 [nM][nm], |Gam_i|, vol_i, row sums of M_H */
    double *u, *v;            /* state: u [nM], v [nM][nm] */
    double *fv, *g, *fu, *ud; /* optional sources for the next step(s), NULL when absent */
    int *is_dir;              /* [nM] 1 on Dirichlet nodes */
    or_stats st;
} or_problem;

static int boundary_node(int N, int k)
{
    int n1 = N + 1, p = k % n1, q = k / n1;
    return p == 0 || q == 0 || p == N || q == N;
}

void or_destroy(or_problem *P)
{
    if (!P) return;
    free(P->prm); free(P->rp); free(P->ci); free(P->rpH); free(P->ciH);
    free(P->Mv); free(P->Av); free(P->Rv); free(P->Sv); free(P->MH); free(P->KH);
    free(P->r); free(P->gam); free(P->vol); free(P->mH); free(P->u); free(P->v);
    free(P->fv); free(P->g); free(P->fu); free(P->ud); free(P->is_dir);
    free(P);
}

/* Build meshes, pull-back data and all matrices (Sec. 3.3 steps 1-4). */
or_problem *or_create(int Nm, int NM, int bc, int family, const double *prm,
                      const double D[3], double kappa, double Du, int *err)
{
    *err = OR_OK;
    if (Nm < 1 || NM < 1 || or_family_nparam(family) < 0 || (bc != 0 && bc != 1)) {
        *err = OR_E_ARG;
        return NULL;
    }
    or_problem *P = (or_problem *)calloc(1, sizeof(or_problem));
    if (!P) { *err = OR_E_OOM; return NULL; }
    P->Nm = Nm; P->NM = NM; P->nm = (Nm + 1) * (Nm + 1); P->nM = (NM + 1) * (NM + 1);
    P->bc = bc; P->family = family; P->nparam = or_family_nparam(family);
    P->D[0] = D[0]; P->D[1] = D[1]; P->D[2] = D[2];
    P->kappa = kappa; P->Du = Du;
    int nm = P->nm, nM = P->nM;
    P->nnz_m = or_q1_nnz(Nm);
    P->nnz_M = or_q1_nnz(NM);
    size_t nz = (size_t)P->nnz_m;
    P->prm = (double *)malloc(sizeof(double) * (size_t)nM * (P->nparam ? P->nparam : 1));
    P->rp = (int *)malloc(sizeof(int) * (nm + 1));
    P->ci = (int *)malloc(sizeof(int) * nz);
    P->rpH = (int *)malloc(sizeof(int) * (nM + 1));
    P->ciH = (int *)malloc(sizeof(int) * P->nnz_M);
    P->Mv = (double *)malloc(sizeof(double) * nz * nM);
    P->Av = (double *)malloc(sizeof(double) * nz * nM);
    P->Rv = (double *)malloc(sizeof(double) * nz * nM);
    P->MH = (double *)malloc(sizeof(double) * P->nnz_M);
    P->KH = (double *)malloc(sizeof(double) * P->nnz_M);
    P->r = (double *)malloc(sizeof(double) * (size_t)nm * nM);
    P->gam = (double *)malloc(sizeof(double) * nM);
    P->vol = (double *)malloc(sizeof(double) * nM);
    P->mH = (double *)malloc(sizeof(double) * nM);
    P->u = (double *)calloc((size_t)nM, sizeof(double));
    P->v = (double *)calloc((size_t)nm * nM, sizeof(double));
    P->is_dir = (int *)calloc((size_t)nM, sizeof(int));
    if (!P->prm || !P->rp || !P->ci || !P->rpH || !P->ciH || !P->Mv || !P->Av || !P->Rv ||
        !P->MH || !P->KH || !P->r || !P->gam || !P->vol || !P->mH || !P->u || !P->v || !P->is_dir) {
        or_destroy(P);
        *err = OR_E_OOM;
        return NULL;
    }
    if (P->nparam) memcpy(P->prm, prm, sizeof(double) * (size_t)nM * P->nparam);
    or_q1_pattern(Nm, P->rp, P->ci);
    or_q1_pattern(NM, P->rpH, P->ciH);

    int bad = 0;
#pragma omp parallel for schedule(dynamic, 4) reduction(| : bad)
    for (int i = 0; i < nM; ++i) {
        const double *pi = P->prm + (size_t)i * P->nparam;
        int e = or_assemble_q1(Nm, family, pi, P->D, P->rp, P->ci, P->Mv + nz * i, P->Av + nz * i,
                               P->Rv + nz * i);
        if (e) bad = 1;
        double *ri = P->r + (size_t)nm * i;
        double gsum = 0.0, vsum = 0.0;
        for (int j = 0; j < nm; ++j) {
            double rs = 0.0, ms = 0.0;
            for (int k = P->rp[j]; k < P->rp[j + 1]; ++k) {
                rs += P->Rv[nz * i + k];
                ms += P->Mv[nz * i + k];
            }
            ri[j] = rs;
            gsum += rs;
            vsum += ms;
        }
        P->gam[i] = gsum;
        P->vol[i] = vsum;
    }
    if (bad) {
        or_destroy(P);
        *err = OR_E_BAD_JACOBIAN;
        return NULL;
    }
    /* macro Q1 mass and stiffness on Omega (first equation of Eq. (17)) */
    const double I2[3] = {1.0, 0.0, 1.0};
    or_assemble_q1(NM, 0, NULL, I2, P->rpH, P->ciH, P->MH, P->KH, NULL);
    for (int k = 0; k < nM; ++k) {
        double s = 0.0;
        for (int e = P->rpH[k]; e < P->rpH[k + 1]; ++e) s += P->MH[e];
        P->mH[k] = s;
        P->is_dir[k] = (bc == 1) && boundary_node(NM, k);
    }
    return P;
}

int or_set_state(or_problem *P, const double *u, const double *v)
{
    memcpy(P->u, u, sizeof(double) * P->nM);
    if (v)
        memcpy(P->v, v, sizeof(double) * (size_t)P->nM * P->nm);
    else
        memset(P->v, 0, sizeof(double) * (size_t)P->nM * P->nm);
    return OR_OK;
}

static int set_opt(double **dst, const double *src, size_t n)
{
    free(*dst);
    *dst = NULL;
    if (!src) return OR_OK;
    *dst = (double *)malloc(sizeof(double) * n);
    if (!*dst) return OR_E_OOM;
    memcpy(*dst, src, sizeof(double) * n);
    return OR_OK;
}

/* Nodal source data used by the following steps (all optional):
 *   fv [nM][nm]    micro volume source at the micro nodes (physical values)
 *   g  [nM][Nm+1]  Robin data on the Robin edge nodes yhat = (1, q h)
 *   fu [nM]        macro volume source at the macro nodes
 *   ud [nM]        Dirichlet values (read on Dirichlet nodes only)
 * Load vectors are the mass (resp. boundary-mass) matrix times the nodal
 * values: b = M fv + R g for the micro problems, M_H fu - L G for the macro
 * problem with G_i = r_i^T g_i, the lumped counterpart of the coupling term. */
int or_set_sources(or_problem *P, const double *fv, const double *g, const double *fu,
                   const double *ud)
{
    int e = 0;
    e |= set_opt(&P->fv, fv, (size_t)P->nM * P->nm);
    e |= set_opt(&P->fu, fu, (size_t)P->nM);
    e |= set_opt(&P->ud, ud, (size_t)P->nM);
    free(P->g);
    P->g = NULL;
    if (g) {
        P->g = (double *)calloc((size_t)P->nM * P->nm, sizeof(double));
        if (!P->g) return OR_E_OOM;
        int n1 = P->Nm + 1;
        for (int i = 0; i < P->nM; ++i)
            for (int q = 0; q < n1; ++q)
                P->g[(size_t)i * P->nm + P->Nm + n1 * q] = g[(size_t)i * n1 + q];
    }
    return e ? OR_E_OOM : OR_OK;
}

static void build_S(or_problem *P, double dt)
{
    if (P->Sv && P->Sdt == dt) return;
    size_t nz = (size_t)P->nnz_m, tot = nz * P->nM;
    if (!P->Sv) P->Sv = (double *)malloc(sizeof(double) * tot);
#pragma omp parallel for schedule(static)
    for (long long e = 0; e < (long long)tot; ++e)
        P->Sv[e] = P->Mv[e] / dt + P->Av[e] + P->kappa * P->Rv[e];
    P->Sdt = dt;
}

/* One or more implicit Euler steps of the coupled system (Sec. 3.3: macro and
 * micro systems decoupled and iterated until the change is below tolerance;
 * here micro first, then macro, which has the same fixed point). */
int or_step(or_problem *P, double dt, int nsteps, double cg_tol, int cg_maxit,
            double coupling_tol, int coupling_maxit, double macro_tol)
{
    int nm = P->nm, nM = P->nM;
    size_t nz = (size_t)P->nnz_m;
    int status = OR_OK;
    build_S(P, dt);
    double *c = (double *)malloc(sizeof(double) * (size_t)nm * nM);  /* micro RHS without the u term */
    double *vk = (double *)malloc(sizeof(double) * (size_t)nm * nM); /* micro iterate */
    double *rho = (double *)malloc(sizeof(double) * nM);
    double *Gsrc = (double *)calloc((size_t)nM, sizeof(double));
    double *cH = (double *)malloc(sizeof(double) * nM);
    double *bH = (double *)malloc(sizeof(double) * nM);
    double *uk = (double *)malloc(sizeof(double) * nM);
    double *unew = (double *)malloc(sizeof(double) * nM);
    double *AH = (double *)malloc(sizeof(double) * P->nnz_M);
    double *tmpH = (double *)malloc(sizeof(double) * nM * 5);
    double *mres = (double *)malloc(sizeof(double) * nM);
    if (!c || !vk || !rho || !Gsrc || !cH || !bH || !uk || !unew || !AH || !tmpH || !mres) {
        status = OR_E_OOM;
        goto done;
    }
    /* macro system matrix with Dirichlet rows/columns eliminated symmetrically */
    for (int k = 0; k < nM; ++k)
        for (int e = P->rpH[k]; e < P->rpH[k + 1]; ++e) {
            int j = P->ciH[e];
            double a = P->MH[e] / dt + P->Du * P->KH[e];
            if (j == k) a += P->kappa * P->mH[k] * P->gam[k];
            if (P->is_dir[k] || P->is_dir[j]) a = (j == k) ? 1.0 : 0.0;
            AH[e] = a;
        }

    for (int step = 0; step < nsteps; ++step) {
        /* per-step right-hand sides: c_i = M_i v_i^n/dt + M_i fv_i + R_i g_i */
#pragma omp parallel for schedule(dynamic, 8)
        for (int i = 0; i < nM; ++i) {
            const double *Mi = P->Mv + nz * i, *Ri = P->Rv + nz * i;
            const double *vi = P->v + (size_t)nm * i;
            double *ci = c + (size_t)nm * i;
            for (int j = 0; j < nm; ++j) {
                double acc = 0.0;
                for (int k = P->rp[j]; k < P->rp[j + 1]; ++k) {
                    int l = P->ci[k];
                    double w = vi[l] / dt;
                    if (P->fv) w += P->fv[(size_t)nm * i + l];
                    acc += Mi[k] * w;
                    if (P->g) acc += Ri[k] * P->g[(size_t)nm * i + l];
                }
                ci[j] = acc;
            }
            if (P->g) Gsrc[i] = dot(nm, P->r + (size_t)nm * i, P->g + (size_t)nm * i);
            memcpy(vk + (size_t)nm * i, vi, sizeof(double) * nm);
        }
        /* macro: cH = M_H u^n/dt + M_H fu - L G */
        for (int k = 0; k < nM; ++k) {
            double acc = 0.0;
            for (int e = P->rpH[k]; e < P->rpH[k + 1]; ++e) {
                int j = P->ciH[e];
                acc += P->MH[e] * (P->u[j] / dt + (P->fu ? P->fu[j] : 0.0));
            }
            cH[k] = acc - P->mH[k] * Gsrc[k];
        }
        memcpy(uk, P->u, sizeof(double) * nM);
        for (int k = 0; k < nM; ++k)
            if (P->is_dir[k] && P->ud) uk[k] = P->ud[k];

        int it;
        double change = 0.0;
        for (it = 1; it <= coupling_maxit; ++it) {
            /* micro solves with the current macro iterate (Sec. 3.5: systems
               distributed over the processors) */
            int mstat = OR_OK;
            int64_t iters_sum = 0;
            int iters_max = 0;
#pragma omp parallel reduction(+ : iters_sum) reduction(max : iters_max) reduction(| : mstat)
            {
                double *b = (double *)malloc(sizeof(double) * nm);
                double *work = (double *)malloc(sizeof(double) * 4 * nm);
#pragma omp for schedule(dynamic, 4)
                for (int i = 0; i < nM; ++i) {
                    const double *ri = P->r + (size_t)nm * i;
                    const double *ci = c + (size_t)nm * i;
                    double *xi = vk + (size_t)nm * i;
                    for (int j = 0; j < nm; ++j) b[j] = ci[j] + P->kappa * uk[i] * ri[j];
                    int iters;
                    double rr;
                    int e = or_pcg(nm, P->rp, P->ci, P->Sv + nz * i, b, xi, cg_tol, cg_maxit, work,
                                   &iters, &rr);
                    if (e) mstat |= 1;
                    iters_sum += iters;
                    if (iters > iters_max) iters_max = iters;
                    rho[i] = dot(nm, ri, xi);
                }
                free(b);
                free(work);
            }
            P->st.inner_iters += iters_sum;
            P->st.micro_solves += nM;
            if (iters_max > P->st.max_inner_iters) P->st.max_inner_iters = iters_max;
            if (mstat && status == OR_OK) status = OR_E_NOT_CONVERGED;

            /* macro solve with the new micro fluxes (first line of Eq. (17),
               coupling integral lumped at the nodes) */
            for (int k = 0; k < nM; ++k) bH[k] = cH[k] + P->kappa * P->mH[k] * rho[k];
            for (int k = 0; k < nM; ++k) {
                if (P->is_dir[k]) continue;
                for (int e = P->rpH[k]; e < P->rpH[k + 1]; ++e) {
                    int j = P->ciH[e];
                    if (P->is_dir[j]) bH[k] -= (P->MH[e] / dt + P->Du * P->KH[e]) * uk[j];
                }
            }
            for (int k = 0; k < nM; ++k)
                if (P->is_dir[k]) bH[k] = uk[k];
            memcpy(unew, uk, sizeof(double) * nM);
            int hit;
            double hres;
            int e = or_pcg(nM, P->rpH, P->ciH, AH, bH, unew, macro_tol, 100000, tmpH, &hit, &hres);
            P->st.macro_iters += hit;
            if (e && status == OR_OK) status = e;

            /* stop rule: relative change of the macro iterate */
            double dn = 0.0, un = 0.0;
            for (int k = 0; k < nM; ++k) {
                double d = unew[k] - uk[k];
                dn += d * d;
                un += unew[k] * unew[k];
            }
            change = un > 0.0 ? sqrt(dn / un) : sqrt(dn);
            /* paper-style monitor: macro residual + mean micro residual of the
               coupled system at (u_new, v_k) (Sec. 3.5) */
            double msum = 0.0;
            for (int i = 0; i < nM; ++i) {
                const double *ri = P->r + (size_t)nm * i;
                const double *ci = c + (size_t)nm * i;
                double bn = 0.0, dn2 = 0.0;
                for (int j = 0; j < nm; ++j) {
                    double bj = ci[j] + P->kappa * unew[i] * ri[j];
                    double dj = P->kappa * (unew[i] - uk[i]) * ri[j];
                    bn += bj * bj;
                    dn2 += dj * dj;
                }
                mres[i] = bn > 0.0 ? sqrt(dn2 / bn) : 0.0;
                msum += mres[i];
            }
            P->st.paper_residual = hres + msum / nM;
            memcpy(uk, unew, sizeof(double) * nM);
            if (change <= coupling_tol) break;
        }
        if (it > coupling_maxit) {
            it = coupling_maxit;
            if (status == OR_OK) status = OR_E_NOT_CONVERGED;
        }
        P->st.coupling_iters_last = it;
        P->st.coupling_iters_total += it;
        P->st.coupling_change = change;
        /* commit */
        memcpy(P->u, uk, sizeof(double) * nM);
        memcpy(P->v, vk, sizeof(double) * (size_t)nm * nM);
    }
done:
    free(c); free(vk); free(rho); free(Gsrc); free(cH); free(bH); free(uk); free(unew);
    free(AH); free(tmpH); free(mres);
    if (P->st.status == OR_OK) P->st.status = status;
    return status;
}

/* ------------------------------------------------------------------------ */
/* Accessors                                                                */
/* ------------------------------------------------------------------------ */
void or_get_u(const or_problem *P, double *u) { memcpy(u, P->u, sizeof(double) * P->nM); }
void or_get_v(const or_problem *P, double *v) { memcpy(v, P->v, sizeof(double) * (size_t)P->nM * P->nm); }

/* micro averages vbar_i = int_{Y_x} v / |Y_x| = 1^T M_i v_i / vol_i */
void or_get_vbar(const or_problem *P, double *vbar)
{
    size_t nz = (size_t)P->nnz_m;
    for (int i = 0; i < P->nM; ++i) {
        const double *vi = P->v + (size_t)P->nm * i;
        double s = 0.0;
        for (int j = 0; j < P->nm; ++j)
            for (int k = P->rp[j]; k < P->rp[j + 1]; ++k) s += P->Mv[nz * i + k] * vi[P->ci[k]];
        vbar[i] = s / P->vol[i];
    }
}

/* boundary flux into each micro problem: F_i = kappa (|Gam_i| u_i - r_i^T v_i) (+ G_i) */
void or_get_flux(const or_problem *P, double *flux)
{
    for (int i = 0; i < P->nM; ++i) {
        const double *vi = P->v + (size_t)P->nm * i;
        double f = P->kappa * (P->gam[i] * P->u[i] - dot(P->nm, P->r + (size_t)P->nm * i, vi));
        if (P->g) f += dot(P->nm, P->r + (size_t)P->nm * i, P->g + (size_t)P->nm * i);
        flux[i] = f;
    }
}

void or_get_geometry(const or_problem *P, double *gam, double *vol, double *mH)
{
    if (gam) memcpy(gam, P->gam, sizeof(double) * P->nM);
    if (vol) memcpy(vol, P->vol, sizeof(double) * P->nM);
    if (mH) memcpy(mH, P->mH, sizeof(double) * P->nM);
}

void or_get_r(const or_problem *P, double *r) { memcpy(r, P->r, sizeof(double) * (size_t)P->nM * P->nm); }

int or_nnz_micro(const or_problem *P) { return P->nnz_m; }
int or_nnz_macro(const or_problem *P) { return P->nnz_M; }

/* which: 0 M, 1 A, 2 R of instance i; pattern copied when rowptr/col != NULL */
void or_get_micro_csr(const or_problem *P, int i, int which, int *rowptr, int *col, double *val)
{
    size_t nz = (size_t)P->nnz_m;
    if (rowptr) memcpy(rowptr, P->rp, sizeof(int) * (P->nm + 1));
    if (col) memcpy(col, P->ci, sizeof(int) * nz);
    const double *src = which == 0 ? P->Mv : which == 1 ? P->Av : P->Rv;
    if (val) memcpy(val, src + nz * i, sizeof(double) * nz);
}

/* which: 0 M_H, 1 K_H */
void or_get_macro_csr(const or_problem *P, int which, int *rowptr, int *col, double *val)
{
    if (rowptr) memcpy(rowptr, P->rpH, sizeof(int) * (P->nM + 1));
    if (col) memcpy(col, P->ciH, sizeof(int) * P->nnz_M);
    if (val) memcpy(val, which == 0 ? P->MH : P->KH, sizeof(double) * P->nnz_M);
}

void or_get_stats(const or_problem *P, or_stats *s) { *s = P->st; }
void or_reset_stats(or_problem *P) { memset(&P->st, 0, sizeof(P->st)); }

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
