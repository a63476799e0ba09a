// tsf3.cu -- the stationary three-field system (Eq. (5): u, v, w with the
// inflow edge Gamma_I and the outflow edge Gamma_O) by exact elimination of
// the micro unknowns.
//
// With S_i = A_i + kappa_2 R_I,i + kappa_4 R_O,i (the micro operator of
// Eq. (17) for node i), the micro solution is affine in the two macro values
// of its node:
//     v_i = v0_i + u_i phi_I,i + w_i phi_O,i,
//     S_i phi_I = kappa_1 r_I,   S_i phi_O = kappa_3 r_O,   S_i v0 = b_i (sources),
// r_I = R_I 1, r_O = R_O 1.  Substituted into the lumped macro equations this
// leaves one coupled system in (u, w).  Scaled by kappa_1/kappa_2 (u rows)
// and kappa_3/kappa_4 (w rows), it is symmetric positive definite (it is the
// Schur complement of the symmetrised monolithic matrix):
//     s_u [K_H u + L (kappa_1 Gam_I - kappa_2 b_II) u] - kappa_1 kappa_3 L c w = s_u F_u + kappa_1 L rho_I0
//     s_w [D^w K_H w + L (kappa_3 Gam_O - kappa_4 b_OO) w] - kappa_1 kappa_3 L c u = s_w F_w + kappa_3 L rho_O0
// with b_II = r_I^T phi_I, b_OO = r_O^T phi_O, c = r_I^T S^-1 r_O (taken as
// the mean of r_I^T phi_O / kappa_3 and r_O^T phi_I / kappa_1, which agree up
// to the solver tolerance), rho_I0 = r_I^T v0, rho_O0 = r_O^T v0, F the macro
// loads.  One solve of it, then v follows pointwise.  The paper iterates
// between the scales instead (Sec. 3.3); both reach the same discrete
// solution.
//
// Kernels: geometry with four edges (k3_geometry), right-hand sides and the
// stored-residual set-up of the micro solves (k3_setup), the micro solves
// (the iterative kernels of tsf_micro.cu, or the direct banded-Cholesky
// solves of tsf_band.cu: S does not change between the three right-hand
// sides and the re-solves), edge moments and macro coefficients
// (k3_moments), the coupled macro PCG in one thread block (k3_macro), and the
// commit.
#include "tsfem3.h"
#include "tsf_geom.cuh"

#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

namespace tsf {

namespace cg = cooperative_groups;

// ---------------------------------------------------------------------------
// geometry: M, S = A + kappa_2 R_I + kappa_4 R_O, and the edge masses of all
// four edges ([4][nM][n1]: diagonal, coupling to the next node, r = R 1)
// ---------------------------------------------------------------------------
struct Geom3Args {
    int Nm, n1, nm, nmp, nM;
    int affine;             // 1: identity or affine family (F constant per problem)
    const double* prm5;
    double D11, D12, D22, k2, k4;
    double* M64;
    double* S64;
    float* S32;
    float* S32lo;
    double* lm;
    double* eRd;
    double* eRu;
    double* er;
    DevCtl* ctl;
};

// One thread per (micro node, instance); nodes whose map has b = 0 take the
// reference-table path (as in k_geometry), the others the quadrature points.
__global__ void __launch_bounds__(128) k3_geometry(Geom3Args a) {
    __shared__ double ref[64];
    fill_reference_tables(ref);  // by the first 16 threads, before any thread leaves
    __syncthreads();
    const int j = blockIdx.y * blockDim.x + threadIdx.x;
    const int i = blockIdx.x;
    if (j >= a.nmp) return;
    const size_t pl = (size_t)a.nmp;
    double* M64 = a.M64 + (size_t)i * kPlanes * pl;
    double* S64 = a.S64 + (size_t)i * kPlanes * pl;
    float* S32 = a.S32 + (size_t)i * kPlanes * pl;
    float* S32lo = a.S32lo ? a.S32lo + (size_t)i * kPlanes * pl : nullptr;
    if (j >= a.nm) {
        for (int k = 0; k < kPlanes; ++k) {
            M64[k * pl + j] = 0.0;
            S64[k * pl + j] = 0.0;
            S32[k * pl + j] = 0.0f;
            if (S32lo) S32lo[k * pl + j] = 0.0f;
        }
        a.lm[(size_t)i * pl + j] = 0.0;
        return;
    }
    const int N = a.Nm, n1 = a.n1;
    const int p = j % n1, q = j / n1;
    const Deform d = load_deform(a.prm5, i);
    double m[kPlanes], k[kPlanes], lump;
    bool bad;
    if (d.bpi == 0.0) node_couplings_affine(d, a.D11, a.D12, a.D22, p, q, N, ref, m, k, lump, bad);
    else node_couplings(d, a.D11, a.D12, a.D22, p, q, N, m, k, lump, bad);
    // edge masses; the Robin edges add to S (their couplings run along q: plane 2)
    const bool on_edge[4] = {p == 0, p == N, q == 0, q == N};
    const int along[4] = {q, q, p, p};
    const double kap[4] = {a.k2, a.k4, 0.0, 0.0};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        if (!on_edge[e]) continue;
        double Rd, Ru, Rdn;
        edge_node_mass(d, e, along[e], N, Rd, Ru, Rdn);
        const size_t o = ((size_t)e * a.nM + i) * n1 + along[e];
        a.eRd[o] = Rd;
        a.eRu[o] = Ru;
        a.er[o] = Rd + Ru + Rdn;
        if (e < 2) {
            k[0] = fma(kap[e], Rd, k[0]);
            k[2] = fma(kap[e], Ru, k[2]);
        }
    }
#pragma unroll
    for (int c = 0; c < kPlanes; ++c) {
        M64[c * pl + j] = m[c];
        S64[c * pl + j] = k[c];
        const float hi = (float)k[c];
        S32[c * pl + j] = hi;
        if (S32lo) S32lo[c * pl + j] = (float)(k[c] - (double)hi);
    }
    a.lm[(size_t)i * pl + j] = lump;
    if (bad) atomicOr(&a.ctl->geom_error, 1);
}

// ---------------------------------------------------------------------------
// right-hand sides of the micro solves (0: v0, 1: phi_I, 2: phi_O) and the
// stored-residual set-up from a zero initial guess: res = c, u_used = 0,
// bnorm = (||c||^2, 0, 0).  One block per instance.
// ---------------------------------------------------------------------------
struct Setup3Args {
    int n1, nm, nmp, nM;
    int nsolve;             // 1: v0 only, 3: v0, phi_I, phi_O
    double k1, k3;
    const double* M64;
    const double* eRd;
    const double* eRu;
    const double* er;
    const double* fv;       // [nM][nmp] or nullptr
    const double* gI;       // [nM][n1] or nullptr
    const double* gO;
    const double* gN;       // [nM][2][n1] or nullptr
    double* c[3];
    double* x[3];
    double* res[3];
    double* uu[3];
    double* bnorm[3];
    double* G;              // [nM][2] out: r_I^T g_1, r_O^T g_2
};

// (R_e g)_t along edge e for nodal edge data g (n1 values)
__device__ __forceinline__ double edge_apply(const double* Rd, const double* Ru, const double* g, int t, int n1) {
    double y = Rd[t] * g[t];
    if (t + 1 < n1) y = fma(Ru[t], g[t + 1], y);
    if (t > 0) y = fma(Ru[t - 1], g[t - 1], y);
    return y;
}

__global__ void __launch_bounds__(256) k3_setup(Setup3Args a) {
    __shared__ double buf[5 * 32];
    const int i = blockIdx.x, n1 = a.n1, N = n1 - 1;
    const size_t pl = (size_t)a.nmp;
    const double* M = a.M64 + (size_t)i * kPlanes * pl;
    auto edge = [&](const double* base, int e) { return base + ((size_t)e * a.nM + i) * n1; };
    const double* gI = a.gI ? a.gI + (size_t)i * n1 : nullptr;
    const double* gO = a.gO ? a.gO + (size_t)i * n1 : nullptr;
    const double* gB = a.gN ? a.gN + (size_t)i * 2 * n1 : nullptr;
    const double* gT = a.gN ? gB + n1 : nullptr;
    const double* fv = a.fv ? a.fv + (size_t)i * pl : nullptr;
    double s[5] = {0.0, 0.0, 0.0, 0.0, 0.0};   // ||c0||^2, ||cI||^2, ||cO||^2, r_I^T g_1, r_O^T g_2
    for (int j = threadIdx.x; j < a.nmp; j += blockDim.x) {
        double c[3] = {0.0, 0.0, 0.0};
        if (j < a.nm) {
            const int p = j % n1, q = j / n1;
            double b = fv ? plane_apply(M, pl, fv, j, p, q, n1) : 0.0;
            if (p == 0 && gI) b += edge_apply(edge(a.eRd, kEdgeLeft), edge(a.eRu, kEdgeLeft), gI, q, n1);
            if (p == N && gO) b += edge_apply(edge(a.eRd, kEdgeRight), edge(a.eRu, kEdgeRight), gO, q, n1);
            if (q == 0 && gB) b += edge_apply(edge(a.eRd, kEdgeBottom), edge(a.eRu, kEdgeBottom), gB, p, n1);
            if (q == N && gT) b += edge_apply(edge(a.eRd, kEdgeTop), edge(a.eRu, kEdgeTop), gT, p, n1);
            c[0] = b;
            if (p == 0) {
                const double r = edge(a.er, kEdgeLeft)[q];
                c[1] = a.k1 * r;
                if (gI) s[3] = fma(r, gI[q], s[3]);
            }
            if (p == N) {
                const double r = edge(a.er, kEdgeRight)[q];
                c[2] = a.k3 * r;
                if (gO) s[4] = fma(r, gO[q], s[4]);
            }
        }
        for (int t = 0; t < a.nsolve; ++t) {
            const size_t o = (size_t)i * pl + j;
            a.c[t][o] = c[t];
            a.x[t][o] = 0.0;
            a.res[t][o] = c[t];
            s[t] = fma(c[t], c[t], s[t]);
        }
    }
    block_allreduce<double, 5>(s, buf);
    if (threadIdx.x == 0) {
        for (int t = 0; t < a.nsolve; ++t) {
            a.uu[t][i] = 0.0;
            double* bn = a.bnorm[t] + (size_t)i * 3;
            bn[0] = s[t];
            bn[1] = 0.0;
            bn[2] = 0.0;
        }
        a.G[2 * i] = s[3];
        a.G[2 * i + 1] = s[4];
    }
}

// ---------------------------------------------------------------------------
// edge moments of the micro solutions and the per-node coefficients of the
// scaled macro system: coef[k] = (d_u, d_w, off, b_u, b_w); one warp per node
// ---------------------------------------------------------------------------
struct Moments3Args {
    int n1, nm, nmp, nM, NM;
    double H, k1, k2, k3, k4;
    const double* er;
    const double* lm;
    const double* phiI;
    const double* phiO;
    const double* v0;
    const double* G;
    double* coef;
    double* vol;
};

__global__ void __launch_bounds__(128) k3_moments(Moments3Args a) {
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= a.nM) return;
    const int n1 = a.n1;
    const size_t pl = (size_t)a.nmp, base = (size_t)i * pl;
    const double* rI = a.er + ((size_t)kEdgeLeft * a.nM + i) * n1;
    const double* rO = a.er + ((size_t)kEdgeRight * a.nM + i) * n1;
    // gI, gO, b_II, b_IO, b_OI, b_OO, rho_I0, rho_O0, vol
    double s[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int q = lane; q < n1; q += 32) {
        const size_t jl = base + (size_t)n1 * q, jr = jl + n1 - 1;
        const double ri = rI[q], ro = rO[q];
        s[0] += ri;
        s[1] += ro;
        s[2] = fma(ri, a.phiI[jl], s[2]);
        s[3] = fma(ri, a.phiO[jl], s[3]);
        s[4] = fma(ro, a.phiI[jr], s[4]);
        s[5] = fma(ro, a.phiO[jr], s[5]);
        s[6] = fma(ri, a.v0[jl], s[6]);
        s[7] = fma(ro, a.v0[jr], s[7]);
    }
    for (int j = lane; j < a.nm; j += 32) s[8] += a.lm[base + j];
#pragma unroll
    for (int t = 0; t < 9; ++t)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s[t] += __shfl_xor_sync(0xffffffffu, s[t], o);
    if (lane == 0) {
        const int N1 = a.NM + 1, p = i % N1, q = i / N1;
        const double cx = (p == 0 || p == a.NM) ? 1.0 : 2.0, cy = (q == 0 || q == a.NM) ? 1.0 : 2.0;
        const double m = cx * cy * 0.25 * a.H * a.H;
        const double su = a.k1 / a.k2, sw = a.k3 / a.k4;
        const double c = 0.5 * (s[3] / a.k3 + s[4] / a.k1);
        double* o = a.coef + (size_t)i * 5;
        o[0] = su * m * (a.k1 * s[0] - a.k2 * s[2]);
        o[1] = sw * m * (a.k3 * s[1] - a.k4 * s[5]);
        o[2] = -a.k1 * a.k3 * m * c;
        o[3] = fma(a.k1 * m, s[6], -su * m * a.G[2 * i]);
        o[4] = fma(a.k3 * m, s[7], -sw * m * a.G[2 * i + 1]);
        a.vol[i] = s[8];
    }
}

// ---------------------------------------------------------------------------
// coupled macro solve in (u, w): PCG with 2x2 block-Jacobi preconditioner,
// matrix-free on the uniform mesh, one cooperative grid
// ---------------------------------------------------------------------------
constexpr int kMacro3Threads = 256;

struct Macro3Args {
    int NM, N1, nM, dir_mask;
    double H, Dw, su, sw;
    const double* coef;
    const double* fu;
    const double* fw;
    const double* ud;
    const double* gu;
    const double* gw;
    double* u;
    double* w;
    double* x;              // [2 nM] scratch: (u, w)
    double* r;
    double* z;
    double* pv;
    double* qv;
    double* pinv;           // [nM][3] inverse 2x2 diagonal blocks
    double tol;
    int maxit;
    DevCtl* ctl;
};

__device__ __forceinline__ bool dir_node3(int mask, int N, int p, int q) {
    return ((mask & 1) && q == 0) || ((mask & 2) && p == N) || ((mask & 4) && q == N) || ((mask & 8) && p == 0);
}

// K_H x at node (p, q): Ke = 1/6 [4 -1 -1 -2] per cell (diag, E/W, N/S, diagonal)
__device__ __forceinline__ double stiff_apply(const double* x, int k, int p, int q, int N, int n1) {
    const double cx = (p == 0 || p == N) ? 1.0 : 2.0, cy = (q == 0 || q == N) ? 1.0 : 2.0;
    const bool e = p < N, w = p > 0, nn = q < N, s = q > 0;
    const double ew = (e ? x[k + 1] : 0.0) + (w ? x[k - 1] : 0.0);
    const double ns = (nn ? x[k + n1] : 0.0) + (s ? x[k - n1] : 0.0);
    const double dg = ((e && nn) ? x[k + n1 + 1] : 0.0) + ((w && nn) ? x[k + n1 - 1] : 0.0) +
                      ((e && s) ? x[k - n1 + 1] : 0.0) + ((w && s) ? x[k - n1 - 1] : 0.0);
    return (4.0 / 6.0) * cx * cy * x[k] - (1.0 / 6.0) * (cy * ew + cx * ns) - (1.0 / 3.0) * dg;
}

// M_H f at node (p, q): Me = H^2/36 [4 2 2 1]
__device__ __forceinline__ double mass_apply(const double* f, int k, int p, int q, int N, int n1, double H) {
    const double cx = (p == 0 || p == N) ? 1.0 : 2.0, cy = (q == 0 || q == N) ? 1.0 : 2.0;
    const bool e = p < N, w = p > 0, nn = q < N, s = q > 0;
    const double ew = (e ? f[k + 1] : 0.0) + (w ? f[k - 1] : 0.0);
    const double ns = (nn ? f[k + n1] : 0.0) + (s ? f[k - n1] : 0.0);
    const double dg = ((e && nn) ? f[k + n1 + 1] : 0.0) + ((w && nn) ? f[k + n1 - 1] : 0.0) +
                      ((e && s) ? f[k - n1 + 1] : 0.0) + ((w && s) ? f[k - n1 - 1] : 0.0);
    return (H * H / 36.0) * (4.0 * cx * cy * f[k] + 2.0 * cy * ew + 2.0 * cx * ns + dg);
}

// int_boundary g xi_k for per-edge nodal data g [4][n1] (edges bottom, right,
// top, left; skip = edges not to load): 1D Q1 mass H/6 [2 1; 1 2]
__device__ __forceinline__ double boundary_apply(const double* g, int skip, int p, int q, int N, int n1, double H) {
    double y = 0.0;
    const bool on[4] = {q == 0, p == N, q == N, p == 0};
    const int t[4] = {p, q, p, q};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        if (!on[e] || (skip >> e & 1)) continue;
        const double* ge = g + (size_t)e * n1;
        const int s = t[e];
        if (s < N) y += (H / 6.0) * (2.0 * ge[s] + ge[s + 1]);
        if (s > 0) y += (H / 6.0) * (ge[s - 1] + 2.0 * ge[s]);
    }
    return y;
}

__device__ __forceinline__ void macro3_apply(const Macro3Args& a, const double* x, double* y, int k, int p, int q) {
    const int N = a.NM, n1 = a.N1, nM = a.nM;
    const double* c = a.coef + (size_t)k * 5;
    const double xu = x[k], xw = x[nM + k];
    y[k] = dir_node3(a.dir_mask, N, p, q)
               ? 0.0
               : fma(a.su, stiff_apply(x, k, p, q, N, n1), fma(c[0], xu, c[2] * xw));
    y[nM + k] = fma(a.sw * a.Dw, stiff_apply(x + nM, k, p, q, N, n1), fma(c[1], xw, c[2] * xu));
}

// Sum over the blocks of the per-block partials part[b][slot] (after a grid
// barrier); every block sums them in the same order, so all get the same value.
__device__ __forceinline__ double grid_total(const double* part, int slot, double* buf) {
    double v[1] = {0.0};
    for (int b = threadIdx.x; b < gridDim.x; b += blockDim.x) v[0] += part[4 * b + slot];
    block_allreduce<double, 1>(v, buf);
    return v[0];
}

// One cooperative grid (all blocks resident), one macro node per thread for
// both fields; three grid barriers per CG iteration.  part: [gridDim.x][4].
__global__ void __launch_bounds__(kMacro3Threads) k3_macro(Macro3Args a, double* part) {
    cg::grid_group grid = cg::this_grid();
    // four reduction buffers of 64 (a two-value block reduction uses 64);
    // consecutive reductions rotate through them, so a buffer is reused only
    // after three more block-wide barriers
    __shared__ double red[4 * 64];
    int rb = 0;
    auto nextbuf = [&]() { double* b = red + 64 * rb; rb = (rb + 1) & 3; return b; };
    const int nM = a.nM, n1 = a.N1, N = a.NM;
    const int T = gridDim.x * blockDim.x;
    const int k0 = blockIdx.x * blockDim.x + threadIdx.x;
    auto block_partial = [&](double v, int slot) {
        double t[1] = {v};
        block_allreduce<double, 1>(t, nextbuf());
        if (threadIdx.x == 0) part[4 * blockIdx.x + slot] = t[0];
    };
    auto block_partial2 = [&](double v0, double v1, int slot) {
        double t[2] = {v0, v1};
        block_allreduce<double, 2>(t, nextbuf());
        if (threadIdx.x == 0) {
            part[4 * blockIdx.x + slot] = t[0];
            part[4 * blockIdx.x + slot + 1] = t[1];
        }
    };
    // right-hand side (in q), initial iterate (Dirichlet values of u, zero
    // elsewhere) and the inverse 2x2 diagonal blocks
    for (int k = k0; k < nM; k += T) {
        const int p = k % n1, q = k / n1;
        const double* c = a.coef + (size_t)k * 5;
        const bool dir = dir_node3(a.dir_mask, N, p, q);
        double bu = c[3], bw = c[4];
        double lu = 0.0, lw = 0.0;
        if (a.fu) lu += mass_apply(a.fu, k, p, q, N, n1, a.H);
        if (a.gu) lu += boundary_apply(a.gu, a.dir_mask, p, q, N, n1, a.H);
        if (a.fw) lw += mass_apply(a.fw, k, p, q, N, n1, a.H);
        if (a.gw) lw += boundary_apply(a.gw, 0, p, q, N, n1, a.H);
        bu = fma(a.su, lu, bu);
        bw = fma(a.sw, lw, bw);
        a.qv[k] = dir ? 0.0 : bu;
        a.qv[nM + k] = bw;
        a.x[k] = dir ? (a.ud ? a.ud[k] : 0.0) : 0.0;
        a.x[nM + k] = 0.0;
        const double cx = (p == 0 || p == N) ? 1.0 : 2.0, cy = (q == 0 || q == N) ? 1.0 : 2.0;
        const double kd = (4.0 / 6.0) * cx * cy;
        const double a11 = fma(a.su, kd, c[0]), a22 = fma(a.sw * a.Dw, kd, c[1]), a12 = c[2];
        double* pi = a.pinv + (size_t)k * 3;
        if (dir) {
            pi[0] = 0.0;
            pi[1] = 0.0;
            pi[2] = 1.0 / a22;
        } else {
            const double id = 1.0 / fma(a11, a22, -a12 * a12);
            pi[0] = a22 * id;
            pi[1] = -a12 * id;
            pi[2] = a11 * id;
        }
    }
    grid.sync();
    // r = b - A x0 (x0 carries only the Dirichlet values), z = P r, p = z
    double rr = 0.0, rz = 0.0;
    for (int k = k0; k < nM; k += T) {
        const int p = k % n1, q = k / n1;
        macro3_apply(a, a.x, a.r, k, p, q);
        const double ru = a.qv[k] - a.r[k], rw = a.qv[nM + k] - a.r[nM + k];
        a.r[k] = ru;
        a.r[nM + k] = rw;
        const double* pi = a.pinv + (size_t)k * 3;
        const double zu = fma(pi[0], ru, pi[1] * rw), zw = fma(pi[1], ru, pi[2] * rw);
        a.pv[k] = zu;
        a.pv[nM + k] = zw;
        rr = fma(ru, ru, fma(rw, rw, rr));
        rz = fma(ru, zu, fma(rw, zw, rz));
    }
    block_partial2(rr, rz, 0);
    grid.sync();
    rr = grid_total(part, 0, nextbuf());
    rz = grid_total(part, 1, nextbuf());
    const double stop2 = a.tol * a.tol * rr;
    int it = 0;
    bool fail = false;
    if (rr > 0.0) {
        while (it < a.maxit) {
            // p is complete (barrier above / at the end of the previous iteration)
            double pq = 0.0;
            for (int k = k0; k < nM; k += T) {
                const int p = k % n1, q = k / n1;
                macro3_apply(a, a.pv, a.qv, k, p, q);
                pq = fma(a.pv[k], a.qv[k], fma(a.pv[nM + k], a.qv[nM + k], pq));
            }
            block_partial(pq, 2);
            grid.sync();
            pq = grid_total(part, 2, nextbuf());
            ++it;
            if (!(pq > 0.0)) {
                fail = true;
                break;
            }
            const double alpha = rz / pq;
            double rn2 = 0.0, rzn = 0.0;
            for (int k = k0; k < nM; k += T) {
                a.x[k] = fma(alpha, a.pv[k], a.x[k]);
                a.x[nM + k] = fma(alpha, a.pv[nM + k], a.x[nM + k]);
                const double ru = fma(-alpha, a.qv[k], a.r[k]), rw = fma(-alpha, a.qv[nM + k], a.r[nM + k]);
                a.r[k] = ru;
                a.r[nM + k] = rw;
                const double* pi = a.pinv + (size_t)k * 3;
                const double zu = fma(pi[0], ru, pi[1] * rw), zw = fma(pi[1], ru, pi[2] * rw);
                a.z[k] = zu;
                a.z[nM + k] = zw;
                rn2 = fma(ru, ru, fma(rw, rw, rn2));
                rzn = fma(ru, zu, fma(rw, zw, rzn));
            }
            block_partial2(rn2, rzn, 0);
            grid.sync();
            rn2 = grid_total(part, 0, nextbuf());
            rzn = grid_total(part, 1, nextbuf());
            if (!(rn2 == rn2)) {
                fail = true;
                break;
            }
            if (rn2 <= stop2) break;
            const double beta = rzn / rz;
            rz = rzn;
            for (int k = k0; k < nM; k += T) {
                a.pv[k] = fma(beta, a.pv[k], a.z[k]);
                a.pv[nM + k] = fma(beta, a.pv[nM + k], a.z[nM + k]);
            }
            grid.sync();
        }
        if (it >= a.maxit) fail = true;
    }
    for (int k = k0; k < nM; k += T) {
        a.u[k] = a.x[k];
        a.w[k] = a.x[nM + k];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.ctl->macro_iters += (unsigned long long)it;
        if (fail) set_status(a.ctl, kNotConverged);
    }
}

// v = v0 + u_i phi_I + w_i phi_O
__global__ void k3_commit(int nmp, size_t total, const double* __restrict__ v0, const double* __restrict__ phiI,
                          const double* __restrict__ phiO, const double* __restrict__ u,
                          const double* __restrict__ w, double* __restrict__ v) {
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        const size_t i = t / nmp;
        v[t] = fma(w[i], phiO[t], fma(u[i], phiI[t], v0[t]));
    }
}

}  // namespace tsf

using namespace tsf;

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct tsf3_ctx {
    tsf_options opt{};
    int device = 0, smem_optin = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int Nm = 0, n1 = 0, nm = 0, nmp = 0, NM = 0, N1 = 0, nM = 0, dir_mask = 0;
    double x0 = 0.0, L = 1.0;
    double D[3] = {1.0, 0.0, 1.0}, Dw = 1.0, kap[4] = {1.0, 1.0, 1.0, 1.0};
    int family = 0, nparam = 0;
    std::vector<void*> allocs;
    // device arrays
    double *params = nullptr, *prm5 = nullptr;
    float* map32 = nullptr;
    double *M64 = nullptr, *S64 = nullptr, *lm = nullptr;
    float* S32 = nullptr;
    // column-strip micro solves: the scaled operator and the diagonal scalings as FP32 pairs
    float4 *chat = nullptr, *chatlo = nullptr, *dsc = nullptr;
    double *eRd = nullptr, *eRu = nullptr, *er = nullptr;
    double *fu = nullptr, *fw = nullptr, *ud = nullptr, *gu = nullptr, *gw = nullptr;
    double *fv = nullptr, *gI = nullptr, *gO = nullptr, *gN = nullptr;
    bool has_fu = false, has_fw = false, has_ud = false, has_gu = false, has_gw = false;
    bool has_fv = false, has_gI = false, has_gO = false, has_gN = false;
    double *c[3] = {}, *x[3] = {}, *res[3] = {}, *uu[3] = {}, *bnorm[3] = {};
    int* iters = nullptr;
    double *zero = nullptr, *rho = nullptr, *G = nullptr, *coef = nullptr, *vol = nullptr;
    double *u = nullptr, *w = nullptr, *v = nullptr, *vbar = nullptr;
    double *mx = nullptr, *mr = nullptr, *mz = nullptr, *mp = nullptr, *mq = nullptr, *pinv = nullptr;
    double* mpart = nullptr;    // [blocks][4] partial sums of the cooperative macro solve
    DevCtl* ctl = nullptr;
    bool geom_valid = false, phi_valid = false, solved = false;
    int tiling = -1;
    // direct micro solves (tiling kTilingDirect): the FP32 band factor is kept while S stays the same
    float* Lband = nullptr;
    float* yband[3] = {nullptr, nullptr, nullptr};
    int* done[3] = {nullptr, nullptr, nullptr};
    int* open_count = nullptr;
    int* flag = nullptr;
    bool factor_valid = false;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaEvent_t bev[2] = {nullptr, nullptr};    // direct solve: factor and triangular-solve timing
    tsf3_stats stats{};
    std::string err;
};

static tsf_status fail3(tsf3_ctx* ctx, tsf_status st, const char* fmt, ...) {
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        ctx->err = buf;
    }
    return st;
}

#define CU3(call)                                                                                         \
    do {                                                                                                  \
        cudaError_t e_ = (call);                                                                          \
        if (e_ != cudaSuccess)                                                                            \
            return fail3(ctx, e_ == cudaErrorMemoryAllocation ? TSF_E_OOM : TSF_E_CUDA, "%s: %s (%s:%d)", \
                         #call, cudaGetErrorString(e_), __FILE__, __LINE__);                              \
    } while (0)

static void free_all(tsf3_ctx* ctx) {
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    for (void* p : ctx->allocs) cudaFree(p);
    ctx->allocs.clear();
    ctx->geom_valid = ctx->phi_valid = ctx->solved = ctx->factor_valid = false;
    ctx->Lband = nullptr;
    for (int t = 0; t < 3; ++t) ctx->yband[t] = nullptr;
    ctx->has_fu = ctx->has_fw = ctx->has_ud = ctx->has_gu = ctx->has_gw = false;
    ctx->has_fv = ctx->has_gI = ctx->has_gO = ctx->has_gN = false;
}

template <typename T>
static cudaError_t dalloc(tsf3_ctx* ctx, T** p, size_t n) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, std::max<size_t>(n, 1) * sizeof(T));
    if (e != cudaSuccess) return e;
    ctx->allocs.push_back(q);
    *p = reinterpret_cast<T*>(q);
    return cudaSuccess;
}

extern "C" {

tsf_status tsf3_create(tsf3_ctx** out, const tsf_options* opt) {
    if (!out) return TSF_E_ARG;
    *out = nullptr;
    tsf_options o;
    tsf_default_options(&o);
    if (opt) o = *opt;
    if ((o.precision != TSF_FP64 && o.precision != TSF_MIXED) || !(o.cg_tol > 0.0) || !(o.macro_tol > 0.0) ||
        o.cg_maxit < 1 || o.macro_maxit < 1 || o.tiling < -1 || o.tiling >= kNumTilings)
        return TSF_E_ARG;
    tsf3_ctx* ctx = new (std::nothrow) tsf3_ctx();
    if (!ctx) return TSF_E_OOM;
    ctx->opt = o;
    cudaError_t e = cudaGetDevice(&ctx->device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&ctx->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device);
    if (e == cudaSuccess) {
        if (o.cuda_stream) {
            ctx->stream = (cudaStream_t)o.cuda_stream;
        } else {
            e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
            ctx->own_stream = (e == cudaSuccess);
        }
    }
    for (int k = 0; k < 4 && e == cudaSuccess; ++k) e = cudaEventCreate(&ctx->ev[k]);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = cudaEventCreate(&ctx->bev[k]);
    if (e == cudaSuccess) e = configure_micro_kernels(ctx->smem_optin);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->ctl, sizeof(DevCtl));
    if (e == cudaSuccess) e = cudaMemset(ctx->ctl, 0, sizeof(DevCtl));
    if (e != cudaSuccess) {
        for (int k = 0; k < 4; ++k)
            if (ctx->ev[k]) cudaEventDestroy(ctx->ev[k]);
        for (int k = 0; k < 2; ++k)
            if (ctx->bev[k]) cudaEventDestroy(ctx->bev[k]);
        if (ctx->ctl) cudaFree(ctx->ctl);
        if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
        delete ctx;
        return TSF_E_CUDA;
    }
    *out = ctx;
    return TSF_OK;
}

void tsf3_destroy(tsf3_ctx* ctx) {
    if (!ctx) return;
    free_all(ctx);
    for (int k = 0; k < 4; ++k)
        if (ctx->ev[k]) cudaEventDestroy(ctx->ev[k]);
    for (int k = 0; k < 2; ++k)
        if (ctx->bev[k]) cudaEventDestroy(ctx->bev[k]);
    if (ctx->ctl) cudaFree(ctx->ctl);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

const char* tsf3_last_error(const tsf3_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

tsf_status tsf3_set_meshes(tsf3_ctx* ctx, int Nm, int NM, double x0, double L, int dir_mask) {
    if (!ctx) return TSF_E_ARG;
    if (Nm < 1 || Nm > 64) return fail3(ctx, TSF_E_ARG, "micro mesh must have 1..64 cells per side (got %d)", Nm);
    if (NM < 1 || NM > 256) return fail3(ctx, TSF_E_ARG, "macro mesh must have 1..256 cells per side (got %d)", NM);
    if (!(L > 0.0) || !std::isfinite(x0) || !std::isfinite(L)) return fail3(ctx, TSF_E_ARG, "bad macro domain");
    // without a Dirichlet edge the constant state u = c, v = c kappa_1/kappa_2,
    // w = c kappa_1 kappa_4 / (kappa_2 kappa_3) solves the homogeneous system
    // (Sec. 2.2 asks for a non-empty Dirichlet boundary)
    if (dir_mask < 1 || dir_mask > 15)
        return fail3(ctx, TSF_E_ARG, "dir_mask must name at least one Dirichlet edge (1..15, got %d)", dir_mask);
    free_all(ctx);
    ctx->Nm = Nm;
    ctx->n1 = Nm + 1;
    ctx->nm = ctx->n1 * ctx->n1;
    ctx->nmp = (ctx->nm + 31) / 32 * 32;
    ctx->NM = NM;
    ctx->N1 = NM + 1;
    ctx->nM = ctx->N1 * ctx->N1;
    ctx->x0 = x0;
    ctx->L = L;
    ctx->dir_mask = dir_mask;
    ctx->family = 0;
    ctx->nparam = 0;
    ctx->tiling = -1;
    const size_t nM = ctx->nM, F = nM * ctx->nmp, E = 4 * nM * ctx->n1;
    // a failed allocation leaves no half-built context behind: everything is
    // released and the meshes must be set again
    cudaError_t err = cudaSuccess;
#define AL(call)                            \
    do {                                    \
        if (err == cudaSuccess) err = (call); \
    } while (0)
    AL(dalloc(ctx, &ctx->params, nM * 6));
    AL(dalloc(ctx, &ctx->prm5, nM * 5));
    AL(dalloc(ctx, &ctx->map32, nM * 8));
    AL(dalloc(ctx, &ctx->M64, F * kPlanes));
    AL(dalloc(ctx, &ctx->S64, F * kPlanes));
    AL(dalloc(ctx, &ctx->S32, F * kPlanes));
    AL(dalloc(ctx, &ctx->chat, F * 2));
    AL(dalloc(ctx, &ctx->chatlo, F * 2));
    AL(dalloc(ctx, &ctx->dsc, F));
    AL(dalloc(ctx, &ctx->lm, F));
    AL(dalloc(ctx, &ctx->eRd, E));
    AL(dalloc(ctx, &ctx->eRu, E));
    AL(dalloc(ctx, &ctx->er, E));
    AL(dalloc(ctx, &ctx->fu, nM));
    AL(dalloc(ctx, &ctx->fw, nM));
    AL(dalloc(ctx, &ctx->ud, nM));
    AL(dalloc(ctx, &ctx->gu, 4 * (size_t)ctx->N1));
    AL(dalloc(ctx, &ctx->gw, 4 * (size_t)ctx->N1));
    AL(dalloc(ctx, &ctx->fv, F));
    AL(dalloc(ctx, &ctx->gI, nM * ctx->n1));
    AL(dalloc(ctx, &ctx->gO, nM * ctx->n1));
    AL(dalloc(ctx, &ctx->gN, 2 * nM * ctx->n1));
    for (int t = 0; t < 3; ++t) {
        AL(dalloc(ctx, &ctx->c[t], F));
        AL(dalloc(ctx, &ctx->x[t], F));
        AL(dalloc(ctx, &ctx->res[t], F));
        AL(dalloc(ctx, &ctx->uu[t], nM));
        AL(dalloc(ctx, &ctx->bnorm[t], 3 * nM));
    }
    AL(dalloc(ctx, &ctx->iters, nM));
    AL(dalloc(ctx, &ctx->zero, nM));
    AL(dalloc(ctx, &ctx->rho, nM));
    AL(dalloc(ctx, &ctx->G, 2 * nM));
    AL(dalloc(ctx, &ctx->coef, 5 * nM));
    AL(dalloc(ctx, &ctx->vol, nM));
    AL(dalloc(ctx, &ctx->u, nM));
    AL(dalloc(ctx, &ctx->w, nM));
    AL(dalloc(ctx, &ctx->v, F));
    AL(dalloc(ctx, &ctx->vbar, nM));
    AL(dalloc(ctx, &ctx->mx, 2 * nM));
    AL(dalloc(ctx, &ctx->mr, 2 * nM));
    AL(dalloc(ctx, &ctx->mz, 2 * nM));
    AL(dalloc(ctx, &ctx->mp, 2 * nM));
    AL(dalloc(ctx, &ctx->mq, 2 * nM));
    AL(dalloc(ctx, &ctx->pinv, 3 * nM));
    AL(dalloc(ctx, &ctx->mpart, 4 * ((nM + kMacro3Threads - 1) / kMacro3Threads) + 4));
    for (int t = 0; t < 3; ++t) AL(dalloc(ctx, &ctx->done[t], nM));
    AL(dalloc(ctx, &ctx->open_count, 1));
    AL(dalloc(ctx, &ctx->flag, 1));
    AL(cudaMemsetAsync(ctx->zero, 0, nM * sizeof(double), ctx->stream));
    AL(cudaMemsetAsync(ctx->fv, 0, F * sizeof(double), ctx->stream));
    AL(cudaMemsetAsync(ctx->eRd, 0, E * sizeof(double), ctx->stream));
    AL(cudaMemsetAsync(ctx->eRu, 0, E * sizeof(double), ctx->stream));
    AL(cudaMemsetAsync(ctx->er, 0, E * sizeof(double), ctx->stream));
#undef AL
    if (err != cudaSuccess) {
        free_all(ctx);
        ctx->nM = 0;
        cudaGetLastError();
        return fail3(ctx, err == cudaErrorMemoryAllocation ? TSF_E_OOM : TSF_E_CUDA,
                     "allocating the three-field state (%d x %d macro, %d x %d micro): %s", NM, NM, Nm, Nm,
                     cudaGetErrorString(err));
    }
    return TSF_OK;
}

tsf_status tsf3_set_physics(tsf3_ctx* ctx, const double D[3], double Dw, const double kappa[4]) {
    if (!ctx || !D || !kappa) return fail3(ctx, TSF_E_ARG, "null argument");
    if (!(D[0] > 0.0) || !(D[0] * D[2] - D[1] * D[1] > 0.0))
        return fail3(ctx, TSF_E_ARG, "D^v must be symmetric positive definite");
    if (!(Dw > 0.0)) return fail3(ctx, TSF_E_ARG, "D^w must be positive");
    for (int k = 0; k < 4; ++k)
        if (!(kappa[k] > 0.0) || !std::isfinite(kappa[k]))
            return fail3(ctx, TSF_E_ARG, "kappa_%d must be positive", k + 1);
    for (int k = 0; k < 3; ++k) ctx->D[k] = D[k];
    for (int k = 0; k < 4; ++k) ctx->kap[k] = kappa[k];
    ctx->Dw = Dw;
    ctx->geom_valid = ctx->phi_valid = ctx->factor_valid = false;
    return TSF_OK;
}

tsf_status tsf3_set_deformation(tsf3_ctx* ctx, int family, int nparam, const double* params, int on_device) {
    if (!ctx) return TSF_E_ARG;
    if (!ctx->nM) return fail3(ctx, TSF_E_STATE, "set the meshes first");
    static const int need[5] = {0, 1, 2, 6, 5};
    if (family < 0 || family > 4) return fail3(ctx, TSF_E_ARG, "unknown deformation family %d", family);
    if (nparam != need[family])
        return fail3(ctx, TSF_E_ARG, "family %d takes %d parameters (got %d)", family, need[family], nparam);
    if (nparam && !params) return fail3(ctx, TSF_E_ARG, "null parameters");
    if (nparam)
        CU3(cudaMemcpyAsync(ctx->params, params, (size_t)ctx->nM * nparam * sizeof(double),
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->stream));
    ctx->family = family;
    ctx->nparam = nparam;
    ctx->geom_valid = ctx->phi_valid = ctx->factor_valid = false;
    CU3(cudaStreamSynchronize(ctx->stream));
    return TSF_OK;
}

static cudaError_t put(tsf3_ctx* ctx, double* dst, const double* src, size_t n, int on_device, bool& flag) {
    flag = src != nullptr;
    if (!src) return cudaSuccess;
    return cudaMemcpyAsync(dst, src, n * sizeof(double), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                           ctx->stream);
}

tsf_status tsf3_set_sources(tsf3_ctx* ctx, const double* fu, const double* fw, const double* ud, const double* gu,
                            const double* gw, const double* fv, const double* gI, const double* gO,
                            const double* gN, int on_device) {
    if (!ctx) return TSF_E_ARG;
    if (!ctx->nM) return fail3(ctx, TSF_E_STATE, "set the meshes first");
    const size_t nM = ctx->nM, n1 = ctx->n1, N1 = ctx->N1;
    CU3(put(ctx, ctx->fu, fu, nM, on_device, ctx->has_fu));
    CU3(put(ctx, ctx->fw, fw, nM, on_device, ctx->has_fw));
    CU3(put(ctx, ctx->ud, ud, nM, on_device, ctx->has_ud));
    CU3(put(ctx, ctx->gu, gu, 4 * N1, on_device, ctx->has_gu));
    CU3(put(ctx, ctx->gw, gw, 4 * N1, on_device, ctx->has_gw));
    CU3(put(ctx, ctx->gI, gI, nM * n1, on_device, ctx->has_gI));
    CU3(put(ctx, ctx->gO, gO, nM * n1, on_device, ctx->has_gO));
    CU3(put(ctx, ctx->gN, gN, 2 * nM * n1, on_device, ctx->has_gN));
    ctx->has_fv = fv != nullptr;
    if (fv)
        CU3(cudaMemcpy2DAsync(ctx->fv, ctx->nmp * sizeof(double), fv, ctx->nm * sizeof(double),
                              ctx->nm * sizeof(double), nM, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                              ctx->stream));
    CU3(cudaStreamSynchronize(ctx->stream));
    return TSF_OK;
}

static MicroArgs micro3_args(tsf3_ctx* ctx, int t) {
    MicroArgs a{};
    a.n1 = ctx->n1;
    a.nm = ctx->nm;
    a.nmp = ctx->nmp;
    a.W = ctx->n1 + 2;
    a.nM = ctx->nM;
    a.S32 = ctx->S32;
    a.S64 = ctx->S64;
    a.chat = ctx->chat;
    a.chatlo = ctx->chatlo;
    a.dsc = ctx->dsc;
    a.c = ctx->c[t];
    a.v = ctx->x[t];
    a.u = ctx->zero;                                   // the macro values enter through c, not the edge term
    a.redge = ctx->er + (size_t)kEdgeRight * ctx->nM * ctx->n1;
    a.kappa = 0.0;
    a.tol = ctx->opt.cg_tol;
    a.inner_tol = ctx->opt.inner_tol;
    a.maxit = ctx->opt.cg_maxit;
    a.max_sweeps = ctx->opt.max_sweeps;
    a.rho = ctx->rho;
    a.inst_iters = ctx->iters;
    a.ctl = ctx->ctl;
    a.res = ctx->res[t];
    a.u_used = ctx->uu[t];
    a.bnorm = ctx->bnorm[t];
    return a;
}

static cudaError_t enqueue_setup(tsf3_ctx* ctx, int nsolve) {
    Setup3Args a{};
    a.n1 = ctx->n1;
    a.nm = ctx->nm;
    a.nmp = ctx->nmp;
    a.nM = ctx->nM;
    a.nsolve = nsolve;
    a.k1 = ctx->kap[0];
    a.k3 = ctx->kap[2];
    a.M64 = ctx->M64;
    a.eRd = ctx->eRd;
    a.eRu = ctx->eRu;
    a.er = ctx->er;
    a.fv = ctx->has_fv ? ctx->fv : nullptr;
    a.gI = ctx->has_gI ? ctx->gI : nullptr;
    a.gO = ctx->has_gO ? ctx->gO : nullptr;
    a.gN = ctx->has_gN ? ctx->gN : nullptr;
    for (int t = 0; t < 3; ++t) {
        a.c[t] = ctx->c[t];
        a.x[t] = ctx->x[t];
        a.res[t] = ctx->res[t];
        a.uu[t] = ctx->uu[t];
        a.bnorm[t] = ctx->bnorm[t];
    }
    a.G = ctx->G;
    k3_setup<<<ctx->nM, 256, 0, ctx->stream>>>(a);
    return cudaGetLastError();
}

static tsf_status build_geometry(tsf3_ctx* ctx) {
    CU3(launch_expand_params(ctx->family, ctx->nparam, ctx->params, ctx->prm5, ctx->map32, ctx->nM, ctx->stream));
    CU3(cudaMemsetAsync(&ctx->ctl->geom_error, 0, sizeof(int), ctx->stream));
    Geom3Args g{};
    g.Nm = ctx->Nm;
    g.n1 = ctx->n1;
    g.nm = ctx->nm;
    g.nmp = ctx->nmp;
    g.nM = ctx->nM;
    g.prm5 = ctx->prm5;
    g.D11 = ctx->D[0];
    g.D12 = ctx->D[1];
    g.D22 = ctx->D[2];
    g.k2 = ctx->kap[1];
    g.k4 = ctx->kap[3];
    g.M64 = ctx->M64;
    g.S64 = ctx->S64;
    g.S32 = ctx->S32;
    g.S32lo = nullptr;
    g.lm = ctx->lm;
    g.eRd = ctx->eRd;
    g.eRu = ctx->eRu;
    g.er = ctx->er;
    g.ctl = ctx->ctl;
    g.affine = ctx->family == TSF_FAMILY_IDENTITY || ctx->family == TSF_FAMILY_AFFINE;
    dim3 grid(ctx->nM, (ctx->nmp + 127) / 128);
    k3_geometry<<<grid, 128, 0, ctx->stream>>>(g);
    CU3(cudaGetLastError());
    int bad = 0;
    CU3(cudaMemcpyAsync(&bad, &ctx->ctl->geom_error, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CU3(cudaStreamSynchronize(ctx->stream));
    if (bad) return fail3(ctx, TSF_E_BAD_JACOBIAN, "det F <= 0 at a quadrature point of some micro cell");
    // operator data of the column-strip micro solves (the residual array of the
    // third right-hand side is free here: every solve starts from k3_setup)
    StripSetupArgs ss{};
    ss.n1 = ctx->n1;
    ss.nm = ctx->nm;
    ss.nmp = ctx->nmp;
    ss.nM = ctx->nM;
    ss.S64 = ctx->S64;
    ss.rs = ctx->res[2];
    ss.chat = ctx->chat;
    ss.chatlo = ctx->chatlo;
    ss.dsc = ctx->dsc;
    CU3(launch_strip_setup(ss, ctx->stream));
    ctx->geom_valid = true;
    ctx->phi_valid = false;
    return TSF_OK;
}

// Micro-solve variant: fixed by the options, or the fastest of the variants
// that fit, timed on the phi_I solve of the actual problem.
static size_t band_bytes(const tsf3_ctx* ctx) {
    return (size_t)ctx->nM * ctx->nm * (ctx->n1 + 2) * sizeof(float) + 3 * (size_t)ctx->nM * ctx->nmp * sizeof(float);
}

static tsf_status choose_tiling(tsf3_ctx* ctx) {
    const int prec = ctx->opt.precision;
    if (ctx->opt.tiling == kTilingDirect) {
        if (prec != TSF_MIXED)
            return fail3(ctx, TSF_E_ARG, "the direct micro solve (tiling %d) is a mixed-precision method", kTilingDirect);
        ctx->tiling = kTilingDirect;
        return TSF_OK;
    }
    if (ctx->opt.tiling < 0 && prec == TSF_MIXED) {
        size_t free_b = 0, total_b = 0;
        CU3(cudaMemGetInfo(&free_b, &total_b));
        if (band_bytes(ctx) <= free_b / 2) {
            ctx->tiling = kTilingDirect;
            return TSF_OK;
        }
    }
    if (ctx->opt.tiling >= 0) {
        if (!tiling_fits(ctx->opt.tiling, prec, ctx->n1, ctx->smem_optin))
            return fail3(ctx, TSF_E_ARG, "tiling %d does not fit this micro mesh / precision", ctx->opt.tiling);
        ctx->tiling = ctx->opt.tiling;
        return TSF_OK;
    }
    DevCtl saved;
    CU3(cudaMemcpyAsync(&saved, ctx->ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, ctx->stream));
    float best = 1e30f;
    int best_t = -1;
    for (int t = 0; t < kNumTilings; ++t) {
        if (!tiling_fits(t, prec, ctx->n1, ctx->smem_optin)) continue;
        float ms = 0.f;
        for (int rep = 0; rep < 2; ++rep) {
            CU3(enqueue_setup(ctx, 3));
            CU3(cudaEventRecord(ctx->ev[0], ctx->stream));
            CU3(launch_micro_solve(micro3_args(ctx, 1), prec, t, ctx->stream));
            CU3(cudaEventRecord(ctx->ev[1], ctx->stream));
            CU3(cudaEventSynchronize(ctx->ev[1]));
            CU3(cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[1]));
        }
        if (ms < best) {
            best = ms;
            best_t = t;
        }
    }
    CU3(cudaMemcpyAsync(ctx->ctl, &saved, sizeof(DevCtl), cudaMemcpyHostToDevice, ctx->stream));
    CU3(cudaStreamSynchronize(ctx->stream));
    if (best_t < 0) return fail3(ctx, TSF_E_ARG, "no micro-solve variant fits this mesh in this precision");
    ctx->tiling = best_t;
    return TSF_OK;
}

// FP32 band factor of every S_i (once per geometry and physics), then
// refinement sweeps on the nsolve right-hand sides set up by k3_setup:
// x += L^-T L^-1 r, r = c - S x (FP64), until every problem meets the tolerance.
static tsf_status direct_solves(tsf3_ctx* ctx, int nsolve) {
    ctx->stats.factor_ms = 0.0;
    ctx->stats.band_solve_ms = 0.0;
    ctx->stats.band_launches = 0;
    ctx->stats.band_rhs = nsolve;
    if (!ctx->factor_valid) {
        // allocated on first use; whatever a failed attempt left out is allocated next time
        if (!ctx->Lband) CU3(dalloc(ctx, &ctx->Lband, (size_t)ctx->nM * ctx->nm * (ctx->n1 + 2)));
        for (int t = 0; t < 3; ++t)
            if (!ctx->yband[t]) CU3(dalloc(ctx, &ctx->yband[t], (size_t)ctx->nM * ctx->nmp));
        CU3(cudaMemsetAsync(ctx->flag, 0, sizeof(int), ctx->stream));
        BandArgs f{};
        f.n1 = ctx->n1;
        f.nm = ctx->nm;
        f.nmp = ctx->nmp;
        f.nM = ctx->nM;
        f.S32 = ctx->S32;
        f.L = ctx->Lband;
        f.flag = ctx->flag;
        CU3(cudaEventRecord(ctx->bev[0], ctx->stream));
        CU3(launch_band_factor(f, ctx->stream));
        CU3(cudaEventRecord(ctx->bev[1], ctx->stream));
        int bad = 0;
        CU3(cudaMemcpyAsync(&bad, ctx->flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
        CU3(cudaStreamSynchronize(ctx->stream));
        float fm = 0.f;
        CU3(cudaEventElapsedTime(&fm, ctx->bev[0], ctx->bev[1]));
        ctx->stats.factor_ms = fm;
        if (bad) return fail3(ctx, TSF_E_BREAKDOWN, "non-positive pivot in the FP32 band factor of a micro operator");
        ctx->factor_valid = true;
    }
    BandSolveArgs b{};
    b.n1 = ctx->n1;
    b.nm = ctx->nm;
    b.nmp = ctx->nmp;
    b.nM = ctx->nM;
    b.L = ctx->Lband;
    BandResidualArgs r{};
    r.n1 = ctx->n1;
    r.nm = ctx->nm;
    r.nmp = ctx->nmp;
    r.nM = ctx->nM;
    r.nrhs = nsolve;
    r.tol = ctx->opt.cg_tol;
    r.S64 = ctx->S64;
    r.open_count = ctx->open_count;
    r.ctl = ctx->ctl;
    for (int t = 0; t < 3; ++t) {
        b.r[t] = ctx->res[t];
        b.x[t] = ctx->x[t];
        b.y[t] = ctx->yband[t];
        b.done[t] = ctx->done[t];
        r.c[t] = ctx->c[t];
        r.x[t] = ctx->x[t];
        r.r[t] = ctx->res[t];
        r.bnorm[t] = ctx->bnorm[t];
        r.done[t] = ctx->done[t];
    }
    for (int t = 0; t < nsolve; ++t) CU3(cudaMemsetAsync(ctx->done[t], 0, ctx->nM * sizeof(int), ctx->stream));
    const int max_sweeps = std::max(ctx->opt.max_sweeps, 30);
    int open = 1;
    for (int sweep = 0; sweep < max_sweeps && open; ++sweep) {
        CU3(cudaEventRecord(ctx->bev[0], ctx->stream));
        CU3(launch_band_solve(b, nsolve, ctx->stream));
        CU3(cudaEventRecord(ctx->bev[1], ctx->stream));
        CU3(cudaMemsetAsync(ctx->open_count, 0, sizeof(int), ctx->stream));
        CU3(launch_band_residual(r, ctx->stream));
        CU3(cudaMemcpyAsync(&open, ctx->open_count, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
        CU3(cudaStreamSynchronize(ctx->stream));
        float sm = 0.f;
        CU3(cudaEventElapsedTime(&sm, ctx->bev[0], ctx->bev[1]));
        ctx->stats.band_solve_ms += sm;
        ctx->stats.band_launches += 1;
    }
    const unsigned long long solved = (unsigned long long)nsolve * ctx->nM;
    DevCtl* c = ctx->ctl;
    // count the solved problems like the iterative kernels do
    unsigned long long ms = 0;
    CU3(cudaMemcpyAsync(&ms, &c->micro_solves, sizeof ms, cudaMemcpyDeviceToHost, ctx->stream));
    CU3(cudaStreamSynchronize(ctx->stream));
    ms += solved;
    CU3(cudaMemcpyAsync(&c->micro_solves, &ms, sizeof ms, cudaMemcpyHostToDevice, ctx->stream));
    if (open) {
        const int st = (int)TSF_E_NOT_CONVERGED;
        CU3(cudaMemcpyAsync(&c->status, &st, sizeof st, cudaMemcpyHostToDevice, ctx->stream));
    }
    return TSF_OK;
}

// The coupled macro solve as one cooperative grid: one node per thread, at
// most as many blocks as can be resident at once.
static cudaError_t launch_macro3(tsf3_ctx* ctx, Macro3Args& ma) {
    int per_sm = 0, sms = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k3_macro, kMacro3Threads, 0);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int want = (ctx->nM + kMacro3Threads - 1) / kMacro3Threads;
    const int blocks = std::max(1, std::min(want, per_sm * sms));
    double* part = ctx->mpart;
    void* args[] = {&ma, &part};
    return cudaLaunchCooperativeKernel((void*)k3_macro, dim3(blocks), dim3(kMacro3Threads), args, 0, ctx->stream);
}

tsf_status tsf3_solve(tsf3_ctx* ctx) {
    if (!ctx) return TSF_E_ARG;
    if (!ctx->nM) return fail3(ctx, TSF_E_STATE, "set the meshes first");
    tsf_status st;
    if (!ctx->geom_valid && (st = build_geometry(ctx))) return st;
    if (ctx->tiling < 0 && (st = choose_tiling(ctx))) return st;
    DevCtl before;
    CU3(cudaMemcpyAsync(&before, ctx->ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, ctx->stream));
    CU3(cudaStreamSynchronize(ctx->stream));
    CU3(cudaMemsetAsync(&ctx->ctl->status, 0, sizeof(int), ctx->stream));
    const int prec = ctx->opt.precision;
    const int nsolve = ctx->phi_valid ? 1 : 3;
    CU3(cudaEventRecord(ctx->ev[0], ctx->stream));
    CU3(enqueue_setup(ctx, nsolve));
    if (ctx->tiling == kTilingDirect) {
        if ((st = direct_solves(ctx, nsolve))) return st;
    } else {
        for (int t = 0; t < nsolve; ++t) CU3(launch_micro_solve(micro3_args(ctx, t), prec, ctx->tiling, ctx->stream));
    }
    CU3(cudaEventRecord(ctx->ev[1], ctx->stream));
    Moments3Args mo{};
    mo.n1 = ctx->n1;
    mo.nm = ctx->nm;
    mo.nmp = ctx->nmp;
    mo.nM = ctx->nM;
    mo.NM = ctx->NM;
    mo.H = ctx->L / ctx->NM;
    mo.k1 = ctx->kap[0];
    mo.k2 = ctx->kap[1];
    mo.k3 = ctx->kap[2];
    mo.k4 = ctx->kap[3];
    mo.er = ctx->er;
    mo.lm = ctx->lm;
    mo.phiI = ctx->x[1];
    mo.phiO = ctx->x[2];
    mo.v0 = ctx->x[0];
    mo.G = ctx->G;
    mo.coef = ctx->coef;
    mo.vol = ctx->vol;
    k3_moments<<<(ctx->nM + 3) / 4, 128, 0, ctx->stream>>>(mo);
    CU3(cudaGetLastError());
    Macro3Args ma{};
    ma.NM = ctx->NM;
    ma.N1 = ctx->N1;
    ma.nM = ctx->nM;
    ma.dir_mask = ctx->dir_mask;
    ma.H = ctx->L / ctx->NM;
    ma.Dw = ctx->Dw;
    ma.su = ctx->kap[0] / ctx->kap[1];
    ma.sw = ctx->kap[2] / ctx->kap[3];
    ma.coef = ctx->coef;
    ma.fu = ctx->has_fu ? ctx->fu : nullptr;
    ma.fw = ctx->has_fw ? ctx->fw : nullptr;
    ma.ud = ctx->has_ud ? ctx->ud : nullptr;
    ma.gu = ctx->has_gu ? ctx->gu : nullptr;
    ma.gw = ctx->has_gw ? ctx->gw : nullptr;
    ma.u = ctx->u;
    ma.w = ctx->w;
    ma.x = ctx->mx;
    ma.r = ctx->mr;
    ma.z = ctx->mz;
    ma.pv = ctx->mp;
    ma.qv = ctx->mq;
    ma.pinv = ctx->pinv;
    ma.tol = ctx->opt.macro_tol;
    ma.maxit = std::max(ctx->opt.macro_maxit, 50 * ctx->N1);
    ma.ctl = ctx->ctl;
    CU3(launch_macro3(ctx, ma));
    CU3(cudaEventRecord(ctx->ev[2], ctx->stream));
    const size_t total = (size_t)ctx->nM * ctx->nmp;
    k3_commit<<<(unsigned)std::min<size_t>((total + 255) / 256, 152 * 16), 256, 0, ctx->stream>>>(
        ctx->nmp, total, ctx->x[0], ctx->x[1], ctx->x[2], ctx->u, ctx->w, ctx->v);
    CU3(cudaGetLastError());
    CU3(launch_vbar(ctx->nm, ctx->nmp, ctx->nM, ctx->lm, ctx->vol, ctx->v, ctx->vbar, ctx->stream));
    CU3(cudaEventRecord(ctx->ev[3], ctx->stream));
    DevCtl after;
    CU3(cudaMemcpyAsync(&after, ctx->ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, ctx->stream));
    CU3(cudaStreamSynchronize(ctx->stream));
    float t01 = 0.f, t12 = 0.f, t03 = 0.f;
    CU3(cudaEventElapsedTime(&t01, ctx->ev[0], ctx->ev[1]));
    CU3(cudaEventElapsedTime(&t12, ctx->ev[1], ctx->ev[2]));
    CU3(cudaEventElapsedTime(&t03, ctx->ev[0], ctx->ev[3]));
    tsf3_stats& s = ctx->stats;
    s.inner_iters += (int64_t)(after.inner_iters - before.inner_iters);
    s.dof_cg_iters += (int64_t)(after.inner_iters - before.inner_iters) * ctx->nm;
    s.refine_sweeps += (int64_t)(after.sweeps - before.sweeps);
    s.micro_solves += (int64_t)(after.micro_solves - before.micro_solves);
    s.macro_iters += (int64_t)(after.macro_iters - before.macro_iters);
    s.status = after.status;
    s.tiling = ctx->tiling;
    s.micro_ms = t01;
    s.macro_ms = t12;
    s.total_ms = t03;
    ctx->solved = true;
    if (after.status) {
        ctx->phi_valid = false;
        return fail3(ctx, (tsf_status)after.status, "device status %d (micro or macro solve)", after.status);
    }
    ctx->phi_valid = true;
    return TSF_OK;
}

tsf_status tsf3_get_fields(tsf3_ctx* ctx, double* u, double* w, double* v, double* vbar, int on_device) {
    if (!ctx) return TSF_E_ARG;
    if (!ctx->solved) return fail3(ctx, TSF_E_STATE, "no solution yet");
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    const size_t nM = ctx->nM;
    if (u) CU3(cudaMemcpyAsync(u, ctx->u, nM * sizeof(double), k, ctx->stream));
    if (w) CU3(cudaMemcpyAsync(w, ctx->w, nM * sizeof(double), k, ctx->stream));
    if (vbar) CU3(cudaMemcpyAsync(vbar, ctx->vbar, nM * sizeof(double), k, ctx->stream));
    if (v)
        CU3(cudaMemcpy2DAsync(v, ctx->nm * sizeof(double), ctx->v, ctx->nmp * sizeof(double), ctx->nm * sizeof(double),
                              nM, k, ctx->stream));
    if (!on_device) CU3(cudaStreamSynchronize(ctx->stream));
    return TSF_OK;
}

tsf_status tsf3_get_pushforward(tsf3_ctx* ctx, float scale, float* out, int on_device) {
    if (!ctx || !out) return TSF_E_ARG;
    if (!(scale > 0.0f) || !std::isfinite(scale)) return fail3(ctx, TSF_E_ARG, "scale must be positive");
    if (!ctx->solved) return fail3(ctx, TSF_E_STATE, "no solution yet");
    const size_t n = (size_t)ctx->nM * ctx->nm * 3;
    float* dst = out;
    if (!on_device) {
        cudaError_t e = cudaMalloc((void**)&dst, n * sizeof(float));
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail3(ctx, TSF_E_OOM, "cudaMalloc of %zu bytes for the push-forward failed", n * sizeof(float));
        }
    }
    cudaError_t e = launch_pushforward(ctx->Nm, ctx->n1, ctx->nm, ctx->nmp, ctx->NM, ctx->nM, ctx->map32, ctx->v,
                                       (float)ctx->x0, (float)(ctx->L / ctx->NM), scale, 1, dst, ctx->stream);
    if (e == cudaSuccess && !on_device)
        e = cudaMemcpyAsync(out, dst, n * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (!on_device) cudaFree(dst);
    if (e != cudaSuccess) return fail3(ctx, TSF_E_CUDA, "push-forward: %s", cudaGetErrorString(e));
    return TSF_OK;
}

tsf_status tsf3_get_stats(tsf3_ctx* ctx, tsf3_stats* out) {
    if (!ctx || !out) return TSF_E_ARG;
    *out = ctx->stats;
    return TSF_OK;
}

}  // extern "C"
