// tsf_macro.cu -- the macro solve that closes each coupling iteration, and the
// coupling-loop control.
//
// Macro problem (first line of Eq. (17) with a time derivative, the coupling
// integral lumped at the collocation nodes):
//     (M_H/dt + Du K_H + kappa L Gam) u = M_H (u^n/dt + fu) - L G + kappa L rho
// on a uniform NM x NM Q1 mesh of [0,1]^2.  The operator is applied matrix-free
// from the node position alone: on a uniform square mesh every Q1 cell has the
// same element matrices, so an entry of M_H or K_H is (number of cells shared
// by the two nodes) x (the element entry), and L = diag(row sums of M_H) is
// H^2 (cells around the node)/4.
//
// Solver: flexible preconditioned CG in FP64 (Sec. 3.5: CG for every system).
// Preconditioner: exact fast diagonalisation of
//     P = M_H/dt + Du K_H + kappa gamma_bar L
// in FP32.  On a uniform mesh the 1D Q1 matrices M1, K1 and the lumped mass
// H W are all diagonalised by the same cosine basis cos(pi j k/NM) (Neumann;
// sine basis on the interior nodes for Dirichlet), so P^-1 is four dense
// n x n transforms and one diagonal scaling.  With |Gamma_i| equal for all
// nodes (bump families) P is the operator itself up to FP32 rounding and CG
// needs two or three iterations.  Meshes too large for the shared-memory
// transforms fall back to Jacobi.
//
// The macro problem is small (4225 unknowns for a 64x64 mesh), so it runs in
// one thread block, or in one thread-block cluster of kMacroCluster CTAs
// (k_macro_solve_cl).  Its cost is FP64 arithmetic at GB300's FP64 rate (about
// 30 FP64 operations per node and CG iteration; one SM does 1.65 a clock) and
// latency, not bandwidth.  The cluster variant spreads the node loops and the
// dense transforms over its CTAs, with cluster barriers in place of block
// barriers and the dot products gathered through distributed shared memory.
#include "tsf_internal.cuh"

#include <cooperative_groups.h>

#include <algorithm>

namespace tsf {

namespace cg = cooperative_groups;

__device__ __forceinline__ bool is_dir_node(int bc, int N, int p, int q) {
    return bc == 1 && (p == 0 || q == 0 || p == N || q == N);
}

// Entries of M_H/dt + Du K_H on the uniform mesh: with Me = H^2/36 [4 2 2 1]
// and Ke = 1/6 [4 -1 -1 -2] (self, edge neighbour, edge neighbour, diagonal
// neighbour of a cell), a node shared by cx x cy cells gets
//   cx cy A0 on the diagonal, cy A1 to E/W, cx A1 to N/S, A2 to diagonals,
// plus kappa |Gam_k| m_k with the lumped mass m_k = cx cy H^2 / 4.
struct MacroCoef {
    double A0, A1, A2, km;
};

__device__ __forceinline__ MacroCoef macro_coef(const MacroArgs& a) {
    const double h36 = a.H * a.H / (36.0 * a.dt);
    return {4.0 * h36 + (4.0 / 6.0) * a.Du, 2.0 * h36 - a.Du / 6.0, h36 - a.Du / 3.0, 0.25 * a.kappa * a.H * a.H};
}

// (M_H/dt + Du K_H + kappa L Gam) x at node k = (p, q)
__device__ __forceinline__ double macro_apply(const MacroArgs& a, const MacroCoef& m, const double* x, int k, int p,
                                              int q) {
    const int N = a.NM, n1 = a.N1;
    const double cx = (p == 0 || p == N) ? 1.0 : 2.0, cy = (q == 0 || q == N) ? 1.0 : 2.0;
    const bool e = p < N, w = p > 0, nn = q < N, s = q > 0;
    const double ew = (e ? x[k + 1] : 0.0) + (w ? x[k - 1] : 0.0);
    const double ns = (nn ? x[k + n1] : 0.0) + (s ? x[k - n1] : 0.0);
    const double dg = ((e && nn) ? x[k + n1 + 1] : 0.0) + ((w && nn) ? x[k + n1 - 1] : 0.0) +
                      ((e && s) ? x[k - n1 + 1] : 0.0) + ((w && s) ? x[k - n1 - 1] : 0.0);
    const double diag = cx * cy * fma(m.km, a.gam[k], m.A0);
    return fma(diag, x[k], fma(m.A1, fma(cy, ew, cx * ns), m.A2 * dg));
}

__device__ __forceinline__ double macro_diag(const MacroArgs& a, const MacroCoef& m, int k, int p, int q) {
    const int N = a.NM;
    const double cx = (p == 0 || p == N) ? 1.0 : 2.0, cy = (q == 0 || q == N) ? 1.0 : 2.0;
    return cx * cy * fma(m.km, a.gam[k], m.A0);
}

// One 2x2 block (rows r0, r0 + 1; columns c0, c0 + 1) of in * V (right) or
// V * in (left); np x np row-major, np even, V symmetric.
__device__ __forceinline__ float4 mm_block(const float* __restrict__ in, const float* __restrict__ V, int np,
                                          bool left, int r0, int c0) {
    float a00 = 0.f, a01 = 0.f, a10 = 0.f, a11 = 0.f;
    if (!left) {
        const float* x0 = in + r0 * np;
        const float* x1 = x0 + np;
        for (int m = 0; m < np; ++m) {
            const float2 v = *reinterpret_cast<const float2*>(V + m * np + c0);
            const float u0 = x0[m], u1 = x1[m];
            a00 = fmaf(u0, v.x, a00);
            a01 = fmaf(u0, v.y, a01);
            a10 = fmaf(u1, v.x, a10);
            a11 = fmaf(u1, v.y, a11);
        }
    } else {
        const float* v0 = V + r0 * np;
        const float* v1 = v0 + np;
        for (int m = 0; m < np; ++m) {
            const float2 x = *reinterpret_cast<const float2*>(in + m * np + c0);
            const float w0 = v0[m], w1 = v1[m];
            a00 = fmaf(w0, x.x, a00);
            a01 = fmaf(w0, x.y, a01);
            a10 = fmaf(w1, x.x, a10);
            a11 = fmaf(w1, x.y, a11);
        }
    }
    return make_float4(a00, a01, a10, a11);
}

// out = in * V (right) or V * in (left), all 2x2 blocks, by the threads of one block
__device__ void mm_pass(const float* __restrict__ in, float* __restrict__ out, const float* __restrict__ V, int np,
                        bool left) {
    const int nb = np >> 1, nblk = nb * nb;
    for (int blk = threadIdx.x; blk < nblk; blk += blockDim.x) {
        const int r0 = (blk / nb) * 2, c0 = (blk % nb) * 2;
        const float4 t = mm_block(in, V, np, left, r0, c0);
        *reinterpret_cast<float2*>(out + r0 * np + c0) = make_float2(t.x, t.y);
        *reinterpret_cast<float2*>(out + (r0 + 1) * np + c0) = make_float2(t.z, t.w);
    }
}

struct DctView {
    int n, np, off;     // transform size, padded size, node offset (1 for Dirichlet interior)
    float *X0, *X1, *V, *lamM, *lamK, *Dn;
    float gterm;        // kappa * gamma_bar * H^2
};

// Who runs the macro solve: one thread block ...
// Sums for the macro solve.  Every thread holds NV partial sums (NV <= 2);
// the warp butterflies them, lane 0 of each warp puts the warp sums into buf
// (slots i 32 + warp), and after a block barrier warp 0 alone sums the warp
// sums: the FP64 adds of a sum no longer grow with the warps times the warps.
// The block total goes to slot 64 + i; the cluster variant gathers the G
// block totals there through distributed shared memory (warp 0 again) and
// leaves the cluster total in slot 80 + i.  Fixed order throughout, so every
// thread of every CTA gets the same bits.  buf: one of the 96-entry buffers,
// reused only after three more sums.
template <class T, int NV>
__device__ __forceinline__ void warp_sums_to_buf(T (&v)[NV], T* buf) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
    }
    if (lane == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) buf[i * 32 + warp] = v[i];
    }
}
template <class T, int NV>
__device__ __forceinline__ void warp0_block_total(T* buf) {  // (warp 0 only)
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        T s = lane < nw ? buf[i * 32 + lane] : T(0);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) buf[64 + i] = s;
    }
}

// Who runs the macro solve: one thread block ...
struct MacroBlock {
    __device__ int gtid() const { return threadIdx.x; }
    __device__ int gsize() const { return blockDim.x; }
    __device__ bool leader() const { return threadIdx.x == 0; }
    __device__ void sync() const { __syncthreads(); }
    template <class T, int NV>
    __device__ void allreduce(T (&v)[NV], T* buf) const {
        static_assert(NV <= 2, "slots 64.. of the 96-entry buffer hold the totals");
        warp_sums_to_buf<T, NV>(v, buf);
        __syncthreads();
        if (threadIdx.x < 32) warp0_block_total<T, NV>(buf);
        __syncthreads();
#pragma unroll
        for (int i = 0; i < NV; ++i) v[i] = buf[64 + i];
    }
};
// ... or the CTAs of one cluster: thread t = rank T + threadIdx.x takes the
// nodes t, t + G T, ... of every loop (the same nodes in every loop); the
// barrier is the cluster's (release / acquire at cluster scope, so global
// writes before it are seen by every CTA after it).
struct MacroCluster {
    int rank, G;
    __device__ int gtid() const { return rank * (int)blockDim.x + (int)threadIdx.x; }
    __device__ int gsize() const { return G * (int)blockDim.x; }
    __device__ bool leader() const { return rank == 0 && threadIdx.x == 0; }
    __device__ void sync() const { cg::this_cluster().sync(); }
    template <class T, int NV>
    __device__ void allreduce(T (&v)[NV], T* buf) const {
        static_assert(NV <= 2, "slots 64.. and 80.. of the 96-entry buffer hold the totals");
        warp_sums_to_buf<T, NV>(v, buf);
        __syncthreads();
        if (threadIdx.x < 32) warp0_block_total<T, NV>(buf);
        cg::cluster_group cl = cg::this_cluster();
        cl.sync();
        if (threadIdx.x < 32) {
            const int lane = threadIdx.x;
#pragma unroll
            for (int i = 0; i < NV; ++i) {
                T s = lane < G ? *cl.map_shared_rank(buf + 64 + i, lane) : T(0);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                if (lane == 0) buf[80 + i] = s;
            }
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < NV; ++i) v[i] = buf[80 + i];
    }
};

// The diagonal scaling of the transformed residual, X <- X / (Dn Dn lambda),
// elements e0, e0 + es, ...
__device__ __forceinline__ void dct_scale(const MacroArgs& a, const DctView& d, float* X, int e0, int es) {
    const int n = d.n, np = d.np;
    const float idt = (float)(1.0 / a.dt), Du = (float)a.Du;
    for (int e = e0; e < n * n; e += es) {
        const int l = e / n, k = e % n;
        const float lam = d.lamM[k] * d.lamM[l] * idt + Du * (d.lamK[k] * d.lamM[l] + d.lamM[k] * d.lamK[l]) +
                          d.gterm;
        X[l * np + k] *= 1.0f / (d.Dn[l] * d.Dn[k] * lam);
    }
}

// z = P^{-1} r (fast diagonalisation, FP32 transforms): V (V r V) V with the
// scaling in between, and the sums dots = (r^T z, r^T zo) (the second only
// with use_zo), whose reduction is the step's last barrier.  All threads of
// one block.
__device__ void dct_precond(const MacroArgs& a, const DctView& d, const double* r, double* z, const MacroBlock& tm,
                            bool use_zo, double (&dots)[2], double* buf) {
    const int n = d.n, np = d.np, n1 = a.N1;
    for (int e = threadIdx.x; e < np * np; e += blockDim.x) {
        const int rr = e / np, cc = e % np;
        float val = 0.f;
        if (rr < n && cc < n) val = (float)r[(cc + d.off) + n1 * (rr + d.off)];
        d.X0[e] = val;
    }
    __syncthreads();
    mm_pass(d.X0, d.X1, d.V, np, false);
    __syncthreads();
    mm_pass(d.X1, d.X0, d.V, np, true);
    __syncthreads();
    dct_scale(a, d, d.X0, threadIdx.x, blockDim.x);
    __syncthreads();
    mm_pass(d.X0, d.X1, d.V, np, false);
    __syncthreads();
    mm_pass(d.X1, d.X0, d.V, np, true);
    __syncthreads();
    double rz = 0.0, rzo = 0.0;
    for (int k = threadIdx.x; k < a.nM; k += blockDim.x) {
        const int p = k % n1, q = k / n1;
        const int cc = p - d.off, rr = q - d.off;
        const double zk = (cc >= 0 && rr >= 0 && cc < n && rr < n) ? (double)d.X0[rr * np + cc] : 0.0;
        z[k] = zk;
        rz = fma(r[k], zk, rz);
        if (use_zo) rzo = fma(r[k], a.zo[k], rzo);
    }
    dots[0] = rz;
    dots[1] = rzo;
    tm.allreduce(dots, buf);
}

// The same by the CTAs of a cluster.  Every CTA keeps whole copies of the two
// transform buffers in its shared memory; CTA g computes the 2x2 blocks of
// block rows [g nb / G, (g + 1) nb / G) of each product from its own copies
// and stores them into every CTA's copy through distributed shared memory
// (the last product into its own copy only: each CTA then writes z for the
// rows it computed).  One cluster barrier after each broadcast product.
__device__ void mm_pass_cl(const float* __restrict__ in, float* __restrict__ out, const float* __restrict__ V, int np,
                           bool left, const MacroCluster& tm, bool broadcast) {
    cg::cluster_group cl = cg::this_cluster();
    const int nb = np >> 1;
    const int b0 = tm.rank * nb / tm.G, b1 = (tm.rank + 1) * nb / tm.G;
    const int nblk = (b1 - b0) * nb;
    for (int blk = threadIdx.x; blk < nblk; blk += blockDim.x) {
        const int r0 = (b0 + blk / nb) * 2, c0 = (blk % nb) * 2;
        const float4 t = mm_block(in, V, np, left, r0, c0);
        const float2 lo = make_float2(t.x, t.y), hi = make_float2(t.z, t.w);
        if (broadcast) {
            for (int g = 0; g < tm.G; ++g) {
                float* o = cl.map_shared_rank(out, g);
                *reinterpret_cast<float2*>(o + r0 * np + c0) = lo;
                *reinterpret_cast<float2*>(o + (r0 + 1) * np + c0) = hi;
            }
        } else {
            *reinterpret_cast<float2*>(out + r0 * np + c0) = lo;
            *reinterpret_cast<float2*>(out + (r0 + 1) * np + c0) = hi;
        }
    }
}

__device__ void dct_precond(const MacroArgs& a, const DctView& d, const double* r, double* z,
                            const MacroCluster& tm, bool use_zo, double (&dots)[2], double* buf) {
    const int n = d.n, np = d.np, n1 = a.N1;
    // every CTA reads the whole residual (global, complete after the last barrier)
    for (int e = threadIdx.x; e < np * np; e += blockDim.x) {
        const int rr = e / np, cc = e % np;
        float val = 0.f;
        if (rr < n && cc < n) val = (float)r[(cc + d.off) + n1 * (rr + d.off)];
        d.X0[e] = val;
    }
    __syncthreads();
    mm_pass_cl(d.X0, d.X1, d.V, np, false, tm, true);
    tm.sync();
    mm_pass_cl(d.X1, d.X0, d.V, np, true, tm, true);
    tm.sync();
    dct_scale(a, d, d.X0, threadIdx.x, blockDim.x);  // (every CTA its whole copy)
    __syncthreads();
    mm_pass_cl(d.X0, d.X1, d.V, np, false, tm, true);
    tm.sync();
    mm_pass_cl(d.X1, d.X0, d.V, np, true, tm, false);
    __syncthreads();
    const int nb = np >> 1;
    const int rlo = 2 * (tm.rank * nb / tm.G), rhi = 2 * ((tm.rank + 1) * nb / tm.G);
    double rz = 0.0, rzo = 0.0;
    for (int e = threadIdx.x; e < (rhi - rlo) * np; e += blockDim.x) {
        const int rr = rlo + e / np, cc = e % np;
        if (rr < n && cc < n) {
            const int k = (cc + d.off) + n1 * (rr + d.off);
            const double zk = (double)d.X0[rr * np + cc];
            z[k] = zk;
            rz = fma(r[k], zk, rz);
            if (use_zo) rzo = fma(r[k], a.zo[k], rzo);
        }
    }
    if (d.off) {  // Dirichlet: the boundary nodes outside the transform get z = 0
        for (int k = tm.gtid(); k < a.nM; k += tm.gsize()) {
            const int p = k % n1, q = k / n1;
            if (p < d.off || q < d.off || p >= n + d.off || q >= n + d.off) z[k] = 0.0;
        }
    }
    dots[0] = rz;
    dots[1] = rzo;
    tm.allreduce(dots, buf);  // (its cluster barrier publishes z)
}

// one block of this many threads runs the macro solve (launch and launch
// bounds); each CTA of the cluster variant has kMacroClThreads (fewer threads
// a CTA: fewer FP64 adds in every sum, and the node loops still fill them)
constexpr int kMacroThreads = 512;
constexpr int kMacroClThreads = 256;

// reductions, basis V, eigenvalues and scaling, then the two transform
// buffers (every CTA of the cluster variant holds all of them)
size_t macro_smem_bytes(int N1, int bc, int use_dct) {
    size_t b = 4 * 96 * sizeof(double);
    if (use_dct) {
        const int n = bc ? N1 - 2 : N1;
        const int np = (n + 1) & ~1;
        b += (3 * (size_t)np * np + 3 * (size_t)np) * sizeof(float);
    }
    return b;
}
static size_t macro_cl_smem_bytes(int N1, int bc, int use_dct) { return macro_smem_bytes(N1, bc, use_dct); }

// The solve, by one block or one cluster (TEAM).  X0, X1: the transform
// buffers (shared memory of the block, or global scratch the cluster shares).
template <class TEAM>
__device__ void macro_solve_body(const MacroArgs& a, const TEAM& tm, unsigned char* smem, float* X0, float* X1) {
    double* red = reinterpret_cast<double*>(smem);  // 4 x 96
    const int tid = tm.gtid(), T = tm.gsize();
    const int nM = a.nM, n1 = a.N1, N = a.NM;
    int rb = 0;
    auto nextbuf = [&]() { double* b = red + 96 * rb; rb = (rb + 1) & 3; return b; };
    const int my_iter = a.ctl->coupling_iter;
    const MacroCoef mc = macro_coef(a);

    DctView d{};
    if (a.use_dct) {
        d.n = a.bc ? N - 1 : N + 1;
        d.off = a.bc ? 1 : 0;
        d.np = (d.n + 1) & ~1;
        float* f = reinterpret_cast<float*>(red + 4 * 96);
        d.X0 = X0;
        d.X1 = X1;
        d.V = f;
        d.lamM = f + d.np * d.np;
        d.lamK = d.lamM + d.np;
        d.Dn = d.lamK + d.np;
        // basis: cos (Neumann) or sin (Dirichlet interior) of pi (a+off)(b+off)/N,
        // in every CTA's own shared memory
        for (int e = threadIdx.x; e < d.np * d.np; e += blockDim.x) {
            const int r = e / d.np, c = e % d.np;
            float v = 0.f;
            if (r < d.n && c < d.n) {
                const int m = ((r + d.off) * (c + d.off)) % (2 * N);
                v = a.bc ? sinpif((float)m / (float)N) : cospif((float)m / (float)N);
            }
            d.V[e] = v;
        }
        const float H = (float)a.H;
        for (int k = threadIdx.x; k < d.n; k += blockDim.x) {
            const float ck = cospif((float)(k + d.off) / (float)N);
            d.lamM[k] = (H / 6.f) * (4.f + 2.f * ck);
            d.lamK[k] = (2.f / H) * (1.f - ck);
            // sum_j w_j basis_j^2: N/2, doubled for the constant and alternating cosines
            d.Dn[k] = 0.5f * (float)N * ((!a.bc && (k == 0 || k == N)) ? 2.f : 1.f);
        }
    }
    // gamma_bar: mean |Gamma| over unknown (non-Dirichlet) nodes (FP32: it
    // only enters the preconditioner)
    {
        float sg = 0.f, cnt = 0.f;
        for (int k = tid; k < nM; k += T) {
            if (!is_dir_node(a.bc, N, k % n1, k / n1)) {
                sg += (float)a.gam[k];
                cnt += 1.f;
            }
        }
        float t[2] = {sg, cnt};
        tm.allreduce(t, reinterpret_cast<float*>(nextbuf()));
        d.gterm = (float)a.kappa * (t[1] > 0.f ? t[0] / t[1] : 1.f) * (float)(a.H * a.H);
    }
    // right-hand side and initial guess; b kept in q until the residual is formed
    for (int k = tid; k < nM; k += T) {
        const int p = k % n1, q = k / n1;
        const double H2 = a.H * a.H;
        const double cx = (p == 0 || p == N) ? 1.0 : 2.0, cy = (q == 0 || q == N) ? 1.0 : 2.0;
        const double b = is_dir_node(a.bc, N, p, q) ? a.uk[k] : a.cH[k] + a.kappa * (cx * cy * 0.25 * H2) * a.rho[k];
        a.q[k] = b;
        a.x[k] = a.uk[k];
    }
    tm.sync();
    // stopping norms in FP64 like everything else here: FP32 sums of squares
    // would underflow for data scaled below about 1e-19 and stop the solve
    // before it starts
    double bn2 = 0.0, rr = 0.0;
    for (int k = tid; k < nM; k += T) {
        const int p = k % n1, q = k / n1;
        const double b = a.q[k];
        const double res = is_dir_node(a.bc, N, p, q) ? 0.0 : b - macro_apply(a, mc, a.x, k, p, q);
        a.r[k] = res;
        bn2 = fma(b, b, bn2);
        rr = fma(res, res, rr);
    }
    {
        double t[2] = {bn2, rr};
        tm.allreduce(t, nextbuf());
        bn2 = t[0];
        rr = t[1];
    }
    const double stop2 = a.tol * a.tol * bn2;
    int it = 0;
    bool fail = false;
    if (rr > stop2 && bn2 > 0.0) {
        // z = P r and the sums r^T z, r^T zo (zo: the z of the previous
        // iteration) in one phase that ends with the sums' barrier
        auto precond = [&](bool use_zo, double (&dots)[2]) {
            if (a.use_dct) {
                dct_precond(a, d, a.r, a.z, tm, use_zo, dots, nextbuf());
            } else {
                double rz = 0.0, rzo = 0.0;
                for (int k = tid; k < nM; k += T) {
                    const double zk = a.r[k] / macro_diag(a, mc, k, k % n1, k / n1);
                    a.z[k] = zk;
                    rz = fma(a.r[k], zk, rz);
                    if (use_zo) rzo = fma(a.r[k], a.zo[k], rzo);
                }
                dots[0] = rz;
                dots[1] = rzo;
                tm.allreduce(dots, nextbuf());
            }
        };
        double dots[2];
        precond(false, dots);
        double rz = dots[0], beta = 0.0;
        while (it < a.maxit) {
            // p = z + beta p and q = A p = A z + beta q in one pass: A z needs
            // only z, complete after the last sums' barrier, so no barrier
            // separates the direction update from the operator
            double pq = 0.0;
            for (int k = tid; k < nM; k += T) {
                const int p = k % n1, q = k / n1;
                const double az = is_dir_node(a.bc, N, p, q) ? 0.0 : macro_apply(a, mc, a.z, k, p, q);
                // (the first pass reads no p, q: they hold whatever the last solve left)
                const double pk = it ? fma(beta, a.p[k], a.z[k]) : a.z[k];
                const double qk = it ? fma(beta, a.q[k], az) : az;
                a.p[k] = pk;
                a.q[k] = qk;
                pq = fma(pk, qk, pq);
            }
            {
                double t[1] = {pq};
                tm.allreduce(t, nextbuf());
                pq = t[0];
            }
            ++it;
            if (!(pq > 0.0)) {
                fail = true;
                break;
            }
            const double alpha = rz / pq;
            rr = 0.0;
            for (int k = tid; k < nM; k += T) {
                a.x[k] = fma(alpha, a.p[k], a.x[k]);
                const double rn = fma(-alpha, a.q[k], a.r[k]);
                a.r[k] = rn;
                a.zo[k] = a.z[k];
                rr = fma(rn, rn, rr);
            }
            {
                double t[1] = {rr};
                tm.allreduce(t, nextbuf());
                rr = t[0];
            }
            if (!(rr == rr)) {
                fail = true;
                break;
            }
            if (rr <= stop2) break;
            precond(true, dots);
            // flexible (Polak-Ribiere) beta: robust to the FP32 preconditioner
            beta = (dots[0] - dots[1]) / rz;
            rz = dots[0];
        }
        if (!fail && rr > stop2) fail = true;
    }

    // coupling control: relative change of the macro iterate (FP64 sums, for
    // the same reason)
    double dn2 = 0.0, un2 = 0.0;
    for (int k = tid; k < nM; k += T) {
        const double xn = a.x[k];
        const double dd = xn - a.uk[k];
        dn2 = fma(dd, dd, dn2);
        un2 = fma(xn, xn, un2);
    }
    {
        double t[2] = {dn2, un2};
        tm.allreduce(t, nextbuf());
        dn2 = t[0];
        un2 = t[1];
    }
    const double change = un2 > 0.0 ? sqrt(dn2 / un2) : sqrt(dn2);
    const int iter = my_iter + 1;
    const bool converged = change <= a.coupling_tol;
    const bool last = converged || iter >= a.coupling_maxit || !(change == change);
    for (int k = tid; k < nM; k += T) {
        const double xn = a.x[k];
        a.uk[k] = xn;
        if (last) a.u[k] = xn;
    }
    if (tm.leader()) {
        DevCtl* c = a.ctl;
        c->macro_iters += (unsigned long long)it;
        c->coupling_iter = iter;
        c->change = change;
        if (fail) set_status(c, kNotConverged);
        if (!(change == change)) set_status(c, kNaN);
        if (last) {
            c->coupling_iters_last = iter;
            c->coupling_iters_total += iter;
            c->steps += 1;
            if (!converged) set_status(c, kNotConverged);
            c->cont = 0;
        } else {
            c->cont = 1;
        }
        if (a.set_cond) cudaGraphSetConditional(a.cond, last ? 0u : 1u);
    }
}

__global__ void __launch_bounds__(kMacroThreads, 1) k_macro_solve(MacroArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    // the transform buffers after the reduction buffers, the basis and the eigenvalues
    float* f = reinterpret_cast<float*>(smem + 4 * 96 * sizeof(double));
    const int np = a.use_dct ? ((a.bc ? a.NM - 1 : a.NM + 1) + 1) & ~1 : 0;
    float* X0 = f + np * np + 3 * np;
    macro_solve_body(a, MacroBlock{}, smem, X0, X0 + np * np);
}

__global__ void __launch_bounds__(kMacroClThreads, 1) k_macro_solve_cl(MacroArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    cg::cluster_group cl = cg::this_cluster();
    const MacroCluster tm{(int)cl.block_rank(), (int)cl.num_blocks()};
    float* f = reinterpret_cast<float*>(smem + 4 * 96 * sizeof(double));
    const int np = a.use_dct ? ((a.bc ? a.NM - 1 : a.NM + 1) + 1) & ~1 : 0;
    float* X0 = f + np * np + 3 * np;
    macro_solve_body(a, tm, smem, X0, X0 + np * np);
    cl.sync();  // no CTA leaves while another may still read or write its shared memory
}

// Whether a cluster of kMacroCluster CTAs of the macro solve fits the device
// (queried once per shared-memory size).
bool macro_cluster_ok(int N1, int bc, int use_dct) {
    static int cached_dev = -1;
    static size_t cached_sm = 0;
    static bool cached_ok = false;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    const size_t sm = macro_cl_smem_bytes(N1, bc, use_dct);
    if (dev == cached_dev && sm == cached_sm) return cached_ok;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(kMacroCluster);
    cfg.blockDim = dim3(kMacroClThreads);
    cfg.dynamicSmemBytes = sm;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = kMacroCluster;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    const bool ok = cudaOccupancyMaxActiveClusters(&n, k_macro_solve_cl, &cfg) == cudaSuccess && n > 0;
    cudaGetLastError();
    cached_dev = dev;
    cached_sm = sm;
    cached_ok = ok;
    return ok;
}

cudaError_t launch_macro_solve(const MacroArgs& a, cudaStream_t s, int priority, size_t reserve_smem) {
    if (a.ncta > 1) {
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3(a.ncta);
        cfg.blockDim = dim3(kMacroClThreads);
        cfg.dynamicSmemBytes = macro_cl_smem_bytes(a.N1, a.bc, a.use_dct);
        cfg.stream = s;
        cudaLaunchAttribute at[2];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = a.ncta;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        at[1].id = cudaLaunchAttributePriority;
        at[1].val.priority = priority;
        cfg.attrs = at;
        cfg.numAttrs = priority ? 2 : 1;
        return cudaLaunchKernelEx(&cfg, k_macro_solve_cl, a);
    }
    const size_t sm = std::max(macro_smem_bytes(a.N1, a.bc, a.use_dct), reserve_smem);
    if (priority == 0) {
        k_macro_solve<<<1, kMacroThreads, sm, s>>>(a);
        return cudaGetLastError();
    }
    // a scheduling priority for the block (kept by graph capture)
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(1);
    cfg.blockDim = dim3(kMacroThreads);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributePriority;
    at[0].val.priority = priority;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_macro_solve, a);
}

cudaError_t configure_macro_kernels(int smem_optin) {
    cudaError_t e = cudaFuncSetAttribute(k_macro_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_macro_solve_cl, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin);
    return e;
}

// cH = M_H (u^n/dt + fu) - L G ; initial macro iterate with the Dirichlet values;
// resets the per-step coupling counter.  One thread per macro node.
__global__ void k_macro_prologue(MacroPrologueArgs a) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k == 0) {
        a.ctl->coupling_iter = 0;
        a.ctl->cont = 1;
    }
    if (k >= a.nM) return;
    const int N = a.NM, n1 = a.N1;
    const int p = k % n1, q = k / n1;
    const double idt = 1.0 / a.dt;
    auto w = [&](int l) { return a.fu ? fma(a.u[l], idt, a.fu[l]) : a.u[l] * idt; };
    const double cx = (p == 0 || p == N) ? 1.0 : 2.0, cy = (q == 0 || q == N) ? 1.0 : 2.0;
    const bool e = p < N, wst = p > 0, nn = q < N, s = q > 0;
    const double ew = (e ? w(k + 1) : 0.0) + (wst ? w(k - 1) : 0.0);
    const double ns = (nn ? w(k + n1) : 0.0) + (s ? w(k - n1) : 0.0);
    const double dg = ((e && nn) ? w(k + n1 + 1) : 0.0) + ((wst && nn) ? w(k + n1 - 1) : 0.0) +
                      ((e && s) ? w(k - n1 + 1) : 0.0) + ((wst && s) ? w(k - n1 - 1) : 0.0);
    const double H2 = a.H * a.H;
    const double Mw = (H2 / 36.0) * (4.0 * cx * cy * w(k) + 2.0 * cy * ew + 2.0 * cx * ns + dg);
    const double m = cx * cy * 0.25 * H2;
    // G_k = int_Gamma g = r_k^T g_k (compensated sum over the Robin-edge nodes)
    double G = 0.0;
    if (a.g) {
        const double* r = a.redge + (size_t)k * a.n1m;
        const double* g = a.g + (size_t)k * a.n1m;
        double c = 0.0;
        for (int j = 0; j < a.n1m; ++j) {
            double sum, err;
            two_sum(G, r[j] * g[j], sum, err);
            G = sum;
            c += err + fma(r[j], g[j], -(r[j] * g[j]));
        }
        G += c;
    }
    a.G[k] = G;
    a.cH[k] = Mw - m * G;
    double uk = a.u[k];
    if (is_dir_node(a.bc, N, p, q) && a.ud) uk = a.ud[k];
    a.uk[k] = uk;
    if (a.rho_eff) {
        double rw;
        if (a.ring2) {
            // r^T w of the w the last column-strip solve pushed (ring slot
            // hist_step + 2 after k_elim_start), compensated FP64 over the
            // Robin-edge nodes of micro problem k
            const size_t slot = (size_t)((a.ctl->hist_step + 2) % 3) * a.nM * a.nmp + (size_t)k * a.nmp;
            const double* r = a.redge + (size_t)k * a.n1m;
            double c = 0.0;
            rw = 0.0;
            for (int q = 0; q < a.n1m; ++q) {
                const float2 wq = a.ring2[slot + (a.n1m - 1) + (size_t)a.n1m * q];
                const double x = (double)wq.x + (double)wq.y;
                double sum, err;
                two_sum(rw, r[q] * x, sum, err);
                rw = sum;
                c += err + fma(r[q], x, -(r[q] * x));
            }
            rw += c;
        } else {
            rw = a.rho_w[k];
        }
        a.rho_eff[k] = fma(a.u[k], a.gam_psi[k], rw);  // r^T (w + u psi)
    }
}

cudaError_t launch_macro_prologue(const MacroPrologueArgs& a, cudaStream_t s) {
    k_macro_prologue<<<(a.nM + 255) / 256, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace tsf
