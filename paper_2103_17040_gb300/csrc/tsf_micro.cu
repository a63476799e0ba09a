// tsf_micro.cu -- the batched micro solve (hot path) and its per-step
// prologue / epilogue kernels.
//
// Every micro problem i (one per macro node, Sec. 3.3) solves
//     S_i v_i = c_i + kappa u_i r_i,      S_i = M_i/dt + A_i + kappa R_i,
// with Jacobi-preconditioned CG (Sec. 3.5, last paragraph: CG for every
// system, the systems distributed over the processors).  One thread block
// owns one micro problem for the whole solve:
//   * the five stencil planes of S_i are staged once into shared memory on a
//     zero-haloed (n1+2)^2 grid, so the matrix-free Q1 apply needs no bounds
//     checks and touches HBM zero times per CG iteration;
//   * the CG vectors live in registers (K nodes per thread, node j of the
//     instance handled by thread j mod T), only the search direction goes
//     through shared memory for the 9-point stencil;
//   * dot products are warp-shuffle trees plus one cross-warp tree (fixed
//     order, so identical instances give bitwise identical results).
// Precision variants:
//   FP64  : CG in FP64 on the FP64 stencil until ||b - S v|| <= tol ||b||.
//   MIXED : FP64 iterative refinement around an FP32 CG on the FP32 stencil:
//           r = b - S64 v in FP64, FP32 solve of S32 d = r to inner_tol,
//           v += d, until the FP64 residual meets tol.
// The boundary-flux integral rho_i = r_i^T v_i that feeds the macro source is
// reduced in the epilogue of the same kernel with compensated (TwoSum) FP64
// sums.
#include "tsf_internal.cuh"

namespace tsf {

__device__ __forceinline__ float tfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double tfma(double a, double b, double c) { return fma(a, b, c); }

// y = S x at shared-memory grid index s (zero halo: no bounds checks).
template <typename TI>
__device__ __forceinline__ TI stencil_smem(const TI* __restrict__ cf, const TI* __restrict__ x, int s, int W,
                                           int W2) {
    const TI* C = cf;
    const TI* E = cf + W2;
    const TI* N = cf + 2 * W2;
    const TI* NE = cf + 3 * W2;
    const TI* NW = cf + 4 * W2;
    TI y = C[s] * x[s];
    y = tfma(E[s], x[s + 1], y);
    y = tfma(E[s - 1], x[s - 1], y);
    y = tfma(N[s], x[s + W], y);
    y = tfma(N[s - W], x[s - W], y);
    y = tfma(NE[s], x[s + W + 1], y);
    y = tfma(NE[s - W - 1], x[s - W - 1], y);
    y = tfma(NW[s], x[s + W - 1], y);
    y = tfma(NW[s - W + 1], x[s - W + 1], y);
    return y;
}

// y = S x for node j = (p, q) with planes and x in global memory (FP64).
__device__ __forceinline__ double stencil_global(const double* __restrict__ S, size_t pl, const double* x, int j,
                                                 int p, int q, int n1) {
    double y = S[j] * x[j];
    const bool e = p + 1 < n1, w = p > 0;
    if (e) y = fma(S[pl + j], x[j + 1], y);
    if (w) y = fma(S[pl + j - 1], x[j - 1], y);
    if (q + 1 < n1) {
        y = fma(S[2 * pl + j], x[j + n1], y);
        if (e) y = fma(S[3 * pl + j], x[j + n1 + 1], y);
        if (w) y = fma(S[4 * pl + j], x[j + n1 - 1], y);
    }
    if (q > 0) {
        y = fma(S[2 * pl + j - n1], x[j - n1], y);
        if (w) y = fma(S[3 * pl + j - n1 - 1], x[j - n1 - 1], y);
        if (e) y = fma(S[4 * pl + j - n1 + 1], x[j - n1 + 1], y);
    }
    return y;
}

// Jacobi-PCG on the shared-memory stencil.  On entry x holds the initial
// guess and r = rhs - S x (per node, registers), with ||r||^2 > stop2.
// Iterates until ||r||^2 <= stop2 or maxit iterations.  Returns the number
// of iterations; *flag receives kBreakdown / kNaN on failure.
template <typename TI, int K>
__device__ int pcg_smem(const TI* cf, TI* pp, int W, int W2, const int (&sidx)[K], const bool (&valid)[K],
                        const TI (&dinv)[K], TI (&x)[K], TI (&r)[K], TI stop2, int maxit, TI* redA, TI* redB,
                        int* flag) {
    TI z[K], p[K];
    TI rz = TI(0);
#pragma unroll
    for (int k = 0; k < K; ++k) {
        z[k] = dinv[k] * r[k];
        p[k] = z[k];
        rz = tfma(r[k], z[k], rz);
    }
    {
        TI t[1] = {rz};
        block_allreduce<TI, 1>(t, redB);
        rz = t[0];
    }
    int it = 0;
    while (it < maxit) {
#pragma unroll
        for (int k = 0; k < K; ++k)
            if (valid[k]) pp[sidx[k]] = p[k];
        __syncthreads();
        TI q[K];
        TI pq = TI(0);
#pragma unroll
        for (int k = 0; k < K; ++k) {
            q[k] = valid[k] ? stencil_smem<TI>(cf, pp, sidx[k], W, W2) : TI(0);
            pq = tfma(p[k], q[k], pq);
        }
        {
            TI t[1] = {pq};
            block_allreduce<TI, 1>(t, redA);
            pq = t[0];
        }
        ++it;
        if (!(pq > TI(0))) {
            *flag = (pq == pq) ? kBreakdown : kNaN;
            break;
        }
        const TI alpha = rz / pq;
        if (!isfinite(alpha)) {  // pq lost to underflow: end this solve like a breakdown
            *flag = kBreakdown;
            break;
        }
        TI rzn = TI(0), rr = TI(0);
#pragma unroll
        for (int k = 0; k < K; ++k) {
            x[k] = tfma(alpha, p[k], x[k]);
            r[k] = tfma(-alpha, q[k], r[k]);
            z[k] = dinv[k] * r[k];
            rzn = tfma(r[k], z[k], rzn);
            rr = tfma(r[k], r[k], rr);
        }
        {
            TI t[2] = {rzn, rr};
            block_allreduce<TI, 2>(t, redB);
            rzn = t[0];
            rr = t[1];
        }
        if (!(rr == rr)) {
            *flag = kNaN;
            break;
        }
        if (rr <= stop2) break;
        const TI beta = rzn / rz;
        rz = rzn;
#pragma unroll
        for (int k = 0; k < K; ++k) p[k] = tfma(beta, p[k], z[k]);
    }
    return it;
}

template <typename TI>
__device__ __forceinline__ const TI* planes_of(const MicroArgs& a, int i);
template <>
__device__ __forceinline__ const float* planes_of<float>(const MicroArgs& a, int i) {
    return a.S32 + (size_t)i * kPlanes * a.nmp;
}
template <>
__device__ __forceinline__ const double* planes_of<double>(const MicroArgs& a, int i) {
    return a.S64 + (size_t)i * kPlanes * a.nmp;
}

template <int K>
struct MaxThreads {
    static constexpr int value = K <= 2 ? 1024 : (K == 4 ? 512 : 544);
};

template <typename TI, bool MIXED, int K>
__global__ void __launch_bounds__(MaxThreads<K>::value) k_micro_solve(MicroArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int W = a.W, W2 = W * W;
    TI* cf = reinterpret_cast<TI*>(smem);
    TI* pp = cf + kPlanes * W2;
    size_t off = (size_t)(kPlanes + 1) * W2 * sizeof(TI);
    off = (off + 15) & ~(size_t)15;
    TI* redA = reinterpret_cast<TI*>(smem + off);
    TI* redB = redA + 64;
    double* dA = reinterpret_cast<double*>(redB + 64);
    double* dB = dA + 96;

    const int i = blockIdx.x;
    const int tid = threadIdx.x, T = blockDim.x;
    const int n1 = a.n1, nm = a.nm;
    const size_t pl = (size_t)a.nmp;

    for (int e = tid; e < (kPlanes + 1) * W2; e += T) cf[e] = TI(0);
    __syncthreads();

    int sidx[K];
    bool valid[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int j = tid + k * T;
        valid[k] = j < nm;
        const int p = valid[k] ? j % n1 : 0, q = valid[k] ? j / n1 : 0;
        sidx[k] = (p + 1) + W * (q + 1);
    }
#define JJ(k) (tid + (k) * T)
    const TI* Sg = planes_of<TI>(a, i);
#pragma unroll
    for (int c = 0; c < kPlanes; ++c) {
#pragma unroll
        for (int k = 0; k < K; ++k)
            if (valid[k]) cf[c * W2 + sidx[k]] = Sg[c * pl + JJ(k)];
    }
    __syncthreads();
    TI dinv[K];
#pragma unroll
    for (int k = 0; k < K; ++k) dinv[k] = valid[k] ? TI(1) / cf[sidx[k]] : TI(0);

    const double* ci = a.c + (size_t)i * pl;
    double* vi = a.v + (size_t)i * pl;
    const double* re = a.redge + (size_t)i * n1;
    const double ku = a.kappa * a.u[i];
    // right-hand side b = c + kappa u_i r_i, re-read from global memory where
    // needed (keeping it in registers would cost 2K registers per thread)
    auto bval = [&](int j) {
        double b = ci[j];
        if (j % n1 == n1 - 1) b = fma(ku, re[j / n1], b);
        return b;
    };
    double bn2 = 0.0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const double b = valid[k] ? bval(JJ(k)) : 0.0;
        bn2 = fma(b, b, bn2);
    }

    int inner = 0, sweeps = 0, flag = 0;
    if constexpr (!MIXED) {
        // ---- FP64 Jacobi-PCG, warm start from v ----
        TI x[K], r[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            x[k] = valid[k] ? vi[JJ(k)] : TI(0);
            if (valid[k]) pp[sidx[k]] = x[k];
        }
        __syncthreads();
        double rr = 0.0;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            r[k] = valid[k] ? bval(JJ(k)) - stencil_smem<TI>(cf, pp, sidx[k], W, W2) : TI(0);
            rr = fma(r[k], r[k], rr);
        }
        {
            double t[2] = {bn2, rr};
            block_allreduce<double, 2>(t, dA);
            bn2 = t[0];
            rr = t[1];
        }
        sweeps = 1;
        const double stop2 = a.tol * a.tol * bn2;
        if (bn2 == 0.0) {
#pragma unroll
            for (int k = 0; k < K; ++k) x[k] = TI(0);
        } else if (!(rr == rr)) {
            flag = kNaN;
        } else if (rr > stop2) {
            inner = pcg_smem<TI, K>(cf, pp, W, W2, sidx, valid, dinv, x, r, (TI)stop2, a.maxit, redA, redB, &flag);
            if (!flag && inner >= a.maxit) {
                // converged exactly at the cap is fine; otherwise flag it
                double rr2 = 0.0;
#pragma unroll
                for (int k = 0; k < K; ++k) rr2 = fma(r[k], r[k], rr2);
                double t[1] = {rr2};
                block_allreduce<double, 1>(t, dB);
                if (t[0] > stop2) flag = kNotConverged;
            }
        }
#pragma unroll
        for (int k = 0; k < K; ++k)
            if (valid[k]) vi[JJ(k)] = x[k];
        __syncthreads();
    } else {
        // ---- FP64 iterative refinement around FP32 inner solves ----
        {
            double t[1] = {bn2};
            block_allreduce<double, 1>(t, dA);
            bn2 = t[0];
        }
        const double stop2 = a.tol * a.tol * bn2;
        if (bn2 == 0.0) {
#pragma unroll
            for (int k = 0; k < K; ++k)
                if (valid[k]) vi[JJ(k)] = 0.0;
            __syncthreads();
        } else {
            const double* S64 = a.S64 + (size_t)i * kPlanes * pl;
            int pass = 1;  // dA still holds the ||b|| partials: start on dB
            for (;;) {
                double r64[K];
                double rr = 0.0;
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    const int j = JJ(k);
                    r64[k] = valid[k] ? bval(j) - stencil_global(S64, pl, vi, j, j % n1, j / n1, n1) : 0.0;
                    rr = fma(r64[k], r64[k], rr);
                }
                double* buf = (pass & 1) ? dB : dA;
                ++pass;
                {
                    double t[1] = {rr};
                    block_allreduce<double, 1>(t, buf);
                    rr = t[0];
                }
                ++sweeps;
                if (!(rr == rr)) {
                    flag = kNaN;
                    break;
                }
                if (rr <= stop2) break;
                if (sweeps > a.max_sweeps || inner >= a.maxit) {
                    flag = kNotConverged;
                    break;
                }
                // The FP32 correction is solved for the unit-norm residual
                // r / ||r|| (the FP32 values keep their range however small
                // the residual is) and scaled back in FP64; the inner solve
                // goes inner_tol below it, but no further than half of what
                // the outer tolerance still needs.
                const double rn = sqrt(rr), rs = 1.0 / rn;
                TI d[K], r[K];
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    d[k] = TI(0);
                    r[k] = (TI)(r64[k] * rs);
                }
                const TI stop32 = (TI)fmax(a.inner_tol * a.inner_tol, 0.25 * stop2 / rr);
                inner += pcg_smem<TI, K>(cf, pp, W, W2, sidx, valid, dinv, d, r, stop32, a.maxit - inner, redA,
                                         redB, &flag);
                if (flag == kNaN) break;
                flag = 0;  // an FP32 breakdown only ends this inner solve; the FP64 residual decides
#pragma unroll
                for (int k = 0; k < K; ++k)
                    if (valid[k]) vi[JJ(k)] = fma(rn, (double)d[k], vi[JJ(k)]);
                __syncthreads();
            }
        }
    }

    // ---- epilogue: boundary flux integral rho_i = r_i^T v_i (compensated) ----
    double rl = 0.0;
#pragma unroll
    for (int k = 0; k < K; ++k)
        if (valid[k] && JJ(k) % n1 == n1 - 1) rl = fma(re[JJ(k) / n1], vi[JJ(k)], rl);
    // dB/dA may still be read by slow threads of the last reduction: use a
    // fresh region (the stats buffer after dB).
    const double rho = block_sum_compensated(rl, dB + 96);
    if (tid == 0) {
        a.rho[i] = rho;
        a.inst_iters[i] = inner;
        atomicAdd(&a.ctl->inner_iters, (unsigned long long)inner);
        atomicAdd(&a.ctl->sweeps, (unsigned long long)sweeps);
        atomicAdd(&a.ctl->micro_solves, 1ull);
        atomicMax(&a.ctl->max_inner, inner);
        if (flag) set_status(a.ctl, flag);
    }
#undef JJ
}

static int smem_threads(int nm, int K) {
    int t = (nm + K - 1) / K;
    return (t + 31) / 32 * 32;
}

static size_t smem_kernel_bytes(int n1, int precision) {
    const size_t W = (size_t)n1 + 2;
    const size_t ti = precision == 0 ? sizeof(double) : sizeof(float);
    size_t off = (kPlanes + 1) * W * W * ti;
    off = (off + 15) & ~(size_t)15;
    return off + 2 * 64 * ti + (96 + 96 + 64) * sizeof(double);
}

template <typename TI, bool MIXED, int K>
static cudaError_t launch_smem(const MicroArgs& a, cudaStream_t s) {
    const int T = smem_threads(a.nm, K);
    if (T > MaxThreads<K>::value) return cudaErrorInvalidConfiguration;
    k_micro_solve<TI, MIXED, K><<<a.nM, T, smem_kernel_bytes(a.n1, MIXED ? 1 : 0), s>>>(a);
    return cudaGetLastError();
}

// ===========================================================================
// Column-strip variant (mixed precision).
//
// Thread t owns R consecutive nodes of one column of the micro grid:
// p = t mod n1, rows q0 .. q0+R-1 with q0 = R (t div n1).  The inner FP32 CG
// runs on the symmetrically Jacobi-scaled operator  S^ = D^-1/2 S D^-1/2
// (unit diagonal, so the Jacobi preconditioner becomes the identity): the
// eight off-diagonal couplings of every node, scaled once with the diagonals
// of both end nodes, sit in registers for the whole solve, and the vector the
// operator is applied to reaches the neighbours through one zero-haloed
// shared-memory plane: per iteration a thread stores R values and loads its
// two neighbour columns (2R + 4 values) plus two halo values of its own
// column.  The plane's row stride is padded so that the rows of consecutive
// strips start in the same bank, which keeps warps that straddle two strips
// free of bank conflicts.  The CG is the Chronopoulos-Gear form: one operator
// application and ONE fused reduction (r.r, r.Ar) per iteration.
//
// FP64 refinement without recomputing b - S v from scratch: the residual of
// the current iterate is kept in global memory (written by the step prologue
// and by every solve), so a solve starts from
//     r = res + kappa (u_i - u_used_i) r_i          (only Robin-edge nodes change)
// and after each FP32 correction d updates it as r -= S d, v += d.  The
// products S d are formed in compensated FP32 from S = S32 + S32lo (S64 to
// about 2^-48; d is exact in FP32) and subtracted from the FP64 residual:
// the stored residual stays within about 1e-12 ||b|| of b - S64 v, while
// FP64 instructions (a small fraction of GB300's FP32 rate) are 7 per node
// instead of about 20.
// A micro problem whose residual already meets the tolerance returns before
// staging anything.  ||b(u)||^2 = ||c||^2 + 2 kappa u c^T r + kappa^2 u^2 ||r||^2
// comes from three per-instance scalars of the prologue.  Convergence tests
// use norms accumulated in FP32 from the FP64 residual values (a norm only
// decides when to stop; the residual itself stays FP64).
// ===========================================================================
// Launch bounds per strip height: R = 3 asks for two resident blocks of up to
// 384 threads (register cap 85), R = 5 and 7 for one block of 512 / 384; the
// tall strips (R = 9, 11, 13, couplings in shared memory) take up to 384
// threads at kTallStripRegs registers.
template <int R>
struct StripMaxThreads {
    static constexpr int value = R == 3 ? 384 : (R == 5 ? 512 : 384);
};
template <int R>
struct StripMinBlocks {
    static constexpr int value = R == 3 ? 2 : 1;
};

__host__ __device__ inline int strip_rows(int n1, int R) { return (n1 + R - 1) / R; }

// Row stride of the shared plane: the smallest W >= n1 + 2 with
// R W = n1 (mod 32).  Thread t = s n1 + p reads plane word (s R + m) W + p,
// which is then t + const (mod 32) for every row offset m, so the 32 lanes of
// a warp hit 32 distinct banks even when the warp straddles two strips.
// Needs R odd when n1 is odd (R is then invertible mod 32).
__host__ __device__ inline int strip_stride(int n1, int R) {
    for (int W = n1 + 2; W < n1 + 2 + 32; ++W)
        if ((R * W - n1) % 32 == 0) return W;
    return n1 + 2;  // not reachable for odd R
}

static int strip_threads(int n1, int R) {
    const int t = n1 * strip_rows(n1, R);
    return (t + 31) / 32 * 32;
}

// Shared memory of a strip block: the plane, 4 x 64 reduction floats and,
// with couplings in shared memory (sc), two float4 per node of the padded
// strip grid (n1 columns x strip_rows * R rows).
static size_t strip_smem_bytes(int n1, int R, bool sc) {
    const size_t W = (size_t)strip_stride(n1, R), H = (size_t)strip_rows(n1, R) * R + 2;
    size_t off = (W * H * sizeof(float) + 15) & ~(size_t)15;
    off += 4 * 64 * sizeof(float);
    if (sc) off += 2 * (size_t)n1 * strip_rows(n1, R) * R * sizeof(float4);
    return off;
}

// The eight scaled off-diagonal couplings of one node.
struct Couple8 {
    float E, W, N, S, NE, NW, SE, SW;
};

// Where a strip's couplings live: in registers (short strips) ...
template <int R>
struct RegCouplings {
    Couple8 c[R];
    __device__ __forceinline__ Couple8 get(int k) const { return c[k]; }
};
// ... or in shared memory as two float4 per node, (E, W, N, S) and
// (NE, NW, SE, SW), node (p, q) at index p + n1 q of the padded strip grid
// (tall strips).
// (The loads are volatile so that the compiler re-reads the couplings at
// every operator application instead of hoisting them into registers.)
__device__ __forceinline__ float4 lds_f4(const float4* p) {
    float4 v;
    const unsigned addr = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(addr)
                 : "memory");
    return v;
}
struct SmemCouplings {
    const float4* A;
    const float4* B;
    int j0, n1;
    __device__ __forceinline__ Couple8 get(int k) const {
        const float4 a = lds_f4(A + j0 + k * n1), b = lds_f4(B + j0 + k * n1);
        return Couple8{a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
    }
};

// Neighbour values of a strip from the shared plane: L/Rt = columns p-1 / p+1
// at rows q0-1 .. q0+R, xm / xp = own column at rows q0-1 and q0+R.
template <int R>
struct StripHalo {
    float L[R + 2], Rt[R + 2], xm, xp;
    __device__ __forceinline__ void load(const float* P, int Wd, int p, int q0) {
#pragma unroll
        for (int m = 0; m < R + 2; ++m) {
            const float* row = P + (q0 + m) * Wd + p;  // plane row of grid row q0-1+m, column p-1
            L[m] = row[0];
            Rt[m] = row[2];
        }
        xm = P[q0 * Wd + p + 1];
        xp = P[(q0 + R + 1) * Wd + p + 1];
    }
};

// y = S^ x = x + off-diagonal part for the R nodes of a strip.
// y = S^ x reading the neighbour columns from the plane with a sliding
// window of three rows (fewer live registers than a loaded halo for tall
// strips).  The plane must hold x.  Entries of nodes outside the mesh (and
// of threads without a strip, whose coupling reads point at node (0, k)) are
// set to zero, so that they stay out of the dot products.
template <int R, class CS>
__device__ __forceinline__ void strip_apply_plane(const CS& cs, const float (&x)[R], const float* P, int Wd, int p,
                                                  int q0, const bool (&valid)[R], float (&y)[R]) {
    const float* cl = P + q0 * Wd + p;  // plane column of grid column p-1, from grid row q0-1
    float l0 = cl[0], l1 = cl[Wd], r0 = cl[2], r1 = cl[Wd + 2];
    const float xm = cl[1], xp = cl[(R + 1) * Wd + 1];
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const float l2 = cl[(k + 2) * Wd], r2 = cl[(k + 2) * Wd + 2];
        const Couple8 c = cs.get(k);
        const float up = (k + 1 < R) ? x[k + 1] : xp;
        const float dn = (k > 0) ? x[k - 1] : xm;
        float t = fmaf(c.E, r1, x[k]);
        t = fmaf(c.W, l1, t);
        t = fmaf(c.N, up, t);
        t = fmaf(c.S, dn, t);
        t = fmaf(c.NE, r2, t);
        t = fmaf(c.NW, l2, t);
        t = fmaf(c.SE, r0, t);
        t = fmaf(c.SW, l0, t);
        y[k] = valid[k] ? t : 0.f;
        l0 = l1;
        l1 = l2;
        r0 = r1;
        r1 = r2;
    }
}

template <int R, class CS>
__device__ __forceinline__ void strip_apply(const CS& cs, const float (&x)[R], const StripHalo<R>& h,
                                            float (&y)[R]) {
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const Couple8 c = cs.get(k);
        const float up = (k + 1 < R) ? x[k + 1] : h.xp;
        const float dn = (k > 0) ? x[k - 1] : h.xm;
        float t = fmaf(c.E, h.Rt[k + 1], x[k]);
        t = fmaf(c.W, h.L[k + 1], t);
        t = fmaf(c.N, up, t);
        t = fmaf(c.S, dn, t);
        t = fmaf(c.NE, h.Rt[k + 2], t);
        t = fmaf(c.NW, h.L[k + 2], t);
        t = fmaf(c.SE, h.Rt[k], t);
        t = fmaf(c.SW, h.L[k], t);
        y[k] = t;
    }
}

template <int R>
__device__ __forceinline__ void strip_store(float* P, int Wd, int p, int q0, const bool (&valid)[R],
                                            const float (&v)[R]) {
#pragma unroll
    for (int k = 0; k < R; ++k)
        if (valid[k]) P[(q0 + k + 1) * Wd + p + 1] = v[k];
}

// Chronopoulos-Gear CG on the scaled operator (Jacobi-PCG on S); x = 0 on
// entry, r = rhs.  Stops when ||r||^2 <= rel2 ||r_0||^2 or after maxit
// iterations; returns the count.  redA/redB: 64-float reduction buffers.
template <int R, class CS>
__device__ int strip_cg(const CS& c, const bool (&valid)[R], float (&x)[R], float (&r)[R], float* P,
                        int Wd, int p, int q0, float rel2, int maxit, float* redA, float* redB, int* flag) {
    float pv[R], s[R], w[R];
    StripHalo<R> h;
    strip_store<R>(P, Wd, p, q0, valid, r);
    __syncthreads();
    if constexpr (R >= 9) {
        strip_apply_plane<R>(c, r, P, Wd, p, q0, valid, w);
    } else {
        h.load(P, Wd, p, q0);
        strip_apply<R>(c, r, h, w);
    }
    float g = 0.f, dl = 0.f;
#pragma unroll
    for (int k = 0; k < R; ++k) {
        g = fmaf(r[k], r[k], g);
        dl = fmaf(r[k], w[k], dl);
        pv[k] = r[k];
        s[k] = w[k];
    }
    {
        float t[2] = {g, dl};
        block_allreduce<float, 2>(t, redA);
        g = t[0];
        dl = t[1];
    }
    const float stop = rel2 * g;
    if (!(dl > 0.f)) {
        *flag = (dl == dl) ? kBreakdown : kNaN;
        return 0;
    }
    // CG scalars with the fast division (a few ulp): they steer the FP32 inner
    // solve only, whose result is checked by the FP64 residual
    float alpha = __fdividef(g, dl);
    int it = 0;
    while (it < maxit) {
#pragma unroll
        for (int k = 0; k < R; ++k) {
            x[k] = fmaf(alpha, pv[k], x[k]);
            r[k] = fmaf(-alpha, s[k], r[k]);
        }
        ++it;
        strip_store<R>(P, Wd, p, q0, valid, r);
        __syncthreads();
        if constexpr (R >= 9) {
            strip_apply_plane<R>(c, r, P, Wd, p, q0, valid, w);
        } else {
            h.load(P, Wd, p, q0);
            strip_apply<R>(c, r, h, w);
        }
        float gn = 0.f, dn = 0.f;
#pragma unroll
        for (int k = 0; k < R; ++k) {
            gn = fmaf(r[k], r[k], gn);
            dn = fmaf(r[k], w[k], dn);
        }
        {
            float t[2] = {gn, dn};
            block_allreduce<float, 2>(t, (it & 1) ? redB : redA);
            gn = t[0];
            dn = t[1];
        }
        if (!(gn == gn) || !(dn == dn)) {
            *flag = kNaN;
            break;
        }
        if (gn <= stop) break;
        const float beta = __fdividef(gn, g);
        const float den = dn - __fdividef(beta * gn, alpha);
        if (!(den > 0.f)) {
            *flag = kBreakdown;
            break;
        }
        alpha = __fdividef(gn, den);
        g = gn;
#pragma unroll
        for (int k = 0; k < R; ++k) {
            pv[k] = fmaf(beta, pv[k], r[k]);
            s[k] = fmaf(beta, s[k], w[k]);
        }
    }
    return it;
}

// Accumulate (hi + lo) x into the unevaluated float pair (s, c) for an FP32
// x: hi x = p + e exactly (TwoProduct with an FMA), s + p = t + err exactly
// (Knuth's TwoSum), and the small parts go to c.  For the nine terms of a
// stencil row the pair carries the FP64 product sum to about 2^-44 of the
// largest partial sum, without the FP64 pipe (a warp-wide FP64 instruction
// costs as much issue as 64 FP32 ones on this part).  The round-to-nearest
// intrinsics keep the compiler from contracting the error-free steps.
__device__ __forceinline__ void df_add_prod(float& s, float& c, float hi, float lo, float x) {
    const float p = __fmul_rn(hi, x);
    const float e = fmaf(hi, x, -p);
    const float t = __fadd_rn(s, p);
    const float bp = __fsub_rn(t, s);
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(p, bp));
    s = t;
    c = __fadd_rn(c, __fadd_rn(err, fmaf(lo, x, e)));
}

template <int R, bool SC, bool PIPE>
__device__ __forceinline__ void micro_strip_body(const MicroArgs& a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int n1 = a.n1, Wd = strip_stride(n1, R);
    const int Hd = strip_rows(n1, R) * R + 2;
    float* P = reinterpret_cast<float*>(smem);
    size_t off = ((size_t)Wd * Hd * sizeof(float) + 15) & ~(size_t)15;
    float* red = reinterpret_cast<float*>(smem + off);  // 4 x 64 floats
    // SC: scaled couplings of the padded strip grid (n1 x strip_rows * R nodes)
    const int ncg = n1 * strip_rows(n1, R) * R;
    float4* cA = reinterpret_cast<float4*>(smem + off + 4 * 64 * sizeof(float));
    float4* cB = cA + ncg;

    const int i = blockIdx.x, tid = threadIdx.x, T = blockDim.x;
    const bool active = tid < n1 * strip_rows(n1, R);
    const int p = active ? tid % n1 : 0;
    const int q0 = active ? (tid / n1) * R : 0;
    const size_t pl = (size_t)a.nmp;
    double* res = a.res + (size_t)i * pl;
    double* v = a.v + (size_t)i * pl;
    const double* re = a.redge + (size_t)i * n1;

    bool valid[R];
#pragma unroll
    for (int k = 0; k < R; ++k) valid[k] = active && (q0 + k) < n1;

    // residual of the current iterate for the new macro value u_i
    const double ui = a.u[i];
    const double kdu = a.kappa * (ui - a.u_used[i]);
    const bool edge = p == n1 - 1;
    // pipelined elimination: right-hand side c = mw + u_old mq, residual
    // res + u_old mq (u_old and the pointers are derived again in the
    // epilogue, so that nothing of this stays live through the CG loop)
    constexpr bool pipe = PIPE;
    double r64[R];
    float rr = 0.f, cc = 0.f;
    {
        const double uo = pipe ? a.u_old[i] : 0.0;
        const double* mqi = a.mq + (size_t)i * pl;
        const double* mwi = a.mw + (size_t)i * pl;
#pragma unroll
        for (int k = 0; k < R; ++k) {
            double r = 0.0;
            if (valid[k]) {
                const int q = q0 + k, j = p + n1 * q;
                r = res[j];
                if (edge) r = fma(kdu, re[q], r);
                if (pipe) {
                    const double m = mqi[j];
                    r = fma(uo, m, r);
                    const float cf = (float)fma(uo, m, mwi[j]);
                    cc = fmaf(cf, cf, cc);
                }
            }
            r64[k] = r;
            rr = fmaf((float)r, (float)r, rr);
        }
    }
    double bn2;
    if (pipe) {
        // ||c||^2 only sets the stopping-test reference: FP32, with an FP64
        // recomputation when the FP32 sum leaves [1e-30, 1e30]
        float t[2] = {rr, cc};
        block_allreduce<float, 2>(t, red + 128);
        rr = t[0];
        bn2 = (double)t[1];
        if (!(bn2 >= 1e-30 && bn2 <= 1e30)) {  // uniform across the block
            const double uo = a.u_old[i];
            const double* mqi = a.mq + (size_t)i * pl;
            const double* mwi = a.mw + (size_t)i * pl;
            double c2[1] = {0.0};
#pragma unroll
            for (int k = 0; k < R; ++k)
                if (valid[k]) {
                    const int j = p + n1 * (q0 + k);
                    const double c = fma(uo, mqi[j], mwi[j]);
                    c2[0] = fma(c, c, c2[0]);
                }
            block_allreduce<double, 1>(c2, reinterpret_cast<double*>(red));
            bn2 = c2[0];
        }
    } else {
        const double* bn = a.bnorm + (size_t)i * 3;
        const double ku = a.kappa * ui;
        bn2 = fma(ku * ku, bn[2], fma(2.0 * ku, bn[1], bn[0]));
        float t[1] = {rr};
        block_allreduce<float, 1>(t, red + 128);
        rr = t[0];
    }
    const float stop2 = (float)(a.tol * a.tol * bn2);
    int inner = 0, sweeps = 0, flag = 0;
    bool solved = false;
    if (!(rr == rr)) flag = kNaN;
    if (bn2 == 0.0) {  // zero right-hand side: the solution is zero
#pragma unroll
        for (int k = 0; k < R; ++k) {
            r64[k] = 0.0;
            if (valid[k]) v[p + n1 * (q0 + k)] = 0.0;
        }
        solved = true;
    } else if (!flag && !(stop2 >= 1.17549435e-38f && bn2 <= 1e37)) {
        // the stopping test and the residual norms are FP32: outside the
        // range where tol^2 ||b||^2 is a normal FP32 number (and ||r||^2 cannot
        // overflow) an underflowed ||r||^2 would read as converged, so the
        // solve reports non-convergence instead (FP64 precision has no limit)
        flag = kNotConverged;
    } else if (!flag && rr > stop2) {
        solved = true;
        // zero the plane (halo and padding stay zero); scaled couplings into
        // registers: c^_jl = c_jl / sqrt(C_j C_l), sc_j = 1 / sqrt(C_j)
        for (int e = tid; e < Wd * Hd; e += T) P[e] = 0.f;
        const float* S = a.S32 + (size_t)i * kPlanes * pl;
        RegCouplings<R> c;
        float sc[R];
#pragma unroll
        for (int k = 0; k < R; ++k) {
            Couple8 s{0, 0, 0, 0, 0, 0, 0, 0};
            float d0 = 1.f;
            if (valid[k]) {
                const int q = q0 + k, j = p + n1 * q;
                const bool w = p > 0, e = p + 1 < n1, sd = q > 0, nd = q + 1 < n1;
                d0 = rsqrtf(S[j]);
                auto dg = [&](int l) { return rsqrtf(S[l]); };
                if (e) s.E = S[pl + j] * dg(j + 1);
                if (w) s.W = S[pl + j - 1] * dg(j - 1);
                if (nd) s.N = S[2 * pl + j] * dg(j + n1);
                if (sd) s.S = S[2 * pl + j - n1] * dg(j - n1);
                if (e && nd) s.NE = S[3 * pl + j] * dg(j + n1 + 1);
                if (w && nd) s.NW = S[4 * pl + j] * dg(j + n1 - 1);
                if (e && sd) s.SE = S[4 * pl + j - n1 + 1] * dg(j - n1 + 1);
                if (w && sd) s.SW = S[3 * pl + j - n1 - 1] * dg(j - n1 - 1);
                s.E *= d0; s.W *= d0; s.N *= d0; s.S *= d0;
                s.NE *= d0; s.NW *= d0; s.SE *= d0; s.SW *= d0;
            }
            c.c[k] = s;
            sc[k] = valid[k] ? d0 : 0.f;
            if (SC && active) {  // padding rows of the last strip get zero couplings
                const int j = p + n1 * (q0 + k);
                cA[j] = make_float4(s.E, s.W, s.N, s.S);
                cB[j] = make_float4(s.NE, s.NW, s.SE, s.SW);
            }
        }
        __syncthreads();
        const SmemCouplings cs{cA, cB, p + n1 * q0, n1};
        const float* Sh = S;                                   // S64 = Sh + Sl to about 2^-48
        const float* Sl = a.S32lo + (size_t)i * kPlanes * pl;
        for (;;) {
            if (sweeps >= a.max_sweeps || inner >= a.maxit) {
                flag = kNotConverged;
                break;
            }
            // FP32 correction on the scaled system S^ y = D^-1/2 r, d = D^-1/2 y,
            // to inner_tol relative, but no further than half the outer
            // tolerance requires.  The FP64 residual waits in global memory.
            float y[R], r[R];
#pragma unroll
            for (int k = 0; k < R; ++k) {
                y[k] = 0.f;
                r[k] = sc[k] * (float)r64[k];
                if (valid[k]) res[p + n1 * (q0 + k)] = r64[k];
            }
            const float rel2 = fmaxf(a.inner_tol * a.inner_tol, 0.25f * stop2 / rr);
            if (SC)
                inner += strip_cg<R>(cs, valid, y, r, P, Wd, p, q0, rel2, a.maxit - inner, red, red + 64, &flag);
            else
                inner += strip_cg<R>(c, valid, y, r, P, Wd, p, q0, rel2, a.maxit - inner, red, red + 64, &flag);
            if (flag == kNaN) break;
            flag = 0;
            // v += d and r -= S d with S = S32 + S32lo (S64 to about 2^-48)
            // and the FP32 correction d: the products and their sum in
            // compensated FP32, one FP64 subtraction from the stored residual
            float d[R];
#pragma unroll
            for (int k = 0; k < R; ++k) d[k] = sc[k] * y[k];
            strip_store<R>(P, Wd, p, q0, valid, d);
            __syncthreads();
            StripHalo<R> h;
            h.load(P, Wd, p, q0);
            rr = 0.f;
#pragma unroll
            for (int k = 0; k < R; ++k) {
                if (!valid[k]) continue;
                const int q = q0 + k, j = p + n1 * q;
                const bool w = p > 0, e = p + 1 < n1, sd = q > 0;
                const float up = (k + 1 < R) ? d[k + 1] : h.xp;
                const float dn = (k > 0) ? d[k - 1] : h.xm;
                float ys = 0.f, yc = 0.f;
                df_add_prod(ys, yc, Sh[j], Sl[j], d[k]);
                df_add_prod(ys, yc, Sh[pl + j], Sl[pl + j], h.Rt[k + 1]);
                if (w) df_add_prod(ys, yc, Sh[pl + j - 1], Sl[pl + j - 1], h.L[k + 1]);
                df_add_prod(ys, yc, Sh[2 * pl + j], Sl[2 * pl + j], up);
                if (sd) df_add_prod(ys, yc, Sh[2 * pl + j - n1], Sl[2 * pl + j - n1], dn);
                df_add_prod(ys, yc, Sh[3 * pl + j], Sl[3 * pl + j], h.Rt[k + 2]);
                df_add_prod(ys, yc, Sh[4 * pl + j], Sl[4 * pl + j], h.L[k + 2]);
                if (e && sd) df_add_prod(ys, yc, Sh[4 * pl + j - n1 + 1], Sl[4 * pl + j - n1 + 1], h.Rt[k]);
                if (w && sd) df_add_prod(ys, yc, Sh[3 * pl + j - n1 - 1], Sl[3 * pl + j - n1 - 1], h.L[k]);
                r64[k] = res[j] - ((double)ys + (double)yc);
                const float rf = (float)r64[k];
                rr = fmaf(rf, rf, rr);
                v[j] += (double)d[k];
            }
            {
                float t[1] = {rr};
                block_allreduce<float, 1>(t, red + 128 + 64 * (sweeps & 1));
                rr = t[0];
            }
            ++sweeps;
            if (!(rr == rr)) {
                flag = kNaN;
                break;
            }
            if (rr <= stop2) break;
        }
    }
    // store the residual of the new iterate (only Robin-edge values change
    // when no correction was needed); the pipelined epilogue stores its own
    if (!pipe) {
#pragma unroll
        for (int k = 0; k < R; ++k)
            if (valid[k] && (solved || (edge && kdu != 0.0))) res[p + n1 * (q0 + k)] = r64[k];
    }
    __syncthreads();
    // pipelined elimination, first half of the epilogue (w = v is final):
    // M w / dt, S w = c - e, push w and S w into the rings at slot hist_step,
    // the extrapolated warm start g with S g from the same combination
    // (quadratic with two older solves, linear with one), and the next
    // residual's u-independent part M w / dt - S g.  Only v is read at
    // neighbours, so everything but g is stored at once.
    double gv[R];
    if (pipe) {
        const int st = a.ctl->hist_step, level = a.ctl->hist_level;
        const double uo = a.u_old[i];
        const double* mqi = a.mq + (size_t)i * pl;
        double* mwi = a.mw + (size_t)i * pl;
        const size_t slot = (size_t)a.nM * pl, io = (size_t)i * pl;
        const double* Mi = a.M64 + (size_t)i * kPlanes * pl;
        double* hc = a.hist + (size_t)(st % 3) * slot + io;
        const double* h1 = a.hist + (size_t)((st + 2) % 3) * slot + io;
        const double* h2 = a.hist + (size_t)((st + 1) % 3) * slot + io;
        double* yc = a.yhist + (size_t)(st % 3) * slot + io;
        const double* y1 = a.yhist + (size_t)((st + 2) % 3) * slot + io;
        const double* y2 = a.yhist + (size_t)((st + 1) % 3) * slot + io;
#pragma unroll
        for (int k = 0; k < R; ++k) {
            gv[k] = 0.0;
            if (!valid[k]) continue;
            const int q = q0 + k, j = p + n1 * q;
            const double w = v[j];
            const double mwn = plane_apply(Mi, pl, v, j, p, q, n1) * a.idt;
            const double sw = fma(uo, mqi[j], mwi[j]) - r64[k];
            double g = w, sg = sw;
            if (level >= 2) {
                g = fma(3.0, w - h1[j], h2[j]);
                sg = fma(3.0, sw - y1[j], y2[j]);
            } else if (level == 1) {
                g = fma(2.0, w, -h1[j]);
                sg = fma(2.0, sw, -y1[j]);
            }
            hc[j] = w;
            yc[j] = sw;
            mwi[j] = mwn;
            res[j] = mwn - sg;
            gv[k] = g;
        }
    }
    // optional epilogue: M v / dt of the solution in FP64 (the next step's
    // right-hand side of the pipelined elimination; the FP64 work overlaps
    // the FP32 iterations of the other blocks on the SM)
    if (a.mw && !pipe) {
        const double* Mi = a.M64 + (size_t)i * kPlanes * pl;
        double* mw = a.mw + (size_t)i * pl;
#pragma unroll
        for (int k = 0; k < R; ++k)
            if (valid[k]) {
                const int q = q0 + k, j = p + n1 * q;
                mw[j] = plane_apply(Mi, pl, v, j, p, q, n1) * a.idt;
            }
    }
    // flux integral rho_i = r_i^T v_i over the Robin-edge nodes, one warp,
    // compensated (TwoSum) FP64
    if (tid < 32) {
        double s = 0.0, cpen = 0.0;
        for (int q = tid; q < n1; q += 32) {
            const double t = re[q] * v[(n1 - 1) + n1 * q];
            double su, er;
            two_sum(s, t, su, er);
            s = su;
            cpen += er;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double so = __shfl_xor_sync(0xffffffffu, s, o);
            const double co = __shfl_xor_sync(0xffffffffu, cpen, o);
            double su, er;
            two_sum(s, so, su, er);
            s = su;
            cpen += co + er;
        }
        if (tid == 0) {
            a.u_used[i] = ui;
            a.rho[i] = s + cpen;
            a.inst_iters[i] = inner;
            atomicAdd(&a.ctl->inner_iters, (unsigned long long)inner);
            atomicAdd(&a.ctl->sweeps, (unsigned long long)sweeps);
            atomicAdd(&a.ctl->micro_solves, 1ull);
            atomicMax(&a.ctl->max_inner, inner);
            if (flag) set_status(a.ctl, flag);
        }
    }
    // pipelined elimination, second half: once every read of w (neighbours,
    // flux) is done, v becomes the warm start of the next solve
    if (pipe) {
        __syncthreads();
#pragma unroll
        for (int k = 0; k < R; ++k)
            if (valid[k]) v[p + n1 * (q0 + k)] = gv[k];
        if (i == 0 && tid == 0) a.ctl->pushed = 1;
    }
}

// Short strips (couplings in registers) and tall strips (couplings in shared
// memory, register budget capped so that several blocks share an SM).  PIPE:
// the pipelined-elimination instantiation (MicroArgs::pipe), separate so that
// its prologue and epilogue cost the other solves no registers.
template <int R, bool PIPE>
__global__ void __launch_bounds__(StripMaxThreads<R>::value, StripMinBlocks<R>::value) k_micro_strip(MicroArgs a) {
    micro_strip_body<R, false, PIPE>(a);
}
constexpr int kTallStripRegs = 160;
template <int R, bool PIPE>
__global__ void __maxnreg__(kTallStripRegs) k_micro_strip_tall(MicroArgs a) {
    micro_strip_body<R, true, PIPE>(a);
}

template <int R, bool SC>
static cudaError_t launch_strip(const MicroArgs& a, cudaStream_t s) {
    const int T = strip_threads(a.n1, R);
    if (T > StripMaxThreads<R>::value) return cudaErrorInvalidConfiguration;
    const size_t sm = strip_smem_bytes(a.n1, R, SC);
    if constexpr (SC) {
        if (a.pipe) k_micro_strip_tall<R, true><<<a.nM, T, sm, s>>>(a);
        else k_micro_strip_tall<R, false><<<a.nM, T, sm, s>>>(a);
    } else {
        if (a.pipe) k_micro_strip<R, true><<<a.nM, T, sm, s>>>(a);
        else k_micro_strip<R, false><<<a.nM, T, sm, s>>>(a);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// variant table
// ---------------------------------------------------------------------------
static const int kSmemK[4] = {1, 2, 4, 8};
static const int kStripR[6] = {3, 5, 7, 9, 11, 13};  // 3..7 couplings in registers, 9..13 in shared memory

bool tiling_uses_stored_residual(int tiling) { return tiling >= 4; }

bool tiling_fits(int tiling, int precision, int n1, int smem_optin) {
    const int nm = n1 * n1;
    if (tiling >= 0 && tiling < 4) {
        const int K = kSmemK[tiling];
        const int maxT = K <= 2 ? 1024 : (K == 4 ? 512 : 544);
        return smem_threads(nm, K) <= maxT && smem_kernel_bytes(n1, precision) <= (size_t)smem_optin;
    }
    if (tiling >= 4 && tiling < kNumTilings) {
        if (precision == 0) return false;
        const int R = kStripR[tiling - 4];
        const bool sc = R >= 9;
        const int maxT = R == 3 ? 384 : (R == 5 ? 512 : 384);
        return strip_threads(n1, R) <= maxT && strip_smem_bytes(n1, R, sc) <= (size_t)smem_optin;
    }
    return false;
}

cudaError_t launch_micro_solve(const MicroArgs& a, int precision, int tiling, cudaStream_t s) {
    if (precision == 0) {
        switch (tiling) {
            case 0: return launch_smem<double, false, 1>(a, s);
            case 1: return launch_smem<double, false, 2>(a, s);
            case 2: return launch_smem<double, false, 4>(a, s);
            case 3: return launch_smem<double, false, 8>(a, s);
        }
    } else {
        switch (tiling) {
            case 0: return launch_smem<float, true, 1>(a, s);
            case 1: return launch_smem<float, true, 2>(a, s);
            case 2: return launch_smem<float, true, 4>(a, s);
            case 3: return launch_smem<float, true, 8>(a, s);
            case 4: return launch_strip<3, false>(a, s);
            case 5: return launch_strip<5, false>(a, s);
            case 6: return launch_strip<7, false>(a, s);
            case 7: return launch_strip<9, true>(a, s);
            case 8: return launch_strip<11, true>(a, s);
            case 9: return launch_strip<13, true>(a, s);
        }
    }
    return cudaErrorInvalidValue;
}

// Allow every variant the device's opt-in shared memory (done once, outside
// any stream capture).
cudaError_t configure_micro_kernels(int smem_optin) {
    const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e = cudaSuccess;
    const void* fns[20] = {(const void*)k_micro_solve<double, false, 1>, (const void*)k_micro_solve<double, false, 2>,
                           (const void*)k_micro_solve<double, false, 4>, (const void*)k_micro_solve<double, false, 8>,
                           (const void*)k_micro_solve<float, true, 1>,   (const void*)k_micro_solve<float, true, 2>,
                           (const void*)k_micro_solve<float, true, 4>,   (const void*)k_micro_solve<float, true, 8>,
                           (const void*)k_micro_strip<3, false>,         (const void*)k_micro_strip<5, false>,
                           (const void*)k_micro_strip<7, false>,         (const void*)k_micro_strip_tall<9, false>,
                           (const void*)k_micro_strip_tall<11, false>,   (const void*)k_micro_strip_tall<13, false>,
                           (const void*)k_micro_strip<3, true>,          (const void*)k_micro_strip<5, true>,
                           (const void*)k_micro_strip<7, true>,          (const void*)k_micro_strip_tall<9, true>,
                           (const void*)k_micro_strip_tall<11, true>,    (const void*)k_micro_strip_tall<13, true>};
    for (int k = 0; k < 20 && e == cudaSuccess; ++k) e = cudaFuncSetAttribute(fns[k], at, smem_optin);
    return e;
}

// ---------------------------------------------------------------------------
// Per-step prologue (one block per instance), all FP64:
//   c   = M (v^n/dt + fv) + R g                (right-hand side without the u term)
//   res = c + kappa u r - S v^n                (residual of the warm start v^n)
//   bnorm = (||c||^2, c^T r, ||r||^2)          (||b(u)|| for any u)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_micro_prologue(PrologueArgs a) {
    __shared__ double buf[3 * 32];
    const int i = blockIdx.x;
    const int n1 = a.n1, nm = a.nm;
    const size_t pl = (size_t)a.nmp;
    const double* M = a.M64 + (size_t)i * kPlanes * pl;
    const double* S = a.S64 + (size_t)i * kPlanes * pl;
    const double* v = a.v + (size_t)i * pl;
    const double* fv = a.fv ? a.fv + (size_t)i * pl : nullptr;
    const double* g = a.g ? a.g + (size_t)i * n1 : nullptr;
    const double* re = a.redge + (size_t)i * n1;
    const double idt = 1.0 / a.dt;
    const double ku = a.kappa * a.u[i];
    double* c = a.c + (size_t)i * pl;
    double* res = a.res + (size_t)i * pl;
    double cc = 0.0, cr = 0.0, rr = 0.0;
    for (int j = threadIdx.x; j < nm; j += blockDim.x) {
        const int p = j % n1, q = j / n1;
        double y = plane_apply(M, pl, v, j, p, q, n1) * idt;
        if (fv) y += plane_apply(M, pl, fv, j, p, q, n1);
        double rj = 0.0;
        if (p == n1 - 1) {
            rj = re[q];
            if (g) {
                const double* Rd = a.Rd + (size_t)i * n1;
                const double* Ru = a.Ru + (size_t)i * n1;
                y = fma(Rd[q], g[q], y);
                if (q + 1 < n1) y = fma(Ru[q], g[q + 1], y);
                if (q > 0) y = fma(Ru[q - 1], g[q - 1], y);
            }
        }
        c[j] = y;
        if (!a.phi) res[j] = fma(ku, rj, y) - plane_apply(S, pl, v, j, p, q, n1);
        cc = fma(y, y, cc);
        cr = fma(y, rj, cr);
        rr = fma(rj, rj, rr);
    }
    if (a.phi) {
        // exact elimination: the unknown is v0 with S v0 = c; its warm start
        // is v^n - u^n phi (= the previous step's v0 when v^n was committed
        // as v0 + u^n phi)
        const double* ph = a.phi + (size_t)i * pl;
        double* vw = a.v + (size_t)i * pl;
        const double uw = a.uw[i];
        __syncthreads();  // every thread has read v^n for c
        for (int j = threadIdx.x; j < nm; j += blockDim.x) vw[j] = fma(-uw, ph[j], vw[j]);
        __syncthreads();
        for (int j = threadIdx.x; j < nm; j += blockDim.x)
            res[j] = c[j] - plane_apply(S, pl, v, j, j % n1, j / n1, n1);
    }
    double t[3] = {cc, cr, rr};
    block_allreduce<double, 3>(t, buf);
    if (threadIdx.x == 0) {
        double* bn = a.bnorm + (size_t)i * 3;
        bn[0] = t[0];
        bn[1] = t[1];
        bn[2] = t[2];
        a.u_used[i] = a.phi ? 0.0 : a.u[i];
    }
}

__global__ void __launch_bounds__(128) k_phi_setup(PhiSetupArgs a) {
    __shared__ double buf[32];
    const int i = blockIdx.x, n1 = a.n1;
    const size_t pl = (size_t)a.nmp;
    const double* re = a.redge + (size_t)i * n1;
    double rr = 0.0;
    for (int j = threadIdx.x; j < a.nmp; j += blockDim.x) {
        const int p = j % n1, q = j / n1;
        const bool edge = j < a.nm && p == n1 - 1;
        const double rj = edge ? re[q] : 0.0;
        a.phi[i * pl + j] = 0.0;
        a.cz[i * pl + j] = 0.0;
        a.res[i * pl + j] = a.kappa * rj;
        rr = fma(rj, rj, rr);
    }
    double t[1] = {rr};
    block_allreduce<double, 1>(t, buf);
    if (threadIdx.x == 0) {
        a.bnorm[(size_t)i * 3] = 0.0;
        a.bnorm[(size_t)i * 3 + 1] = 0.0;
        a.bnorm[(size_t)i * 3 + 2] = t[0];
        a.u_used[i] = 1.0;
    }
}

cudaError_t launch_phi_setup(const PhiSetupArgs& a, cudaStream_t s) {
    k_phi_setup<<<a.nM, 128, 0, s>>>(a);
    return cudaGetLastError();
}

// v_i += u_i phi_i, one thread per (instance, DoF)
__global__ void __launch_bounds__(256) k_commit(int nm, int nmp, const double* __restrict__ u,
                                                const double* __restrict__ phi, double* __restrict__ v) {
    const int i = blockIdx.x;  // instances on grid.x (up to 2^31 - 1)
    const int j = blockIdx.y * blockDim.x + threadIdx.x;
    if (j >= nm) return;
    const size_t o = (size_t)i * nmp + j;
    v[o] = fma(u[i], phi[o], v[o]);
}

cudaError_t launch_commit(int nm, int nmp, int nM, const double* u, const double* phi, double* v, cudaStream_t s) {
    dim3 grid(nM, (nm + 255) / 256);
    k_commit<<<grid, 256, 0, s>>>(nm, nmp, u, phi, v);
    return cudaGetLastError();
}

__global__ void k_sub(const double* a, const double* b, double* out, int n) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) out[k] = a[k] - b[k];
}

cudaError_t launch_sub(const double* a, const double* b, double* out, int n, cudaStream_t s) {
    k_sub<<<(n + 255) / 256, 256, 0, s>>>(a, b, out, n);
    return cudaGetLastError();
}

cudaError_t launch_micro_prologue(const PrologueArgs& a, cudaStream_t s) {
    k_micro_prologue<<<a.nM, 256, 0, s>>>(a);
    return cudaGetLastError();
}

// vbar_i = 1^T M_i v_i / vol_i = lm_i^T v_i / vol_i (M_i symmetric).  One
// warp per instance, plain FP64 sums in a fixed order (a block-wide or
// compensated reduction per instance costs more FP64 issue than the whole sum
// on GB300).
__global__ void __launch_bounds__(256) k_vbar(int nm, int nmp, int nM, const double* __restrict__ lm,
                                              const double* __restrict__ vol, const double* __restrict__ v,
                                              double* vbar) {
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= nM) return;
    const size_t base = (size_t)i * nmp;
    double s = 0.0;
    for (int j = lane; j < nm; j += 32) s = fma(lm[base + j], v[base + j], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) vbar[i] = s / vol[i];
}

cudaError_t launch_vbar(int nm, int nmp, int nM, const double* lm, const double* vol, const double* v, double* vbar,
                        cudaStream_t s) {
    k_vbar<<<(nM + 7) / 8, 256, 0, s>>>(nm, nmp, nM, lm, vol, v, vbar);
    return cudaGetLastError();
}

// rho_i = r_i^T v_i over the Robin-edge nodes (the coupling moment of Eq. (17)
// that feeds the macro source) and F_i = kappa (|Gamma_i| u_i - rho_i) + r_i^T g_i.
// One warp per instance; both sums are compensated (TwoSum along the lanes,
// then a TwoSum butterfly), in a fixed order.  flux and rho may each be null.
__global__ void __launch_bounds__(256) k_flux(int n1, int nmp, int nM, double kappa, const double* __restrict__ gam,
                                              const double* __restrict__ u, const double* __restrict__ v,
                                              const double* __restrict__ redge, const double* __restrict__ g,
                                              double* flux, double* rho_out) {
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= nM) return;
    double s = 0.0, c = 0.0, sg = 0.0, cg = 0.0;
    for (int q = lane; q < n1; q += 32) {
        const double r = redge[(size_t)i * n1 + q];
        double t, e;
        two_sum(s, r * v[(size_t)i * nmp + (n1 - 1) + (size_t)n1 * q], t, e);
        s = t;
        c += e;
        if (g) {
            two_sum(sg, r * g[(size_t)i * n1 + q], t, e);
            sg = t;
            cg += e;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        double t, e;
        two_sum(s, __shfl_xor_sync(0xffffffffu, s, o), t, e);
        s = t;
        c += __shfl_xor_sync(0xffffffffu, c, o) + e;
        two_sum(sg, __shfl_xor_sync(0xffffffffu, sg, o), t, e);
        sg = t;
        cg += __shfl_xor_sync(0xffffffffu, cg, o) + e;
    }
    if (lane == 0) {
        const double rho = s + c;
        if (rho_out) rho_out[i] = rho;
        if (flux) flux[i] = kappa * (gam[i] * u[i] - rho) + (sg + cg);
    }
}

cudaError_t launch_flux(int n1, int nm, int nmp, int nM, double kappa, const double* gam, const double* u,
                        const double* v, const double* redge, const double* g, double* flux, double* rho,
                        cudaStream_t s) {
    (void)nm;
    k_flux<<<(nM + 7) / 8, 256, 0, s>>>(n1, nmp, nM, kappa, gam, u, v, redge, g, flux, rho);
    return cudaGetLastError();
}

}  // namespace tsf
