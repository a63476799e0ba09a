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

// ---------------------------------------------------------------------------
// variant table
// ---------------------------------------------------------------------------
static const int kSmemK[4] = {1, 2, 4, 8};
static const int kStripR[6] = {3, 5, 7, 9, 11, 13};  // 3..7 couplings in registers, 9..13 in shared memory

bool tiling_uses_stored_residual(int tiling) { return tiling >= 4 && tiling != kTilingDirect; }

bool tiling_fits(int tiling, int precision, int n1, int smem_optin) {
    const int nm = n1 * n1;
    if (tiling >= 0 && tiling < 4) {
        const int K = kSmemK[tiling];
        const int maxT = K <= 2 ? 1024 : (K == 4 ? 512 : 544);
        return smem_threads(nm, K) <= maxT && smem_kernel_bytes(n1, precision) <= (size_t)smem_optin;
    }
    if (tiling >= 4 && tiling < kTilingDirect) return precision != 0 && strip_fits(n1, kStripR[tiling - 4], smem_optin);
    if (tiling >= kFirstClusterTiling && tiling < kFirstWarpTiling)
        return precision != 0 && cluster_fits(tiling - kFirstClusterTiling, n1, smem_optin);
    if (tiling >= kFirstWarpTiling && tiling < kNumTilings)
        return precision != 0 && warp_fits(n1, tiling == kFirstWarpTiling ? 3 : 5, smem_optin);
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
        }
        if (tiling >= 4 && tiling < kTilingDirect) return launch_strip_solve(with_fp32_tols(a), kStripR[tiling - 4], s);
        if (tiling >= kFirstClusterTiling && tiling < kFirstWarpTiling)
            return launch_cluster_solve(with_fp32_tols(a), tiling - kFirstClusterTiling, s);
        if (tiling >= kFirstWarpTiling && tiling < kNumTilings)
            return launch_warp_solve(with_fp32_tols(a), tiling == kFirstWarpTiling ? 3 : 5, s);
    }
    return cudaErrorInvalidValue;
}

// Allow every variant the device's opt-in shared memory (done once, outside
// any stream capture).
cudaError_t configure_micro_kernels(int smem_optin) {
    const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e = cudaSuccess;
    const void* fns[8] = {(const void*)k_micro_solve<double, false, 1>, (const void*)k_micro_solve<double, false, 2>,
                          (const void*)k_micro_solve<double, false, 4>, (const void*)k_micro_solve<double, false, 8>,
                          (const void*)k_micro_solve<float, true, 1>,   (const void*)k_micro_solve<float, true, 2>,
                          (const void*)k_micro_solve<float, true, 4>,   (const void*)k_micro_solve<float, true, 8>};
    for (int k = 0; k < 8 && e == cudaSuccess; ++k) e = cudaFuncSetAttribute(fns[k], at, smem_optin);
    if (e == cudaSuccess) e = configure_strip_kernels(smem_optin);
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
