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
                TI d[K], r[K];
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    d[k] = TI(0);
                    r[k] = (TI)r64[k];
                }
                const TI stop32 = (TI)(a.inner_tol * a.inner_tol * rr);
                inner += pcg_smem<TI, K>(cf, pp, W, W2, sidx, valid, dinv, d, r, stop32, a.maxit - inner, redA,
                                         redB, &flag);
                if (flag == kNaN) break;
                flag = 0;  // an FP32 breakdown only ends this inner solve; the FP64 residual decides
#pragma unroll
                for (int k = 0; k < K; ++k)
                    if (valid[k]) vi[JJ(k)] += (double)d[k];
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

int micro_threads(int nm, int K) {
    int t = (nm + K - 1) / K;
    return (t + 31) / 32 * 32;
}

size_t micro_smem_bytes(int n1, int precision) {
    const size_t W = (size_t)n1 + 2;
    const size_t ti = precision == 0 ? sizeof(double) : sizeof(float);
    size_t off = (kPlanes + 1) * W * W * ti;
    off = (off + 15) & ~(size_t)15;
    return off + 2 * 64 * ti + (96 + 96 + 64) * sizeof(double);
}

template <typename TI, bool MIXED, int K>
static cudaError_t launch_one(const MicroArgs& a, cudaStream_t s) {
    const int T = micro_threads(a.nm, K);
    if (T > MaxThreads<K>::value) return cudaErrorInvalidConfiguration;
    const size_t sm = micro_smem_bytes(a.n1, MIXED ? 1 : 0);
    k_micro_solve<TI, MIXED, K><<<a.nM, T, sm, s>>>(a);
    return cudaGetLastError();
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
    return e;
}

cudaError_t launch_micro_solve(const MicroArgs& a, int precision, int K, cudaStream_t s) {
    if (precision == 0) {
        switch (K) {
            case 1: return launch_one<double, false, 1>(a, s);
            case 2: return launch_one<double, false, 2>(a, s);
            case 4: return launch_one<double, false, 4>(a, s);
            case 8: return launch_one<double, false, 8>(a, s);
        }
    } else {
        switch (K) {
            case 1: return launch_one<float, true, 1>(a, s);
            case 2: return launch_one<float, true, 2>(a, s);
            case 4: return launch_one<float, true, 4>(a, s);
            case 8: return launch_one<float, true, 8>(a, s);
        }
    }
    return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// Per-step prologue: c_i = M_i (v_i^n/dt + fv_i) + R_i g_i and G_i = r_i^T g_i
// (right-hand side of the micro equations without the u term, Eq. (17)
// second line, made parabolic).  One block per instance.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_micro_prologue(PrologueArgs a) {
    __shared__ double buf[128];
    const int i = blockIdx.x;
    const int n1 = a.n1, nm = a.nm;
    const size_t pl = (size_t)a.nmp;
    const double* M = a.M64 + (size_t)i * kPlanes * pl;
    const double* v = a.v + (size_t)i * pl;
    const double* fv = a.fv ? a.fv + (size_t)i * pl : nullptr;
    const double* g = a.g ? a.g + (size_t)i * n1 : nullptr;
    const double idt = 1.0 / a.dt;
    double* c = a.c + (size_t)i * pl;
    for (int j = threadIdx.x; j < nm; j += blockDim.x) {
        const int p = j % n1, q = j / n1;
        auto w = [&](int l) { return fv ? fma(v[l], idt, fv[l]) : v[l] * idt; };
        double y = M[j] * w(j);
        const bool e = p + 1 < n1, wst = p > 0;
        if (e) y = fma(M[pl + j], w(j + 1), y);
        if (wst) y = fma(M[pl + j - 1], w(j - 1), y);
        if (q + 1 < n1) {
            y = fma(M[2 * pl + j], w(j + n1), y);
            if (e) y = fma(M[3 * pl + j], w(j + n1 + 1), y);
            if (wst) y = fma(M[4 * pl + j], w(j + n1 - 1), y);
        }
        if (q > 0) {
            y = fma(M[2 * pl + j - n1], w(j - n1), y);
            if (wst) y = fma(M[3 * pl + j - n1 - 1], w(j - n1 - 1), y);
            if (e) y = fma(M[4 * pl + j - n1 + 1], w(j - n1 + 1), y);
        }
        if (g && p == n1 - 1) {
            const double* Rd = a.Rd + (size_t)i * n1;
            const double* Ru = a.Ru + (size_t)i * n1;
            y = fma(Rd[q], g[q], y);
            if (q + 1 < n1) y = fma(Ru[q], g[q + 1], y);
            if (q > 0) y = fma(Ru[q - 1], g[q - 1], y);
        }
        c[j] = y;
    }
    double gl = 0.0;
    if (g)
        for (int q = threadIdx.x; q < n1; q += blockDim.x) gl = fma(a.redge[(size_t)i * n1 + q], g[q], gl);
    const double G = block_sum_compensated(gl, buf);
    if (threadIdx.x == 0) a.G[i] = G;
}

cudaError_t launch_micro_prologue(const PrologueArgs& a, cudaStream_t s) {
    k_micro_prologue<<<a.nM, 256, 0, s>>>(a);
    return cudaGetLastError();
}

// vbar_i = 1^T M_i v_i / vol_i = lm_i^T v_i / vol_i (M_i symmetric)
__global__ void __launch_bounds__(256) k_vbar(int nm, int nmp, const double* __restrict__ lm,
                                              const double* __restrict__ vol, const double* __restrict__ v,
                                              double* vbar) {
    __shared__ double buf[64];
    const int i = blockIdx.x;
    double s = 0.0;
    for (int j = threadIdx.x; j < nm; j += blockDim.x) s = fma(lm[(size_t)i * nmp + j], v[(size_t)i * nmp + j], s);
    const double t = block_sum_compensated(s, buf);
    if (threadIdx.x == 0) vbar[i] = t / vol[i];
}

cudaError_t launch_vbar(int nm, int nmp, int nM, const double* lm, const double* vol, const double* v, double* vbar,
                        cudaStream_t s) {
    k_vbar<<<nM, 256, 0, s>>>(nm, nmp, lm, vol, v, vbar);
    return cudaGetLastError();
}

// F_i = kappa (|Gamma_i| u_i - r_i^T v_i) + r_i^T g_i   (one thread per instance)
__global__ void k_flux(int n1, int nm, int nmp, int nM, double kappa, const double* __restrict__ gam,
                       const double* __restrict__ u, const double* __restrict__ v,
                       const double* __restrict__ redge, const double* __restrict__ g, double* flux) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nM) return;
    double rho = 0.0, G = 0.0;
    for (int q = 0; q < n1; ++q) {
        const double r = redge[(size_t)i * n1 + q];
        rho = fma(r, v[(size_t)i * nmp + (n1 - 1) + (size_t)n1 * q], rho);
        if (g) G = fma(r, g[(size_t)i * n1 + q], G);
    }
    flux[i] = kappa * (gam[i] * u[i] - rho) + G;
}

cudaError_t launch_flux(int n1, int nm, int nmp, int nM, double kappa, const double* gam, const double* u,
                        const double* v, const double* redge, const double* g, double* flux, cudaStream_t s) {
    k_flux<<<(nM + 127) / 128, 128, 0, s>>>(n1, nm, nmp, nM, kappa, gam, u, v, redge, g, flux);
    return cudaGetLastError();
}

}  // namespace tsf
