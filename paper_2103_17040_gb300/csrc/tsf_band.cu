// tsf_band.cu -- direct micro solves for operators that stay fixed across
// many right-hand sides: a banded Cholesky factor of every micro operator in
// FP32, triangular solves for up to three right-hand sides per pass, and FP64
// iterative refinement (residual with the FP64 stencil).
//
// With the nodes in lexicographic order the 9-point Q1 stencil has
// half-bandwidth n1 + 1, and so has its Cholesky factor (no fill outside the
// band).  Layout of the factor of instance i: column k of L at
// L + (i nm + k) B, B = n1 + 2 values: [1 / L_kk, L_{k+1,k}, ..., L_{k+B-1,k}]
// (zero below the matrix).  Both triangular solves read whole columns, so
// every solve streams the factor contiguously.
//
// k_band_factor: one block per micro problem, right-looking band Cholesky on
// a B x B sliding window of the trailing matrix in shared memory (circular
// row/column slots); a finished column leaves the window, the next row of S
// (its five stored couplings) enters it.
// k_band_solve: one warp per micro problem: forward substitution with the
// pending right-hand side values spread over the lanes (3 slots a lane),
// backward substitution as one warp dot product per column.
// k_band_residual: r = c - S x in FP64 for the right-hand sides still open,
// and the per-problem convergence test ||r|| <= tol ||c||.
#include "tsf_internal.cuh"

namespace tsf {

constexpr int kBandFactorThreads = 256;

size_t band_factor_smem(int n1) {
    const int B = n1 + 2, bw = B - 1;
    return (size_t)B * B * sizeof(float) + (size_t)B * sizeof(float) + (size_t)bw * (bw + 1) / 2 * sizeof(uint16_t);
}

// S coupling of node g = (p, q) to node h <= g (both in [0, nm)), FP32
// stencil planes.  The four lower neighbours are stored at h: W = E(h),
// SE = NW(h), S = N(h), SW = NE(h).  For n1 = 2 the W and SE offsets coincide
// (d = 1), told apart by p.
__device__ __forceinline__ float band_entry(const float* S, size_t pl, int n1, int g, int h) {
    const int d = g - h;
    const int p = g % n1;
    if (d == 0) return S[g];
    float v = 0.f;
    if (d == 1 && p > 0) v = S[pl + h];                       // west
    if (d == n1 - 1 && p + 1 < n1) v = S[4 * pl + h];          // south-east
    if (d == n1) v = S[2 * pl + h];                            // south
    if (d == n1 + 1 && p > 0) v = S[3 * pl + h];               // south-west
    return v;
}

__global__ void __launch_bounds__(kBandFactorThreads) k_band_factor(BandArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int n1 = a.n1, nm = a.nm, B = n1 + 2, bw = B - 1;
    float* W = reinterpret_cast<float*>(smem);        // [B][B], row = slot of the larger index
    float* col = W + B * B;                           // [B]
    uint16_t* pairs = reinterpret_cast<uint16_t*>(col + B);
    const int npairs = bw * (bw + 1) / 2;
    const int i = blockIdx.x, tid = threadIdx.x, T = blockDim.x;
    const size_t pl = (size_t)a.nmp;
    const float* S = a.S32 + (size_t)i * kPlanes * pl;
    float* L = a.L + (size_t)i * nm * B;
    // (t, s) pairs of the rank-1 update, 1 <= s <= t <= bw
    for (int idx = tid; idx < npairs; idx += T) {
        int t = (int)((sqrtf(8.f * idx + 1.f) - 1.f) * 0.5f);
        while ((t + 1) * (t + 2) / 2 <= idx) ++t;
        while (t * (t + 1) / 2 > idx) --t;
        const int s = idx - t * (t + 1) / 2;          // 0 <= s <= t
        pairs[idx] = (uint16_t)(((t + 1) << 8) | (s + 1));
    }
    // initial window: rows 0..bw
    for (int e = tid; e < B * B; e += T) {
        const int g = e / B, h = e % B;
        W[e] = (g < nm && h <= g) ? band_entry(S, pl, n1, g, h) : 0.f;
    }
    __syncthreads();
    bool bad = false;
    for (int k = 0; k < nm; ++k) {
        const int base = k % B;
        // finished column k
        if (tid < B) {
            const float d = W[base * B + base];
            const float r = 1.0f / sqrtf(d);
            if (!(d > 0.f)) bad = true;
            const int t = tid;
            float v;
            if (t == 0) {
                v = r;
                col[0] = 0.f;
            } else {
                int st = base + t;
                st -= st >= B ? B : 0;
                v = (k + t < nm) ? W[st * B + base] * r : 0.f;
                col[t] = v;
            }
            L[(size_t)k * B + t] = v;
        }
        __syncthreads();
        // rank-1 update of the trailing window, and the entering row j = k + B
        for (int idx = tid; idx < npairs; idx += T) {
            const int pr = pairs[idx];
            const int t = pr >> 8, s = pr & 0xff;
            if (k + t >= nm) continue;
            int rt = base + t, cs = base + s;
            rt -= rt >= B ? B : 0;
            cs -= cs >= B ? B : 0;
            W[rt * B + cs] = fmaf(-col[t], col[s], W[rt * B + cs]);
        }
        const int j = k + B;
        if (j < nm) {
            for (int o = tid; o < B; o += T) {
                const int h = k + 1 + o;              // columns k+1 .. j of the new row
                int sh = base + 1 + o;
                sh -= sh >= B ? B : 0;
                W[base * B + sh] = band_entry(S, pl, n1, j, h);
            }
        }
        __syncthreads();
    }
    if (bad) atomicOr(a.flag, 1);
}

// ---------------------------------------------------------------------------
// triangular solves: z = L^-T L^-1 r (FP32), x += z (FP64), for the open
// right-hand sides of each problem; one warp per problem
// ---------------------------------------------------------------------------
// Columns are prefetched kBandAhead steps ahead through a register ring, so
// that a warp keeps several column loads in flight (the solve streams the
// factor and is meant to run at HBM speed).
constexpr int kBandAhead = 4;

template <int NR>
__global__ void __launch_bounds__(256) k_band_solve(BandSolveArgs a) {
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= a.nM) return;
    bool open[NR];
    bool any = false;
#pragma unroll
    for (int t = 0; t < NR; ++t) {
        open[t] = !a.done[t][i];
        any = any || open[t];
    }
    if (!any) return;
    const int n1 = a.n1, nm = a.nm, B = n1 + 2, bw = B - 1;
    const size_t pl = (size_t)a.nmp, base = (size_t)i * pl;
    const float* L = a.L + (size_t)i * nm * B;
    float* y[NR];
#pragma unroll
    for (int t = 0; t < NR; ++t) y[t] = a.y[t] + base;
    const bool has1 = lane + 32 <= bw, has2 = lane + 64 <= bw;
    auto load_col = [&](int k, float& c0, float& c1, float& c2) {
        if (k < 0 || k >= nm) {
            c0 = c1 = c2 = 0.f;
            return;
        }
        const float* c = L + (size_t)k * B;
        c0 = (lane < B) ? c[lane] : 0.f;
        c1 = (lane + 32 < B) ? c[lane + 32] : 0.f;
        c2 = (lane + 64 < B) ? c[lane + 64] : 0.f;
    };
    float qa[kBandAhead], qb[kBandAhead], qc[kBandAhead];

    // ---- forward: L y = r; P[m] = pending value of index k + m, m = lane, lane+32, lane+64
    float p0[NR], p1[NR], p2[NR];
#pragma unroll
    for (int t = 0; t < NR; ++t) {
        const double* r = a.r[t] + base;
        p0[t] = (lane <= bw && lane < nm) ? (float)r[lane] : 0.f;
        p1[t] = (has1 && lane + 32 < nm) ? (float)r[lane + 32] : 0.f;
        p2[t] = (has2 && lane + 64 < nm) ? (float)r[lane + 64] : 0.f;
    }
    float ybuf[NR], ent[NR];
#pragma unroll
    for (int t = 0; t < NR; ++t) ybuf[t] = ent[t] = 0.f;
#pragma unroll
    for (int u = 0; u < kBandAhead; ++u) load_col(u, qa[u], qb[u], qc[u]);
    for (int kb = 0; kb < nm; kb += kBandAhead) {
#pragma unroll
        for (int u = 0; u < kBandAhead; ++u) {
            const int k = kb + u;
            if (k >= nm) break;
            if ((k & 31) == 0) {
                // entering values r[k' + 1 + bw] of the 32 steps k' = k .. k + 31 (lane l: step k + l)
#pragma unroll
                for (int t = 0; t < NR; ++t) {
                    const int e = k + lane + 1 + bw;
                    ent[t] = e < nm ? (float)a.r[t][base + e] : 0.f;
                }
            }
            const float c0 = qa[u], c1 = qb[u], c2 = qc[u];
            load_col(k + kBandAhead, qa[u], qb[u], qc[u]);
            const float inv = __shfl_sync(0xffffffffu, c0, 0);
#pragma unroll
            for (int t = 0; t < NR; ++t) {
                const float yk = __shfl_sync(0xffffffffu, p0[t], 0) * inv;
                if ((k & 31) == lane) ybuf[t] = yk;
                const float a0 = lane >= 1 ? fmaf(-c0, yk, p0[t]) : p0[t];
                const float a1 = fmaf(-c1, yk, p1[t]);
                const float a2 = fmaf(-c2, yk, p2[t]);
                // shift down: P'[m] = P[m + 1]; the entering value goes to slot bw
                float n0 = __shfl_down_sync(0xffffffffu, a0, 1);
                const float b1 = __shfl_sync(0xffffffffu, a1, 0);
                float nn1 = __shfl_down_sync(0xffffffffu, a1, 1);
                const float b2 = __shfl_sync(0xffffffffu, a2, 0);
                float nn2 = __shfl_down_sync(0xffffffffu, a2, 1);
                if (lane == 31) {
                    n0 = b1;
                    nn1 = b2;
                    nn2 = 0.f;
                }
                const float e = __shfl_sync(0xffffffffu, ent[t], k & 31);
                if (lane == bw) n0 = e;
                if (lane + 32 == bw) nn1 = e;
                if (lane + 64 == bw) nn2 = e;
                p0[t] = n0;
                p1[t] = nn1;
                p2[t] = nn2;
            }
            if ((k & 31) == 31 || k == nm - 1) {
                const int k0 = k & ~31;
#pragma unroll
                for (int t = 0; t < NR; ++t)
                    if (k0 + lane <= k) y[t][k0 + lane] = ybuf[t];
            }
        }
    }
    __syncwarp();

    // ---- backward: L^T x = y; X[m] = x_{k+m}, m = lane, lane+32, lane+64 (X[0] unused)
    float x0[NR], x1[NR], x2[NR], yc[NR], xbuf[NR];
#pragma unroll
    for (int t = 0; t < NR; ++t) x0[t] = x1[t] = x2[t] = yc[t] = xbuf[t] = 0.f;
#pragma unroll
    for (int u = 0; u < kBandAhead; ++u) load_col(nm - 1 - u, qa[u], qb[u], qc[u]);
    for (int kb = nm - 1; kb >= 0; kb -= kBandAhead) {
#pragma unroll
        for (int u = 0; u < kBandAhead; ++u) {
            const int k = kb - u;
            if (k < 0) break;
            if (k == nm - 1 || (k & 31) == 31) {
                const int k0 = k & ~31;
#pragma unroll
                for (int t = 0; t < NR; ++t) yc[t] = (k0 + lane <= k) ? y[t][k0 + lane] : 0.f;
            }
            const float c0 = qa[u], c1 = qb[u], c2 = qc[u];
            load_col(k - kBandAhead, qa[u], qb[u], qc[u]);
            const float inv = __shfl_sync(0xffffffffu, c0, 0);
#pragma unroll
            for (int t = 0; t < NR; ++t) {
                float part = (lane >= 1 ? c0 * x0[t] : 0.f) + c1 * x1[t] + c2 * x2[t];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
                const float xk = (__shfl_sync(0xffffffffu, yc[t], k & 31) - part) * inv;
                if ((k & 31) == lane) xbuf[t] = xk;
                // shift up: X'[m] = X[m - 1], X'[1] = x_k
                if (lane == 0) x0[t] = xk;
                const float t31a = __shfl_sync(0xffffffffu, x0[t], 31);
                const float t31b = __shfl_sync(0xffffffffu, x1[t], 31);
                float n0 = __shfl_up_sync(0xffffffffu, x0[t], 1);
                float nn1 = __shfl_up_sync(0xffffffffu, x1[t], 1);
                float nn2 = __shfl_up_sync(0xffffffffu, x2[t], 1);
                if (lane == 0) {
                    n0 = 0.f;
                    nn1 = t31a;
                    nn2 = t31b;
                }
                x0[t] = (lane <= bw) ? n0 : 0.f;
                x1[t] = has1 ? nn1 : 0.f;
                x2[t] = has2 ? nn2 : 0.f;
            }
            if ((k & 31) == 0) {
#pragma unroll
                for (int t = 0; t < NR; ++t) {
                    const int g = k + lane;
                    if (open[t] && g < nm) a.x[t][base + g] += (double)xbuf[t];
                }
            }
        }
    }
}

// r = c - S x (FP64) for the open right-hand sides; convergence per problem
__global__ void __launch_bounds__(256) k_band_residual(BandResidualArgs a) {
    __shared__ double buf[3 * 32];
    const int i = blockIdx.x, n1 = a.n1;
    const size_t pl = (size_t)a.nmp, base = (size_t)i * pl;
    const double* S = a.S64 + (size_t)i * kPlanes * pl;
    bool open[3];
    for (int t = 0; t < 3; ++t) open[t] = t < a.nrhs && !a.done[t][i];
    if (!open[0] && !open[1] && !open[2]) return;     // block-uniform
    double rr[3] = {0.0, 0.0, 0.0};
    for (int j = threadIdx.x; j < a.nm; j += blockDim.x) {
        const int p = j % n1, q = j / n1;
        for (int t = 0; t < 3; ++t) {
            if (!open[t]) continue;
            const double r = a.c[t][base + j] - plane_apply(S, pl, a.x[t] + base, j, p, q, n1);
            a.r[t][base + j] = r;
            rr[t] = fma(r, r, rr[t]);
        }
    }
    block_allreduce<double, 3>(rr, buf);
    if (threadIdx.x == 0) {
        int open_after = 0;
        for (int t = 0; t < 3; ++t) {
            if (!open[t]) continue;
            const double bn = a.bnorm[t][(size_t)i * 3];
            const bool conv = rr[t] <= a.tol * a.tol * bn;
            if (!(rr[t] == rr[t])) set_status(a.ctl, kNaN);
            if (conv) a.done[t][i] = 1;
            else ++open_after;
        }
        if (open_after) atomicAdd(a.open_count, open_after);
        atomicAdd(&a.ctl->sweeps, 1ull);
    }
}

cudaError_t launch_band_factor(const BandArgs& a, cudaStream_t s) {
    const size_t sm = band_factor_smem(a.n1);
    cudaError_t e = cudaFuncSetAttribute(k_band_factor, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_band_factor<<<a.nM, kBandFactorThreads, sm, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_band_solve(const BandSolveArgs& a, int nrhs, cudaStream_t s) {
    const unsigned grid = (unsigned)((a.nM + 7) / 8);
    switch (nrhs) {
        case 1: k_band_solve<1><<<grid, 256, 0, s>>>(a); break;
        case 2: k_band_solve<2><<<grid, 256, 0, s>>>(a); break;
        case 3: k_band_solve<3><<<grid, 256, 0, s>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_band_residual(const BandResidualArgs& a, cudaStream_t s) {
    k_band_residual<<<a.nM, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace tsf
