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
// k_band_factor: one block per micro problem, right-looking band Cholesky in
// panels of four columns on a sliding window of the trailing matrix in shared
// memory (circular row/column slots); finished columns leave the window, the
// next rows of S (their five stored couplings, staged ahead with cp.async)
// enter it.
// k_band_solve: one warp per micro problem: forward substitution with the
// pending right-hand side values spread over the lanes (3 slots a lane),
// backward substitution as one warp dot product per column.
// k_band_residual: r = c - S x in FP64 for the right-hand sides still open,
// and the per-problem convergence test ||r|| <= tol ||c||.
#include "tsf_internal.cuh"

namespace tsf {

constexpr int kBandFactorThreads = 128;  // four warps per micro problem

// Staging of the stencil values of the rows that enter the window: chunk c
// (columns 32c .. 32c+31) brings rows j = BW + 32c .. BW + 32c + 31 (BW the
// window size), whose couplings sit at node indices lo = j0 - n1 - 1 ..
// j0 + 31: n1 + 33 values per plane, two chunks in flight (cp.async, loaded
// one chunk ahead).
__host__ __device__ __forceinline__ int band_stage_len(int n1) { return n1 + 33; }

constexpr int kBandPanel = 4;                // columns per panel of the factorisation
constexpr int kPanelVec = kBandPanel / 4;    // float4 per row of panel values

size_t band_factor_smem(int n1) {
    const int BW = n1 + 2 + kBandPanel - 1;  // window of the panel factorisation
    size_t b = (size_t)BW * kPanelVec * sizeof(float4) + (size_t)BW * BW * sizeof(float);
    b = (b + 15) & ~(size_t)15;
    return b + 2 * (size_t)kPlanes * band_stage_len(n1) * sizeof(float);
}

__device__ __forceinline__ void cp_async4(float* smem, const float* gmem, bool valid) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    const int n = valid ? 4 : 0;                        // 0: zero-fill, nothing read
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sa), "l"(gmem), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

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

// band_entry on staged plane values: st = one chunk's [kPlanes][len] values
// starting at node index lo
__device__ __forceinline__ float band_entry_staged(const float* st, int len, int lo, int n1, int g, int h) {
    const int d = g - h;
    const int p = g % n1;
    if (d == 0) return st[g - lo];
    float v = 0.f;
    if (d == 1 && p > 0) v = st[len + h - lo];                     // west: E(h)
    if (d == n1 - 1 && p + 1 < n1) v = st[4 * len + h - lo];       // south-east: NW(h)
    if (d == n1) v = st[2 * len + h - lo];                         // south: N(h)
    if (d == n1 + 1 && p > 0) v = st[3 * len + h - lo];            // south-west: NE(h)
    return v;
}

// One block of kBandFactorThreads per micro problem, panels of kBandPanel
// columns.  The window holds BW = B + kBandPanel - 1 consecutive rows in
// circular slots (slot(g) = g mod BW), lower half valid.  Per panel: the
// kBandPanel columns are finished one after the other (each first takes the
// updates of the earlier columns of the panel), then ONE rank-kBandPanel
// update of the trailing square, then the kBandPanel rows that follow the
// window enter it.  In the rank update lane l of every warp owns the columns
// s = l + 32 g (g < NG) of the trailing square and walks its warp's share of
// the rows; a row's kBandPanel factor values are kPanelVec broadcast float4,
// so a window element is loaded and stored once per kBandPanel columns.  The upper
// half of the square is updated as well (it is never read, and holds finite
// values), so the update needs no predicate.

template <int NG>
__global__ void __launch_bounds__(kBandFactorThreads) k_band_factor(BandArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int n1 = a.n1, nm = a.nm, B = n1 + 2, bw = B - 1;
    const int BW = B + kBandPanel - 1;
    float4* Lp = reinterpret_cast<float4*>(smem);                 // [BW][kPanelVec] panel columns by row slot
    float* W = reinterpret_cast<float*>(Lp + BW * kPanelVec);     // [BW][BW]
    size_t off = (size_t)BW * kPanelVec * sizeof(float4) + (size_t)BW * BW * sizeof(float);
    off = (off + 15) & ~(size_t)15;
    const int slen = band_stage_len(n1);
    float* stage = reinterpret_cast<float*>(smem + off);         // [2][kPlanes][slen]
    const int i = blockIdx.x, tid = threadIdx.x, T = blockDim.x, lane = tid & 31, warp = tid >> 5;
    const int nw = T >> 5;
    const size_t pl = (size_t)a.nmp;
    const float* S = a.S32 + (size_t)i * kPlanes * pl;
    float* L = a.L + (size_t)i * nm * B;
    // this warp's rows q in [q0, q1) of the trailing square (q = 0 .. bw-1)
    const int per = (bw + nw - 1) / nw;
    const int q0 = warp * per, q1 = min(bw, q0 + per);
    auto slot = [&](int g) { return g % BW; };
    // chunk c of entering rows (j = BW + 32c .. BW + 32c + 31) into stage buffer c & 1
    auto issue_chunk = [&](int c) {
        const int lo = BW + 32 * c - n1 - 1;
        float* st = stage + (c & 1) * kPlanes * slen;
        for (int e = tid; e < kPlanes * slen; e += T) {
            const int plane = e / slen, idx = lo + e % slen;
            const bool ok = idx >= 0 && idx < nm;
            cp_async4(st + e, S + plane * pl + (ok ? idx : 0), ok);
        }
        cp_async_commit();
    };
    issue_chunk(0);
    // initial window: rows 0..BW-1
    for (int e = tid; e < BW * BW; e += T) {
        const int g = e / BW, h = e % BW;
        W[e] = (g < nm && h <= g && g - h <= bw) ? band_entry(S, pl, n1, g, h) : 0.f;
    }
    bool bad = false;
    auto wrap = [&](int x) { return x >= BW ? x - BW : x; };     // x < 2 BW
    for (int k = 0; k < nm; k += kBandPanel) {
        if ((k & 31) == 0) {
            // the chunk of this panel's entering rows is complete; fetch the next one
            cp_async_wait_all();
            __syncthreads();
            issue_chunk((k >> 5) + 1);
        }
        const int sk0 = k % BW;                                   // slot of row k
        // ---- warp 0 finishes the panel's columns, one after the other
        if (warp == 0) {
            for (int e = lane; e < BW * kPanelVec; e += 32) Lp[e] = make_float4(0.f, 0.f, 0.f, 0.f);
            __syncwarp();
            for (int c = 0; c < kBandPanel; ++c) {
                const int kc = k + c;
                if (kc >= nm) break;
                const int sk = wrap(sk0 + c);
                const float* lkc = reinterpret_cast<const float*>(&Lp[sk * kPanelVec]);
                float wv[3];
                int sgv[3];
#pragma unroll
                for (int u = 0; u < 3; ++u) {
                    const int t = lane + 32 * u, g = kc + t;
                    const int sg = wrap(sk + t < 2 * BW ? sk + t : sk + t - BW);
                    sgv[u] = sg;
                    float w = 0.f;
                    if (t < BW - c && t <= bw && g < nm) {
                        const float* lgc = reinterpret_cast<const float*>(&Lp[sg * kPanelVec]);
                        w = W[sg * BW + sk];
#pragma unroll
                        for (int cp = 0; cp < kBandPanel; ++cp)
                            if (cp < c) w = fmaf(-lgc[cp], lkc[cp], w);
                    }
                    wv[u] = w;
                }
                const float d = __shfl_sync(0xffffffffu, wv[0], 0);
                const float r = rsqrtf(d);
                if (!(d > 0.f)) bad = true;
                __syncwarp();                                     // every lane has read Lp
#pragma unroll
                for (int u = 0; u < 3; ++u) {
                    const int t = lane + 32 * u, g = kc + t;
                    if (t < BW - c) {
                        const float v = (t <= bw && g < nm) ? wv[u] * r : 0.f;
                        reinterpret_cast<float*>(&Lp[sgv[u] * kPanelVec])[c] = v;
                        if (t == 0) L[(size_t)kc * B] = r;
                        else if (t <= bw) L[(size_t)kc * B + t] = v;
                    }
                }
                __syncwarp();
            }
        }
        __syncthreads();
        // ---- rank-kBandPanel update of the trailing square, rows/columns k+P .. k+BW-1
        {
            const int base = wrap(sk0 + kBandPanel);
            float4 cv[NG][kPanelVec];
            float* Wc[NG];
#pragma unroll
            for (int gi = 0; gi < NG; ++gi) {
                const int s = 32 * gi + lane;
                const bool mine = s < bw;
                const int cs = mine ? wrap(base + s) : sk0;      // sk0: a retired row, zero multiplier
#pragma unroll
                for (int h = 0; h < kPanelVec; ++h)
                    cv[gi][h] = mine ? Lp[cs * kPanelVec + h] : make_float4(0.f, 0.f, 0.f, 0.f);
                Wc[gi] = W + cs;
            }
            auto rows = [&](int r0, int r1) {
                for (int rr = r0; rr < r1; ++rr) {
                    float4 lr[kPanelVec];
#pragma unroll
                    for (int h = 0; h < kPanelVec; ++h) lr[h] = Lp[rr * kPanelVec + h];
#pragma unroll
                    for (int gi = 0; gi < NG; ++gi) {
                        float w = Wc[gi][rr * BW];
#pragma unroll
                        for (int h = 0; h < kPanelVec; ++h) {
                            w = fmaf(-lr[h].x, cv[gi][h].x, w);
                            w = fmaf(-lr[h].y, cv[gi][h].y, w);
                            w = fmaf(-lr[h].z, cv[gi][h].z, w);
                            w = fmaf(-lr[h].w, cv[gi][h].w, w);
                        }
                        Wc[gi][rr * BW] = w;
                    }
                }
            };
            if (q0 < q1) {
                const int r0 = wrap(base + q0);
                const int len = q1 - q0;
                if (r0 + len <= BW) {
                    rows(r0, r0 + len);
                } else {
                    rows(r0, BW);
                    rows(0, r0 + len - BW);
                }
            }
        }
        // ---- meanwhile the rows j = k + BW + m take the retired slots of the
        // panel rows (rows the update does not touch; it only passes through
        // their columns with zero multipliers)
        if (tid < BW) {
            const float* st = stage + ((k >> 5) & 1) * kPlanes * slen;
            const int lo = BW + 32 * (k >> 5) - n1 - 1;
#pragma unroll
            for (int m = 0; m < kBandPanel; ++m) {
                const int j = k + BW + m;
                if (j < nm) {
                    const int h = k + m + 1 + tid;               // columns j-BW+1 .. j of the new row
                    int sh = sk0 + m + 1 + tid;
                    sh = sh >= 2 * BW ? sh - 2 * BW : (sh >= BW ? sh - BW : sh);
                    W[wrap(sk0 + m) * BW + sh] = band_entry_staged(st, slen, lo, n1, j, h);
                }
            }
        }
        __syncthreads();
    }
    cp_async_wait_all();
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

constexpr int kBandSolveThreads = 64;   // two problems per block: fine-grained balance over the SMs

// NR right-hand sides per warp, one pass over the factor for all of them
// (one warp per right-hand side reads the factor NR times and was slower).
template <int NR>
__global__ void __launch_bounds__(kBandSolveThreads) k_band_solve(BandSolveArgs a) {
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= a.nM) return;
    const int n1 = a.n1, nm = a.nm, B = n1 + 2, bw = B - 1;
    const size_t pl = (size_t)a.nmp, base = (size_t)i * pl;
    const double* rp[NR];
    double* xp[NR];
    float* y[NR];
    bool open[NR];
    bool any = false;
#pragma unroll
    for (int t = 0; t < NR; ++t) {
        rp[t] = a.r[t] + base;
        xp[t] = a.x[t] + base;
        y[t] = a.y[t] + base;
        open[t] = !a.done[t][i];
        any = any || open[t];
    }
    if (!any) return;
    const float* L = a.L + (size_t)i * nm * B;
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
        const double* r = rp[t];
        p0[t] = (lane <= bw && lane < nm) ? (float)r[lane] : 0.f;
        p1[t] = (has1 && lane + 32 < nm) ? (float)r[lane + 32] : 0.f;
        p2[t] = (has2 && lane + 64 < nm) ? (float)r[lane + 64] : 0.f;
    }
    float ybuf[NR], ent[NR], ent_next[NR];
    // entering values r[k' + 1 + bw] of the 32 steps k' = c0 .. c0 + 31 (lane l: step c0 + l)
    auto load_ent = [&](int c0, float (&dst)[NR]) {
#pragma unroll
        for (int t = 0; t < NR; ++t) {
            const int e = c0 + lane + 1 + bw;
            dst[t] = e < nm ? (float)rp[t][e] : 0.f;
        }
    };
#pragma unroll
    for (int t = 0; t < NR; ++t) ybuf[t] = 0.f;
    load_ent(0, ent_next);
#pragma unroll
    for (int u = 0; u < kBandAhead; ++u) load_col(u, qa[u], qb[u], qc[u]);
    for (int kb = 0; kb < nm; kb += kBandAhead) {
#pragma unroll
        for (int u = 0; u < kBandAhead; ++u) {
            const int k = kb + u;
            if (k >= nm) break;
            if ((k & 31) == 0) {
                // this chunk's entering values were fetched one chunk ahead
#pragma unroll
                for (int t = 0; t < NR; ++t) ent[t] = ent_next[t];
                load_ent(k + 32, ent_next);
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
    float x0[NR], x1[NR], x2[NR], yc[NR], ynext[NR], xbuf[NR];
    // y of the 32-step chunk [k0, k0 + 31] (lane l: index k0 + l), fetched one chunk ahead
    auto load_y = [&](int k0, float (&dst)[NR]) {
#pragma unroll
        for (int t = 0; t < NR; ++t) dst[t] = (k0 >= 0 && k0 + lane < nm) ? y[t][k0 + lane] : 0.f;
    };
#pragma unroll
    for (int t = 0; t < NR; ++t) x0[t] = x1[t] = x2[t] = yc[t] = xbuf[t] = 0.f;
    load_y((nm - 1) & ~31, ynext);
#pragma unroll
    for (int u = 0; u < kBandAhead; ++u) load_col(nm - 1 - u, qa[u], qb[u], qc[u]);
    for (int kb = nm - 1; kb >= 0; kb -= kBandAhead) {
#pragma unroll
        for (int u = 0; u < kBandAhead; ++u) {
            const int k = kb - u;
            if (k < 0) break;
            if (k == nm - 1 || (k & 31) == 31) {
#pragma unroll
                for (int t = 0; t < NR; ++t) yc[t] = ynext[t];
                load_y((k & ~31) - 32, ynext);
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
                    if (open[t] && g < nm) xp[t][g] += (double)xbuf[t];
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
    const int ng = (a.n1 + 1 + 31) / 32;          // column groups of the half-bandwidth n1 + 1
    cudaError_t e = cudaSuccess;
    switch (ng) {
        case 1:
            e = cudaFuncSetAttribute(k_band_factor<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            if (e == cudaSuccess) k_band_factor<1><<<a.nM, kBandFactorThreads, sm, s>>>(a);
            break;
        case 2:
            e = cudaFuncSetAttribute(k_band_factor<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            if (e == cudaSuccess) k_band_factor<2><<<a.nM, kBandFactorThreads, sm, s>>>(a);
            break;
        case 3:
            e = cudaFuncSetAttribute(k_band_factor<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            if (e == cudaSuccess) k_band_factor<3><<<a.nM, kBandFactorThreads, sm, s>>>(a);
            break;
        default:
            return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_band_solve(const BandSolveArgs& a, int nrhs, cudaStream_t s) {
    const int per_block = kBandSolveThreads / 32;
    const unsigned grid = (unsigned)((a.nM + per_block - 1) / per_block);
    switch (nrhs) {
        case 1: k_band_solve<1><<<grid, kBandSolveThreads, 0, s>>>(a); break;
        case 2: k_band_solve<2><<<grid, kBandSolveThreads, 0, s>>>(a); break;
        case 3: k_band_solve<3><<<grid, kBandSolveThreads, 0, s>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_band_residual(const BandResidualArgs& a, cudaStream_t s) {
    k_band_residual<<<a.nM, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace tsf
