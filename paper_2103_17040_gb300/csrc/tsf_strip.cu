// tsf_strip.cu -- the column-strip micro solves (mixed precision), the hot
// kernels of the two-scale step.
//
// Every micro problem i (one per macro node, Sec. 3.3) solves
//     S_i v_i = b_i,      S_i = M_i/dt + A_i + kappa R_i     (Eq. (17), micro rows)
// by FP64-accurate iterative refinement around FP32 Jacobi-preconditioned CG
// (Sec. 3.5: CG for every system, the systems distributed over the
// processors; here one thread block per system).
//
// Thread t of a block owns R consecutive nodes of one column of the micro
// grid: p = t mod n1, rows q0 .. q0+R-1 with q0 = R (t div n1).
//
// The inner CG runs on the symmetrically Jacobi-scaled operator
//     S^ = D^-1/2 S D^-1/2      (unit diagonal, D = diag(S)),
// whose eight off-diagonal couplings per node are precomputed once per
// (geometry, dt) by k_strip_setup and loaded with two 16-byte loads per node
// (registers for short strips, shared memory for tall ones).  The vector the
// operator is applied to reaches the neighbours through one zero-haloed
// shared-memory plane.  The CG is the Chronopoulos-Gear form: one operator
// application and ONE fused two-value reduction per iteration.
//
// GB300 executes FP64 arithmetic, and conversions from FP64 to FP32, at
// about 1/70 of its FP32 rate, so the refinement works in float-float
// ("double-float") arithmetic: values are unevaluated pairs hi + lo of FP32
// numbers, added with Knuth's TwoSum and multiplied with an FMA-based
// TwoProduct, which carries them to about 2^-44 relative.  The refinement
// residual is such a pair; each sweep forms
//     S d = D^1/2 (S^ y),   d = D^-1/2 y
// from the FP32 correction y of the inner solve, with S^ and D^+-1/2 stored
// as FP32 pairs (about 2^-48), and subtracts it from the residual pair.
//
// Two instantiations:
//  * PIPE = false: the stored residual and the solution are FP64 arrays
//    (res, v), converted to and from float-float once per solve.  Used for the
//    partitioned iteration, the unpipelined elimination, and the one-off
//    solves for phi and psi.
//  * PIPE = true: the pipelined exact elimination (tsf_elim.cu).  Every array
//    of the pipeline is a float pair (8 bytes, like FP64): the warm start, the
//    u-independent part of its residual, M w/dt, M psi/dt and the two history
//    rings of w and S w.  The kernel then executes no FP64 instruction except
//    the flux sum over the Robin edge; its epilogue prepares the next solve.
//
// Norms: the stopping test compares FP32 sums of squares of the residual
// scaled by a per-problem power of two (exact), so the relative tolerance
// has no FP32 range limit.
#include "tsf_internal.cuh"

#include <cooperative_groups.h>

namespace tsf {

namespace cg = cooperative_groups;

// ---------------------------------------------------------------------------
// float-float arithmetic.  The round-to-nearest intrinsics keep the compiler
// from contracting the error-free steps into FMAs.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// renormalise s + e (|e| small against s, or s == 0)
__device__ __forceinline__ float2 fast_two_sum_f(float s, float e) {
    const float h = __fadd_rn(s, e);
    return make_float2(h, __fsub_rn(e, __fsub_rn(h, s)));
}
__device__ __forceinline__ float2 ff_add(float2 a, float2 b) {
    float s, e;
    two_sum_f(a.x, b.x, s, e);
    e = __fadd_rn(e, __fadd_rn(a.y, b.y));
    return fast_two_sum_f(s, e);
}
__device__ __forceinline__ float2 ff_neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 ff_sub(float2 a, float2 b) { return ff_add(a, ff_neg(b)); }
// (ah + al) (bh + bl)
__device__ __forceinline__ float2 ff_mul(float2 a, float2 b) {
    const float p = __fmul_rn(a.x, b.x);
    float e = fmaf(a.x, b.x, -p);
    e = fmaf(a.x, b.y, fmaf(a.y, b.x, e));
    return fast_two_sum_f(p, e);
}
// a * k for a small integer k (exact products of the parts up to rounding of k a.x)
__device__ __forceinline__ float2 ff_scale(float2 a, float k) {
    const float p = __fmul_rn(a.x, k);
    const float e = fmaf(a.x, k, -p);
    return fast_two_sum_f(p, fmaf(a.y, k, e));
}
// the pair nearest to an FP64 value (set-up and head kernels only: the
// FP64 -> FP32 conversions are slow on this part)
__device__ __forceinline__ float2 ff_from_double(double x) {
    const float h = __double2float_rn(x);
    return make_float2(h, __double2float_rn(x - (double)h));
}
__device__ __forceinline__ double ff_to_double(float2 a) { return (double)a.x + (double)a.y; }

// (s, c) += (ch + cl) x for an FP32 coupling pair and an FP32 x: TwoProduct
// of the high part, TwoSum into s, the small terms into c.
__device__ __forceinline__ void ff_acc(float& s, float& c, float ch, float cl, float x) {
    const float p = __fmul_rn(ch, x);
    const float e = fmaf(ch, x, -p);
    float t, err;
    two_sum_f(s, p, t, err);
    s = t;
    c = __fadd_rn(c, __fadd_rn(err, fmaf(cl, x, e)));
}
// (s, c) += (ch + cl) (xh + xl) for a coupling pair and a value pair
__device__ __forceinline__ void ff_acc2(float& s, float& c, float ch, float cl, float xh, float xl) {
    const float p = __fmul_rn(ch, xh);
    const float e = fmaf(ch, xh, -p);
    float t, err;
    two_sum_f(s, p, t, err);
    s = t;
    c = __fadd_rn(c, __fadd_rn(err, fmaf(ch, xl, fmaf(cl, xh, e))));
}

// ---------------------------------------------------------------------------
// Set-up per (geometry, dt): the scaled operator and the split mass planes.
// ---------------------------------------------------------------------------
// rs_j = 1 / sqrt(S_jj), FP64, one thread per padded node
__global__ void __launch_bounds__(256) k_strip_rsqrt(int nm, int nmp, int nM, const double* __restrict__ S64,
                                                     double* __restrict__ rs) {
    const int i = blockIdx.x;
    const int j = blockIdx.y * blockDim.x + threadIdx.x;
    if (j >= nmp) return;
    const size_t pl = (size_t)nmp;
    rs[(size_t)i * pl + j] = j < nm ? 1.0 / sqrt(S64[(size_t)i * kPlanes * pl + j]) : 0.0;
}

// chat / chatlo: the eight couplings of S^ at node j, (E, W, N, S) and
// (NE, NW, SE, SW), as FP32 pairs; dsc = (1/sqrt(S_jj), sqrt(S_jj)) as pairs;
// Mh + Ml = M/dt (five stored planes) when Mh is given.  Padding nodes get
// zeros everywhere.
__global__ void __launch_bounds__(256) k_strip_setup(StripSetupArgs a) {
    const int i = blockIdx.x;
    const int j = blockIdx.y * blockDim.x + threadIdx.x;
    if (j >= a.nmp) return;
    const int n1 = a.n1;
    const size_t pl = (size_t)a.nmp, io = (size_t)i * pl;
    const double* S = a.S64 + (size_t)i * kPlanes * pl;
    const double* rs = a.rs + io;
    float hi[8] = {0, 0, 0, 0, 0, 0, 0, 0}, lo[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    float4 d = make_float4(0.f, 0.f, 0.f, 0.f);
    if (j < a.nm) {
        const int p = j % n1, q = j / n1;
        const bool e = p + 1 < n1, w = p > 0, nd = q + 1 < n1, sd = q > 0;
        const double r0 = rs[j];
        double c[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        if (e) c[0] = S[pl + j] * r0 * rs[j + 1];
        if (w) c[1] = S[pl + j - 1] * r0 * rs[j - 1];
        if (nd) c[2] = S[2 * pl + j] * r0 * rs[j + n1];
        if (sd) c[3] = S[2 * pl + j - n1] * r0 * rs[j - n1];
        if (e && nd) c[4] = S[3 * pl + j] * r0 * rs[j + n1 + 1];
        if (w && nd) c[5] = S[4 * pl + j] * r0 * rs[j + n1 - 1];
        if (e && sd) c[6] = S[4 * pl + j - n1 + 1] * r0 * rs[j - n1 + 1];
        if (w && sd) c[7] = S[3 * pl + j - n1 - 1] * r0 * rs[j - n1 - 1];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const float2 f = ff_from_double(c[k]);
            hi[k] = f.x;
            lo[k] = f.y;
        }
        const float2 sc = ff_from_double(r0), dq = ff_from_double(sqrt(S[j]));
        d = make_float4(sc.x, sc.y, dq.x, dq.y);
    }
    float4* ch = a.chat + (size_t)i * 2 * pl;
    float4* cl = a.chatlo + (size_t)i * 2 * pl;
    ch[j] = make_float4(hi[0], hi[1], hi[2], hi[3]);
    ch[pl + j] = make_float4(hi[4], hi[5], hi[6], hi[7]);
    cl[j] = make_float4(lo[0], lo[1], lo[2], lo[3]);
    cl[pl + j] = make_float4(lo[4], lo[5], lo[6], lo[7]);
    a.dsc[io + j] = d;
    if (a.Mh) {
        const double* M = a.M64 + (size_t)i * kPlanes * pl;
        for (int c = 0; c < kPlanes; ++c) {
            const float2 f = j < a.nm ? ff_from_double(M[c * pl + j] * a.idt) : make_float2(0.f, 0.f);
            a.Mh[(size_t)i * kPlanes * pl + c * pl + j] = f.x;
            a.Ml[(size_t)i * kPlanes * pl + c * pl + j] = f.y;
        }
    }
}

cudaError_t launch_strip_setup(const StripSetupArgs& a, cudaStream_t s) {
    dim3 grid(a.nM, (a.nmp + 255) / 256);
    k_strip_rsqrt<<<grid, 256, 0, s>>>(a.nm, a.nmp, a.nM, a.S64, a.rs);
    k_strip_setup<<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

// out[k] = the float pair nearest to in[k]
__global__ void k_split_pairs(const double* __restrict__ in, float2* __restrict__ out, size_t n) {
    const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) out[k] = ff_from_double(in[k]);
}

cudaError_t launch_split_pairs(const double* in, float2* out, size_t n, cudaStream_t s) {
    k_split_pairs<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(in, out, n);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Strip geometry
// ---------------------------------------------------------------------------
// Launch bounds per strip height: R = 3 asks for two resident blocks of up to
// 384 threads, R = 5 and 7 for one block of 512 / 384; the tall strips (R = 9,
// 11, 13, couplings in shared memory) take up to 384 threads at
// kTallStripRegs registers.
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

__host__ __device__ inline int padded_nodes(int n1) { return (n1 * n1 + 31) / 32 * 32; }

// Shared memory of a strip block: one plane (two with the pipelined
// epilogue, which also moves the low parts of w), 4 x 32 float2 of
// reduction buffers and, with couplings in shared memory (sc), two float4 per
// node of the padded strip grid (n1 columns x strip_rows * R rows); with
// staging (pref) an mbarrier and copies of the low parts of the couplings and
// the diagonal scalings (48 bytes per padded node), and under the pipelined
// epilogue of M/dt (40 more).
__host__ __device__ inline size_t strip_smem_bytes(int n1, int R, bool sc, bool pipe, bool pref) {
    const size_t W = (size_t)strip_stride(n1, R), H = (size_t)strip_rows(n1, R) * R + 2;
    size_t off = ((pipe ? 2 : 1) * W * H * sizeof(float) + 15) & ~(size_t)15;
    off += 4 * 32 * sizeof(float2);
    if (pref) off += 16 + (size_t)padded_nodes(n1) * (48 + (pipe ? 40 : 0));
    if (sc) off += 2 * (size_t)n1 * strip_rows(n1, R) * R * sizeof(float4);
    return off;
}
// Staging is used where it still lets two blocks share an SM (228 KB of
// shared memory per SM, 1 KB of it reserved per block).
constexpr size_t kStageSmemLimit = 113 * 1024;
// An FP32 inner solve stops at kInnerMargin2 (squared norms) of the residual
// the outer tolerance asks for.  The rest of the gap covers the drift of the
// CG's recursively updated residual from the true one (a few FP32 ulps of
// the sweep's starting residual times the iteration count) and the rounding
// of the float-float update, both far smaller on the workloads' tolerances.
constexpr float kInnerMargin2 = 0.81f;
static bool strip_stages(int n1, int R, bool pipe) {
    return R < 9 && strip_smem_bytes(n1, R, false, pipe, true) <= kStageSmemLimit;
}

// The eight scaled off-diagonal couplings of one node.
struct Couple8 {
    float E, W, N, S, NE, NW, SE, SW;
};
__device__ __forceinline__ Couple8 couple8(float4 a, float4 b) { return Couple8{a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w}; }

// Where a strip's couplings live: in registers (short strips) ...
template <int R>
struct RegCouplings {
    Couple8 c[R];
    __device__ __forceinline__ Couple8 get(int k) const { return c[k]; }
};
// ... or in shared memory as two float4 per node, (E, W, N, S) and
// (NE, NW, SE, SW), node (p, q) at index p + n1 q of the padded strip grid
// (tall strips).  The loads are volatile so that the compiler re-reads the
// couplings at every operator application instead of hoisting them into
// registers.
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
    __device__ __forceinline__ Couple8 get(int k) const { return couple8(lds_f4(A + j0 + k * n1), lds_f4(B + j0 + k * n1)); }
};

// Neighbour values of a strip from a shared plane: L/Rt = columns p-1 / p+1
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

// y = S^ x reading the neighbour columns from the plane with a sliding
// window of three rows (fewer live registers than a loaded halo for tall
// strips).  The plane must hold x.  Entries of nodes outside the mesh are set
// to zero, so that they stay out of the dot products.
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

// Block-wide sums of two FP32 values: a butterfly inside each warp, the
// per-warp partials through shared memory, and a second butterfly over them
// in every warp (lanes past the last warp add zeros).  The summation order is
// fixed and the same in every warp, so all threads get the same, reproducible
// value.  buf (32 float2) must not be written again by the block before every
// thread has passed one more __syncthreads.
// Warp sums of two values with the values split across the half-warps: the
// first exchange leaves x in the lower and y in the upper sixteen lanes, so
// every further step moves one value instead of two.  Returns the total of x
// in lanes 0-15 and of y in lanes 16-31 (the same bits in every lane of a
// half: each butterfly step adds the same two operands on both sides).
__device__ __forceinline__ float warp_sum2_split(float x, float y) {
    const bool hi = (threadIdx.x & 16) != 0;
    float v = hi ? y : x;
    v += __shfl_xor_sync(0xffffffffu, hi ? x : y, 16);
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
// (x, y) = the totals of a split sum, in every lane
__device__ __forceinline__ void split_join(float v, float& x, float& y) {
    const float o = __shfl_xor_sync(0xffffffffu, v, 16);
    const bool hi = (threadIdx.x & 16) != 0;
    x = hi ? o : v;
    y = hi ? v : o;
}
// Sums of two values over nw <= 16 warps of 32 consecutive threads starting
// at a warp boundary: split warp sums, the partials through buf (lane 0 of
// each warp writes x, lane 16 y), the barrier `sync`, and a split sum of the
// nw partials in every warp -- a fixed order, so every thread gets the same
// bits.
template <class SYNC>
__device__ __forceinline__ void group_sum2_split(float& x, float& y, float2* buf, int warp, int nw, SYNC sync) {
    const int lane = threadIdx.x & 31;
    float v = warp_sum2_split(x, y);
    float* b = reinterpret_cast<float*>(buf);
    if ((lane & 15) == 0) b[2 * warp + (lane >> 4)] = v;
    sync();
    const int k = lane & 15;
    v = k < nw ? b[2 * k + (lane >> 4)] : 0.f;
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    split_join(v, x, y);
}

__device__ __forceinline__ void block_sum2(float& x, float& y, float2* buf) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (nw <= 16) {
        group_sum2_split(x, y, buf, warp, nw, [] { __syncthreads(); });
        return;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        x += __shfl_xor_sync(0xffffffffu, x, o);
        y += __shfl_xor_sync(0xffffffffu, y, o);
    }
    if (lane == 0) buf[warp] = make_float2(x, y);
    __syncthreads();
    const float2 t = lane < nw ? buf[lane] : make_float2(0.f, 0.f);
    x = t.x;
    y = t.y;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        x += __shfl_xor_sync(0xffffffffu, x, o);
        y += __shfl_xor_sync(0xffffffffu, y, o);
    }
}

// Block-wide maximum of a non-negative FP32 value (the bit patterns of
// non-negative floats order like their values).
__device__ __forceinline__ float block_max_nonneg(float x, float2* buf) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    unsigned m = __reduce_max_sync(0xffffffffu, __float_as_uint(x));
    if (lane == 0) buf[warp].x = __uint_as_float(m);
    __syncthreads();
    float r = 0.f;
    for (int k = 0; k < nw; ++k) r = fmaxf(r, buf[k].x);
    return r;
}

// Block-wide sums of two FP32 values and maximum of a third, non-negative one,
// with one barrier (same fixed summation order as block_sum2).  buf: 32 float4.
__device__ __forceinline__ void block_sum2_max(float& x, float& y, float& m, float4* buf) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        x += __shfl_xor_sync(0xffffffffu, x, o);
        y += __shfl_xor_sync(0xffffffffu, y, o);
    }
    const unsigned mb = __reduce_max_sync(0xffffffffu, __float_as_uint(m));
    if (lane == 0) buf[warp] = make_float4(x, y, __uint_as_float(mb), 0.f);
    __syncthreads();
    float sx = 0.f, sy = 0.f, mx = 0.f;
    for (int k = 0; k < nw; ++k) {
        const float4 t = buf[k];
        sx += t.x;
        sy += t.y;
        mx = fmaxf(mx, t.z);
    }
    x = sx;
    y = sy;
    m = mx;
}

// Who solves one micro problem: a whole thread block (BlockTeam), or one
// warp, several micro problems per block (WarpTeam, for micro meshes whose
// strips fit 32 threads).  A warp synchronises with __syncwarp and reduces
// with shuffles alone, so its CG iterations need no block barrier and no
// shared-memory partials.
struct BlockTeam {
    static constexpr bool kWarp = false;
    __device__ int thread() const { return threadIdx.x; }
    __device__ int size() const { return blockDim.x; }
    __device__ int slot() const { return 0; }  // team index within the block
    __device__ int problem() const { return blockIdx.x; }
    __device__ void sync() const { __syncthreads(); }
    __device__ bool all(bool ok) const { return __syncthreads_and(ok) != 0; }  // (also a barrier)
    __device__ void sum2(float& x, float& y, float2* buf) const { block_sum2(x, y, buf); }
    __device__ void sum2_max(float& x, float& y, float& m, float4* buf) const { block_sum2_max(x, y, m, buf); }
};
// A whole block on a given micro problem (the persistent batch kernel):
// BlockTeam's barriers and sums.
struct BlockTeamAt {
    static constexpr bool kWarp = false;
    int prob;
    __device__ int thread() const { return threadIdx.x; }
    __device__ int size() const { return blockDim.x; }
    __device__ int slot() const { return 0; }
    __device__ int problem() const { return prob; }
    __device__ void sync() const { __syncthreads(); }
    __device__ bool all(bool ok) const { return __syncthreads_and(ok) != 0; }
    __device__ void sum2(float& x, float& y, float2* buf) const { block_sum2(x, y, buf); }
    __device__ void sum2_max(float& x, float& y, float& m, float4* buf) const { block_sum2_max(x, y, m, buf); }
};
struct WarpTeam {
    static constexpr bool kWarp = true;
    __device__ int thread() const { return threadIdx.x & 31; }
    __device__ int size() const { return 32; }
    __device__ int slot() const { return threadIdx.x >> 5; }
    __device__ int problem() const { return blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); }
    __device__ void sync() const { __syncwarp(); }
    __device__ bool all(bool ok) const { return __all_sync(0xffffffffu, ok) != 0; }
    __device__ void sum2(float& x, float& y, float2*) const { split_join(warp_sum2_split(x, y), x, y); }
    __device__ void sum2_max(float& x, float& y, float& m, float4*) const {
        sum2(x, y, nullptr);
        m = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(m)));
    }
};

// Chronopoulos-Gear CG on the scaled operator (Jacobi-PCG on S); x = 0 on
// entry, r = rhs.  Stops when ||r||^2 <= rel2 ||r_0||^2 or after maxit
// iterations; returns the count.  redA/redB: 32-float2 reduction buffers.
template <int R, class CS, class TEAM = BlockTeam>
__device__ int strip_cg(const CS& c, const bool (&valid)[R], float (&x)[R], float (&r)[R], float* P, int Wd, int p,
                        int q0, float rel2, int maxit, float2* redA, float2* redB, int* flag, const TEAM& tm = TEAM()) {
    float pv[R], s[R], w[R];
    StripHalo<R> h;
    strip_store<R>(P, Wd, p, q0, valid, r);
    tm.sync();
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
    tm.sum2(g, dl, redA);
    const float stop = rel2 * g;
    if (!(dl > 0.f)) {
        *flag = (dl == dl) ? kBreakdown : kNaN;
        return 0;
    }
    // CG scalars with the fast division (a few ulp): they steer the FP32 inner
    // solve only, whose result is checked by the float-float residual
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
        tm.sync();
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
        tm.sum2(gn, dn, (it & 1) ? redB : redA);
        // (a NaN fails the test on den below; the refinement's residual norm reports it)
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

// ---------------------------------------------------------------------------
// Bulk asynchronous copies global -> shared memory (the TMA engine's
// non-tensor form), completed on an mbarrier.  Source and destination must be
// 16-byte aligned and the size a multiple of 16 bytes.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
    unsigned ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok)
                 : "r"(smem_u32(bar)), "r"(parity)
                 : "memory");
    return ok != 0;
}
// Bounded wait for phase 0 of the barrier, by every thread of the block; the
// result is the same in every thread.  Each try suspends the thread for a
// short while, so the bound is of the order of a second.
template <class TEAM>
__device__ __forceinline__ bool mbar_wait_team(unsigned long long* bar, const TEAM& tm) {
    bool ok = false;
    for (int k = 0; k < (1 << 22) && !ok; ++k) ok = mbar_try_wait(bar, 0);
    return tm.all(ok);
}
// the barrier object's memory can be initialised again (a persistent team
// stages the next problem through the same barrier)
__device__ __forceinline__ void mbar_inval(unsigned long long* bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// 2^e as an FP32 number, e clamped to the normal range
__device__ __forceinline__ float pow2f(int e) {
    e = max(-126, min(127, e));
    return __int_as_float((127 + e) << 23);
}

// FP64 power of two s with s sqrt(x) in [1, 2) (1 when x is not positive)
__device__ __forceinline__ double pow2_scale_of_norm2(double x) {
    if (!(x > 0.0) || !(x < 1e300)) return 1.0;
    int e;
    frexp(sqrt(x), &e);
    return ldexp(1.0, 1 - e);
}

template <int R, bool SC, bool PIPE, bool PREF, class TEAM = BlockTeam>
__device__ __forceinline__ void strip_body(const MicroArgs& a, const TEAM& tm = TEAM()) {
    static_assert(!(TEAM::kWarp && (PREF || SC)), "one-warp teams keep their couplings in registers, unstaged");
    extern __shared__ __align__(16) unsigned char smem_all[];
    const int n1 = a.n1, Wd = strip_stride(n1, R);
    // this team's part of the block's shared memory
    unsigned char* smem = smem_all + (size_t)tm.slot() * strip_smem_bytes(n1, R, SC, PIPE, PREF);
    const int Hd = strip_rows(n1, R) * R + 2, pw = Wd * Hd;
    const size_t pl = (size_t)a.nmp;
    float* P = reinterpret_cast<float*>(smem);
    float* P2 = P + pw;  // PIPE: the low parts of w in the epilogue
    size_t off = ((size_t)(PIPE ? 2 : 1) * pw * sizeof(float) + 15) & ~(size_t)15;
    float2* red = reinterpret_cast<float2*>(smem + off);  // 4 x 32 float2
    off += 4 * 32 * sizeof(float2);
    // PREF: the low parts of the couplings, the diagonal scalings and (PIPE)
    // M/dt, copied in by the bulk-copy engine while the CG runs
    unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem + off);
    const float4* sLo = reinterpret_cast<const float4*>(smem + off + 16);
    const float4* sDs = sLo + 2 * pl;
    const float* sMh = reinterpret_cast<const float*>(sDs + pl);
    const float* sMl = sMh + kPlanes * pl;
    if (PREF) off += 16 + pl * (48 + (PIPE ? 40 : 0));
    // SC: scaled couplings of the padded strip grid (n1 x strip_rows * R nodes)
    const int ncg = n1 * strip_rows(n1, R) * R;
    float4* cA = reinterpret_cast<float4*>(smem + off);
    float4* cB = cA + ncg;

    const int i = tm.problem(), tid = tm.thread(), T = tm.size();
    if (i >= a.nM) return;  // (one-warp teams: the warps past the last micro problem)
    const bool active = tid < n1 * strip_rows(n1, R);
    const int p = active ? tid % n1 : 0;
    const int q0 = active ? (tid / n1) * R : 0;
    const size_t io = (size_t)i * pl;
    bool staged = false, timed_out = false;
    if constexpr (PREF) {
        if (tid == 0) mbar_init(bar, 1);
        tm.sync();
        if (tid == 0) {
            const unsigned lo = (unsigned)(2 * pl * sizeof(float4)), ds = (unsigned)(pl * sizeof(float4));
            const unsigned mp = PIPE ? (unsigned)(kPlanes * pl * sizeof(float)) : 0u;
            mbar_expect_tx(bar, lo + ds + 2 * mp);
            bulk_copy_g2s((void*)sLo, a.chatlo + io * 2, lo, bar);
            bulk_copy_g2s((void*)sDs, a.dsc + io, ds, bar);
            if (PIPE) {
                bulk_copy_g2s((void*)sMh, a.Mh + io * kPlanes, mp, bar);
                bulk_copy_g2s((void*)sMl, a.Ml + io * kPlanes, mp, bar);
            }
        }
    }
    // every block waits for its copies once, before their first use or its exit
    auto wait_staged = [&]() {
        if (PREF && !staged) {
            staged = true;
            if (!mbar_wait_team(bar, tm)) {
                timed_out = true;
                mbar_wait_team(bar, tm);
            } else if (tid == 0) {
                mbar_inval(bar);  // (every thread is past its wait: the vote is a barrier)
            }
        }
    };
    const double* re = a.redge + (size_t)i * n1;
    const bool edge = p == n1 - 1;
    bool valid[R];
#pragma unroll
    for (int k = 0; k < R; ++k) valid[k] = active && (q0 + k) < n1;

    // ---- residual of the initial iterate as float pairs, ||b||, the scale ----
    float2 r[R];          // PIPE: unscaled; otherwise scaled by s64
    float s = 1.f, si = 1.f;
    double s64 = 1.0;
    float rr = 0.f, stop2 = 0.f;
    bool zero_rhs = false;
    double ui = 0.0, kdu = 0.0;
    float2 uo2 = make_float2(0.f, 0.f);  // PIPE: u_old as a float pair
    if constexpr (PIPE) {
        // right-hand side c = mw + u_old mq, residual res + u_old mq
        uo2 = a.u_old2[i];
        float cv[R];
        float m = 0.f, rs = 0.f, cs = 0.f;
#pragma unroll
        for (int k = 0; k < R; ++k) {
            r[k] = make_float2(0.f, 0.f);
            cv[k] = 0.f;
            if (valid[k]) {
                const size_t j = io + p + n1 * (q0 + k);
                const float2 t = ff_mul(a.mq2[j], uo2);
                r[k] = ff_add(a.res2[j], t);
                cv[k] = a.mw2[j].x + t.x;  // FP32 is enough for ||c||
                m = fmaxf(m, fmaxf(fabsf(cv[k]), fabsf(r[k].x)));
                rs = fmaf(r[k].x, r[k].x, rs);
                cs = fmaf(cv[k], cv[k], cs);
            }
        }
        // one reduction for ||r||^2, ||c||^2 and max |c|, |r|; values far
        // from 1 (whose squares could leave the FP32 range) are summed again
        // scaled by a power of two
        tm.sum2_max(rs, cs, m, reinterpret_cast<float4*>(red));
        if (!(m >= 0x1p-16f && m <= 0x1p+40f) && m > 0.f && m <= 3.0e38f) {
            const int e = ilogbf(m);
            s = pow2f(-e);
            si = pow2f(e);
            rs = 0.f;
            cs = 0.f;
#pragma unroll
            for (int k = 0; k < R; ++k) {
                const float x = r[k].x * s, c = cv[k] * s;
                rs = fmaf(x, x, rs);
                cs = fmaf(c, c, cs);
            }
            tm.sum2(rs, cs, red + 96);
        }
        rr = rs;
        zero_rhs = cs == 0.f;
        stop2 = a.tol2f * cs;
        // residual values below 2^-149 / s are not represented in the pairs
        if (s > 0x1p+100f) {
            const float f = 0x1p-149f * s;
            stop2 = fmaxf(stop2, 16.f * (float)a.nm * f * f);
        }
        if (zero_rhs) {
#pragma unroll
            for (int k = 0; k < R; ++k) r[k] = make_float2(0.f, 0.f);
        }
    } else {
        // stored FP64 residual of the iterate, for the new macro value u_i:
        // r = res + kappa (u_i - u_used_i) r_i (only Robin-edge nodes change)
        ui = a.u[i];
        kdu = a.kappa * (ui - a.u_used[i]);
        const double* bn = a.bnorm + (size_t)i * 3;
        const double ku = a.kappa * ui;
        const double bn2 = fma(ku * ku, bn[2], fma(2.0 * ku, bn[1], bn[0]));
        zero_rhs = !(bn2 > 0.0);
        s64 = pow2_scale_of_norm2(bn2);
        const double* res = a.res + io;
        double r64[R];
#pragma unroll
        for (int k = 0; k < R; ++k) {
            r64[k] = 0.0;
            r[k] = make_float2(0.f, 0.f);
            if (valid[k]) {
                const int q = q0 + k;
                double x = res[p + n1 * q];
                if (edge) x = fma(kdu, re[q], x);
                r64[k] = x * s64;
                r[k].x = __double2float_rn(r64[k]);
                rr = fmaf(r[k].x, r[k].x, rr);
            }
        }
        float dummy = 0.f;
        tm.sum2(rr, dummy, red);
        stop2 = (float)(a.tol * a.tol * bn2 * s64 * s64);
        if (!zero_rhs && rr > stop2) {  // low parts only where a solve follows
#pragma unroll
            for (int k = 0; k < R; ++k) r[k].y = __double2float_rn(r64[k] - (double)r[k].x);
        }
    }

    // ---- refinement: FP32 CG on S^ y = D^-1/2 r, then r -= S d, dv += d ----
    int inner = 0, sweeps = 0, flag = 0;
    bool solved = false, planes_zero = false;
    float2 dv[R];
#pragma unroll
    for (int k = 0; k < R; ++k) dv[k] = make_float2(0.f, 0.f);
    if (!(rr == rr)) {
        flag = kNaN;
    } else if (zero_rhs) {
        solved = true;  // the solution is zero
    } else if (rr > stop2) {
        solved = true;
        planes_zero = true;
        for (int e = tid; e < (PIPE ? 2 : 1) * pw; e += T) P[e] = 0.f;
        const float4* ch = a.chat + (size_t)i * 2 * pl;
        RegCouplings<R> creg;
        float sch[R];  // 1/sqrt(S_jj), high part
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const int j = p + n1 * (q0 + k);
            Couple8 c8{0, 0, 0, 0, 0, 0, 0, 0};
            sch[k] = 0.f;
            if (valid[k]) {
                c8 = couple8(ch[j], ch[pl + j]);
                sch[k] = a.dsc[io + j].x;
            }
            if constexpr (SC) {
                if (active) {  // padding rows of the last strip get zero couplings
                    cA[j] = make_float4(c8.E, c8.W, c8.N, c8.S);
                    cB[j] = make_float4(c8.NE, c8.NW, c8.SE, c8.SW);
                }
            } else {
                creg.c[k] = c8;
            }
        }
        tm.sync();
        const SmemCouplings cs{cA, cB, p + n1 * q0, n1};
        const float4* clo = a.chatlo + (size_t)i * 2 * pl;
        for (;;) {
            if (sweeps >= a.max_sweeps || inner >= a.maxit) {
                flag = kNotConverged;
                break;
            }
            // FP32 correction to inner_tol relative, but no further than 0.9
            // of what the outer tolerance still needs (kInnerMargin2 = 0.9^2).
            // The inner right-hand
            // side is the residual normalised by a power of two t (exact), so
            // the FP32 CG works on values of order one however far the
            // refinement has come; t and s are undone on the correction.
            const int et = ilogbf(sqrtf(rr));
            const float t = pow2f(-et), ti = pow2f(et);
            float y[R], rhs[R];
#pragma unroll
            for (int k = 0; k < R; ++k) {
                y[k] = 0.f;
                rhs[k] = sch[k] * ((PIPE ? r[k].x * s : r[k].x) * t);
            }
            const float rel2 = fmaxf(a.inner2f, kInnerMargin2 * stop2 / rr);
            if constexpr (SC)
                inner += strip_cg<R, SmemCouplings, TEAM>(cs, valid, y, rhs, P, Wd, p, q0, rel2, a.maxit - inner, red, red + 32, &flag, tm);
            else
                inner += strip_cg<R, RegCouplings<R>, TEAM>(creg, valid, y, rhs, P, Wd, p, q0, rel2, a.maxit - inner, red, red + 32, &flag, tm);
            if (flag == kNaN) break;
            flag = 0;  // an FP32 breakdown only ends this inner solve; the residual decides
            // S d = D^1/2 (S^ y) and d = D^-1/2 y in float-float
            strip_store<R>(P, Wd, p, q0, valid, y);
            tm.sync();
            wait_staged();
            StripHalo<R> h;
            h.load(P, Wd, p, q0);
            float rs = 0.f;
#pragma unroll
            for (int k = 0; k < R; ++k) {
                if (!valid[k]) continue;
                const int j = p + n1 * (q0 + k);
                Couple8 c;
                if constexpr (SC)
                    c = cs.get(k);
                else
                    c = creg.get(k);
                const float4 la = PREF ? sLo[j] : clo[j], lb = PREF ? sLo[pl + j] : clo[pl + j];
                const float4 ds = PREF ? sDs[j] : a.dsc[io + j];
                const float up = (k + 1 < R) ? y[k + 1] : h.xp;
                const float dn = (k > 0) ? y[k - 1] : h.xm;
                float ts = y[k], tc = 0.f;
                ff_acc(ts, tc, c.E, la.x, h.Rt[k + 1]);
                ff_acc(ts, tc, c.W, la.y, h.L[k + 1]);
                ff_acc(ts, tc, c.N, la.z, up);
                ff_acc(ts, tc, c.S, la.w, dn);
                ff_acc(ts, tc, c.NE, lb.x, h.Rt[k + 2]);
                ff_acc(ts, tc, c.NW, lb.y, h.L[k + 2]);
                ff_acc(ts, tc, c.SE, lb.z, h.Rt[k]);
                ff_acc(ts, tc, c.SW, lb.w, h.L[k]);
                float2 sd = ff_mul(make_float2(ds.z, ds.w), fast_two_sum_f(ts, tc));
                float2 d = ff_mul(make_float2(ds.x, ds.y), make_float2(y[k], 0.f));
                // back to the residual's scale (exact powers of two)
                sd = make_float2(sd.x * ti, sd.y * ti);
                d = make_float2(d.x * ti, d.y * ti);
                if constexpr (PIPE) {
                    sd = make_float2(sd.x * si, sd.y * si);
                    d = make_float2(d.x * si, d.y * si);
                }
                r[k] = ff_sub(r[k], sd);
                dv[k] = ff_add(dv[k], d);
                const float x = PIPE ? r[k].x * s : r[k].x;
                rs = fmaf(x, x, rs);
            }
            float dummy = 0.f;
            tm.sum2(rs, dummy, red + 64 + 32 * (sweeps & 1));
            rr = rs;
            ++sweeps;
            if (!(rr == rr)) {
                flag = kNaN;
                break;
            }
            if (rr <= stop2) break;
        }
    }

    wait_staged();  // (no copy may still be in flight when the block ends)
    if constexpr (!PIPE) {
        // ---- FP64 solution and stored residual ----
        double* v = a.v + io;
        double* res = a.res + io;
        const double sinv = 1.0 / s64;  // a power of two: exact
#pragma unroll
        for (int k = 0; k < R; ++k) {
            if (!valid[k]) continue;
            const int q = q0 + k, j = p + n1 * q;
            if (zero_rhs) {
                v[j] = 0.0;
                res[j] = 0.0;
            } else if (solved) {
                v[j] += ff_to_double(dv[k]) * sinv;
                res[j] = ff_to_double(r[k]) * sinv;
            } else if (edge && kdu != 0.0) {
                res[j] = fma(kdu, re[q], res[j]);
            }
        }
        tm.sync();
        // flux integral rho_i = r_i^T v_i over the Robin-edge nodes, one warp,
        // compensated (TwoSum) FP64
        if (tid < 32) {
            double sm = 0.0, cp = 0.0;
            for (int q = tid; q < n1; q += 32) {
                double su, er;
                two_sum(sm, re[q] * v[(n1 - 1) + n1 * q], su, er);
                sm = su;
                cp += er;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                double su, er;
                two_sum(sm, __shfl_xor_sync(0xffffffffu, sm, o), su, er);
                sm = su;
                cp += __shfl_xor_sync(0xffffffffu, cp, o) + er;
            }
            if (tid == 0) {
                a.u_used[i] = ui;
                a.rho[i] = sm + cp;
            }
        }
    } else {
        // ---- pipelined epilogue: prepare the next solve ----
        // w = g + dv; M w / dt (float-float, planes of the high and low parts);
        // S w = c - e; push w and S w into the rings at slot hist_step; the
        // extrapolated warm start g' and S g' by the same combination
        // (quadratic with two older solves, linear with one); the next
        // residual's u-independent part M w / dt - S g'.
        const int st = a.ctl->hist_step, level = a.ctl->hist_level;
        const size_t slot = (size_t)a.nM * pl;
        float2* hc = a.hist2 + (size_t)(st % 3) * slot + io;
        const float2* h1 = a.hist2 + (size_t)((st + 2) % 3) * slot + io;
        const float2* h2 = a.hist2 + (size_t)((st + 1) % 3) * slot + io;
        float2* yc = a.yhist2 + (size_t)(st % 3) * slot + io;
        const float2* y1 = a.yhist2 + (size_t)((st + 2) % 3) * slot + io;
        const float2* y2 = a.yhist2 + (size_t)((st + 1) % 3) * slot + io;
        float2 w[R];
        float wh[R], wl[R];
#pragma unroll
        for (int k = 0; k < R; ++k) {
            w[k] = make_float2(0.f, 0.f);
            if (valid[k] && !zero_rhs) {
                const float2 g = a.w2[io + p + n1 * (q0 + k)];
                w[k] = solved ? ff_add(g, dv[k]) : g;
            }
            wh[k] = w[k].x;
            wl[k] = w[k].y;
        }
        tm.sync();  // every read of the plane is done
        if (!planes_zero)
            for (int e = tid; e < 2 * pw; e += T) P[e] = 0.f;
        tm.sync();
        strip_store<R>(P, Wd, p, q0, valid, wh);
        strip_store<R>(P2, Wd, p, q0, valid, wl);
        tm.sync();
        StripHalo<R> hh, hl;
        hh.load(P, Wd, p, q0);
        hl.load(P2, Wd, p, q0);
        const float* Mh = PREF ? sMh : a.Mh + (size_t)i * kPlanes * pl;
        const float* Ml = PREF ? sMl : a.Ml + (size_t)i * kPlanes * pl;
#pragma unroll
        for (int k = 0; k < R; ++k) {
            if (!valid[k]) continue;
            const int q = q0 + k, j = p + n1 * q;
            const bool ww = p > 0, ee = p + 1 < n1, sd = q > 0;
            const float uph = (k + 1 < R) ? wh[k + 1] : hh.xp, upl = (k + 1 < R) ? wl[k + 1] : hl.xp;
            const float dnh = (k > 0) ? wh[k - 1] : hh.xm, dnl = (k > 0) ? wl[k - 1] : hl.xm;
            // forward couplings are stored as zero towards nodes outside the
            // mesh, whose plane values are zero as well
            float ms = 0.f, mc = 0.f;
            ff_acc2(ms, mc, Mh[j], Ml[j], wh[k], wl[k]);
            ff_acc2(ms, mc, Mh[pl + j], Ml[pl + j], hh.Rt[k + 1], hl.Rt[k + 1]);
            ff_acc2(ms, mc, Mh[2 * pl + j], Ml[2 * pl + j], uph, upl);
            ff_acc2(ms, mc, Mh[3 * pl + j], Ml[3 * pl + j], hh.Rt[k + 2], hl.Rt[k + 2]);
            ff_acc2(ms, mc, Mh[4 * pl + j], Ml[4 * pl + j], hh.L[k + 2], hl.L[k + 2]);
            if (ww) ff_acc2(ms, mc, Mh[pl + j - 1], Ml[pl + j - 1], hh.L[k + 1], hl.L[k + 1]);
            if (sd) {
                ff_acc2(ms, mc, Mh[2 * pl + j - n1], Ml[2 * pl + j - n1], dnh, dnl);
                if (ww) ff_acc2(ms, mc, Mh[3 * pl + j - n1 - 1], Ml[3 * pl + j - n1 - 1], hh.L[k], hl.L[k]);
                if (ee) ff_acc2(ms, mc, Mh[4 * pl + j - n1 + 1], Ml[4 * pl + j - n1 + 1], hh.Rt[k], hl.Rt[k]);
            }
            const float2 mwn = fast_two_sum_f(ms, mc);
            const float2 c = ff_add(a.mw2[io + j], ff_mul(a.mq2[io + j], uo2));
            const float2 sw = ff_sub(c, r[k]);
            float2 g = w[k], sg = sw;
            if (level >= 2) {
                g = ff_add(ff_scale(ff_sub(w[k], h1[j]), 3.f), h2[j]);
                sg = ff_add(ff_scale(ff_sub(sw, y1[j]), 3.f), y2[j]);
            } else if (level == 1) {
                g = ff_sub(ff_scale(w[k], 2.f), h1[j]);
                sg = ff_sub(ff_scale(sw, 2.f), y1[j]);
            }
            hc[j] = w[k];
            yc[j] = sw;
            a.mw2[io + j] = mwn;
            a.res2[io + j] = ff_sub(mwn, sg);
            a.w2[io + j] = g;
        }
        // (the flux r^T w of the pushed w is summed by the next macro prologue
        // from the ring, in compensated FP64)
        if (i == 0 && tid == 0) a.ctl->pushed = 1;
    }
    if (timed_out) flag = kTimeout;
    if (tid == 0) {
        a.inst_iters[i] = inner;
        atomicAdd(&a.ctl->inner_iters, (unsigned long long)inner);
        atomicAdd(&a.ctl->sweeps, (unsigned long long)sweeps);
        atomicAdd(&a.ctl->micro_solves, 1ull);
        atomicMax(&a.ctl->max_inner, inner);
        if (flag) set_status(a.ctl, flag);
    }
}

// Short strips (couplings in registers, PREF: staged sweep and epilogue data)
// and tall strips (couplings in shared memory, register budget capped so that
// several blocks share an SM).  PIPE: the pipelined-elimination instantiation
// (MicroArgs::pipe).
template <int R, bool PIPE, bool PREF>
__global__ void __launch_bounds__(StripMaxThreads<R>::value, StripMinBlocks<R>::value) k_micro_strip(MicroArgs a) {
    strip_body<R, false, PIPE, PREF>(a);
}
constexpr int kTallStripRegs = 160;
template <int R, bool PIPE>
__global__ void __maxnreg__(kTallStripRegs) k_micro_strip_tall(MicroArgs a) {
    strip_body<R, true, PIPE, false>(a);
}

// One warp per micro problem, kWarpsPerBlock problems per block (micro meshes
// whose strips fit 32 threads).
constexpr int kWarpsPerBlock = 8;
template <int R>
struct WarpMinBlocks {
    static constexpr int value = R == 3 ? 3 : 2;
};
template <int R, bool PIPE>
__global__ void __launch_bounds__(32 * kWarpsPerBlock, WarpMinBlocks<R>::value) k_micro_warp(MicroArgs a) {
    strip_body<R, false, PIPE, false, WarpTeam>(a);
}

bool warp_fits(int n1, int R, int smem_optin) {
    return n1 * strip_rows(n1, R) <= 32 &&
           kWarpsPerBlock * strip_smem_bytes(n1, R, false, true, false) <= (size_t)smem_optin;
}

cudaError_t launch_warp_solve(const MicroArgs& a, int R, cudaStream_t s) {
    const bool pipe = a.pipe != 0;
    const size_t sm = kWarpsPerBlock * strip_smem_bytes(a.n1, R, false, pipe, false);
    const unsigned nb = (unsigned)((a.nM + kWarpsPerBlock - 1) / kWarpsPerBlock);
    const int T = 32 * kWarpsPerBlock;
    if (a.n1 * strip_rows(a.n1, R) > 32) return cudaErrorInvalidConfiguration;
    if (R == 3) {
        if (pipe) k_micro_warp<3, true><<<nb, T, sm, s>>>(a);
        else k_micro_warp<3, false><<<nb, T, sm, s>>>(a);
    } else if (R == 5) {
        if (pipe) k_micro_warp<5, true><<<nb, T, sm, s>>>(a);
        else k_micro_warp<5, false><<<nb, T, sm, s>>>(a);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Persistent batch kernel.  Each block is one team of the column-strip solve
// (R rows a thread, the block's threads those of one micro problem) and
// loops: take the next item from its queue, read that problem instance's
// arguments from the kernel parameters, solve the item's micro problems one
// after another.  The launch bounds are those of k_micro_strip<R>, so the
// solve body gets the same register allocation.
// ---------------------------------------------------------------------------
int batch_strip_R(int n1) {
    if (strip_threads(n1, 3) <= StripMaxThreads<3>::value) return 3;
    if (strip_threads(n1, 5) <= StripMaxThreads<5>::value) return 5;
    return 0;
}
int batch_threads(int n1, int R) { return strip_threads(n1, R); }
bool batch_stages(int n1, int R) { return strip_stages(n1, R, true); }
size_t batch_smem(int n1, int R, bool pref) { return strip_smem_bytes(n1, R, false, true, pref); }

template <int R, bool PREF>
__global__ void __launch_bounds__(StripMaxThreads<R>::value, StripMinBlocks<R>::value)
    k_micro_batch(const __grid_constant__ BatchSolveArgs b) {
    __shared__ int4 s_item;
    for (;;) {
        if (threadIdx.x == 0) {
            const int it = atomicAdd(b.counter, 1);
            s_item = it < b.nitems ? b.items[it] : make_int4(-1, 0, 0, 0);
        }
        __syncthreads();
        const int4 item = s_item;
        if (item.x < 0) break;  // queue drained (the same in every thread)
        const MicroArgs& a = b.args[item.x];
        for (int j = 0; j < item.z; ++j) strip_body<R, false, true, PREF, BlockTeamAt>(a, BlockTeamAt{item.y + j});
        __syncthreads();  // every thread has read s_item before it is written again
    }
}

const void* k_micro_batch_entry(int R, bool pref) {
    if (R == 3) return pref ? (const void*)k_micro_batch<3, true> : (const void*)k_micro_batch<3, false>;
    if (R == 5) return pref ? (const void*)k_micro_batch<5, true> : (const void*)k_micro_batch<5, false>;
    return nullptr;
}

cudaError_t launch_batch_solve(const BatchSolveArgs& b, int R, bool pref, int threads, size_t smem_bytes, int blocks,
                               int priority, cudaStream_t s) {
    const void* fn = k_micro_batch_entry(R, pref);
    if (!fn) return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem_bytes;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributePriority;
    at[0].val.priority = priority;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    void* params[] = {const_cast<BatchSolveArgs*>(&b)};
    return cudaLaunchKernelExC(&cfg, fn, params);
}

template <int R, bool SC>
static cudaError_t launch_strip(const MicroArgs& a, cudaStream_t s) {
    const int T = strip_threads(a.n1, R);
    if (T > StripMaxThreads<R>::value) return cudaErrorInvalidConfiguration;
    const bool pipe = a.pipe != 0;
    if constexpr (SC) {
        const size_t sm = strip_smem_bytes(a.n1, R, true, pipe, false);
        if (pipe) k_micro_strip_tall<R, true><<<a.nM, T, sm, s>>>(a);
        else k_micro_strip_tall<R, false><<<a.nM, T, sm, s>>>(a);
    } else {
        const bool pref = strip_stages(a.n1, R, pipe);
        const size_t sm = strip_smem_bytes(a.n1, R, false, pipe, pref);
        if (pipe) {
            if (pref) k_micro_strip<R, true, true><<<a.nM, T, sm, s>>>(a);
            else k_micro_strip<R, true, false><<<a.nM, T, sm, s>>>(a);
        } else {
            if (pref) k_micro_strip<R, false, true><<<a.nM, T, sm, s>>>(a);
            else k_micro_strip<R, false, false><<<a.nM, T, sm, s>>>(a);
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_strip_solve(const MicroArgs& a, int R, cudaStream_t s) {
    switch (R) {
        case 3: return launch_strip<3, false>(a, s);
        case 5: return launch_strip<5, false>(a, s);
        case 7: return launch_strip<7, false>(a, s);
        case 9: return launch_strip<9, true>(a, s);
        case 11: return launch_strip<11, true>(a, s);
        case 13: return launch_strip<13, true>(a, s);
    }
    return cudaErrorInvalidValue;
}

// ===========================================================================
// One micro problem per thread-block cluster (multi-CTA per problem).
//
// For micro meshes too large for one block, and for batches with fewer micro
// problems than the GPU has SMs, the strips of one problem are divided among
// the G CTAs of a cluster: CTA g owns strips [g ns / G, (g+1) ns / G).  Each
// CTA keeps its rows in its own shared-memory plane; the rows next to a CTA
// boundary reach the neighbouring CTA by stores into its plane through
// distributed shared memory, and the dot products of the CG go to every CTA
// of the cluster the same way, so that the vectors never leave the chip.
// Barriers are cluster barriers.  The arithmetic per node is that of the
// single-block strip kernels above.
// ===========================================================================
__host__ __device__ inline int cl_strip_begin(int ns, int G, int g) { return (int)(((long long)ns * g) / G); }

// Where the CTA's boundary rows go: the plane of rank g-1 receives this CTA's
// first grid row as its top halo row (rowDn), the plane of rank g+1 this
// CTA's last grid row as its bottom halo row (row 0).
struct ClusterLink {
    int g, G;
    float* Pdn;     // plane of rank g - 1 (nullptr for g = 0)
    float* Pup;     // plane of rank g + 1 (nullptr for the last rank)
    float* P2dn;    // second planes (pipelined epilogue)
    float* P2up;
    int rowDn;      // local row of this CTA's first grid row in rank g - 1's plane
    bool first, last;  // this thread owns the CTA's first / last strip
};

// Store the strip's R values into the local plane (local rows lq0 + 1 ..) and
// the boundary rows into the neighbours' planes.
template <int R>
__device__ __forceinline__ void cl_store(float* P, float* Pdn, float* Pup, const ClusterLink& L, int Wd, int p,
                                         int lq0, const bool (&valid)[R], const float (&v)[R]) {
#pragma unroll
    for (int k = 0; k < R; ++k)
        if (valid[k]) P[(lq0 + k + 1) * Wd + p + 1] = v[k];
    if (L.first && Pdn && valid[0]) Pdn[L.rowDn * Wd + p + 1] = v[0];
    if (L.last && Pup && valid[R - 1]) Pup[p + 1] = v[R - 1];
}

// Sums of two FP32 values over every thread of the cluster: a butterfly in
// each warp, then lane l < G of each warp stores the warp's partial into the
// buffer of CTA l at slot g * 32 + warp; after the cluster barrier every thread
// adds all G x nw partials in the same fixed order.  buf: G x 32 float2, not
// written again before every thread of the cluster has passed one more
// cluster barrier.
__device__ __forceinline__ void cluster_sum2(float& x, float& y, float2* buf, const ClusterLink& L) {
    cg::cluster_group cl = cg::this_cluster();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        x += __shfl_xor_sync(0xffffffffu, x, o);
        y += __shfl_xor_sync(0xffffffffu, y, o);
    }
    if (lane < L.G) cl.map_shared_rank(buf, lane)[L.g * 32 + warp] = make_float2(x, y);
    cl.sync();
    float sx = 0.f, sy = 0.f, tx = 0.f, ty = 0.f;
    for (int r = 0; r < L.G; ++r) {
        const float2* b = buf + r * 32;
        int k = 0;
        for (; k + 1 < nw; k += 2) {
            const float4 t = *reinterpret_cast<const float4*>(b + k);
            sx += t.x;
            sy += t.y;
            tx += t.z;
            ty += t.w;
        }
        if (k < nw) {
            sx += b[k].x;
            sy += b[k].y;
        }
    }
    x = sx + tx;
    y = sy + ty;
}

// The same for two sums and a maximum of a non-negative value.  buf: G x 32 float4.
__device__ __forceinline__ void cluster_sum2_max(float& x, float& y, float& m, float4* buf, const ClusterLink& L) {
    cg::cluster_group cl = cg::this_cluster();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        x += __shfl_xor_sync(0xffffffffu, x, o);
        y += __shfl_xor_sync(0xffffffffu, y, o);
    }
    const float mb = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(m)));
    if (lane < L.G) cl.map_shared_rank(buf, lane)[L.g * 32 + warp] = make_float4(x, y, mb, 0.f);
    cl.sync();
    float sx = 0.f, sy = 0.f, mx = 0.f;
    for (int r = 0; r < L.G; ++r)
        for (int k = 0; k < nw; ++k) {
            const float4 t = buf[r * 32 + k];
            sx += t.x;
            sy += t.y;
            mx = fmaxf(mx, t.z);
        }
    x = sx;
    y = sy;
    m = mx;
}

// Chronopoulos-Gear CG of the cluster (strip_cg with the plane stores and
// reductions of the cluster).
template <int R, class CS>
__device__ int cluster_cg(const CS& c, const bool (&valid)[R], float (&x)[R], float (&r)[R], float* P,
                          const ClusterLink& L, int Wd, int p, int lq0, float rel2, int maxit, float2* redA,
                          float2* redB, int* flag) {
    cg::cluster_group cl = cg::this_cluster();
    float pv[R], s[R], w[R];
    StripHalo<R> h;
    cl_store<R>(P, L.Pdn, L.Pup, L, Wd, p, lq0, valid, r);
    cl.sync();
    if constexpr (R >= 9) {
        strip_apply_plane<R>(c, r, P, Wd, p, lq0, valid, w);
    } else {
        h.load(P, Wd, p, lq0);
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
    cluster_sum2(g, dl, redA, L);
    const float stop = rel2 * g;
    if (!(dl > 0.f)) {
        *flag = (dl == dl) ? kBreakdown : kNaN;
        return 0;
    }
    float alpha = __fdividef(g, dl);
    int it = 0;
    while (it < maxit) {
#pragma unroll
        for (int k = 0; k < R; ++k) {
            x[k] = fmaf(alpha, pv[k], x[k]);
            r[k] = fmaf(-alpha, s[k], r[k]);
        }
        ++it;
        cl_store<R>(P, L.Pdn, L.Pup, L, Wd, p, lq0, valid, r);
        cl.sync();
        if constexpr (R >= 9) {
            strip_apply_plane<R>(c, r, P, Wd, p, lq0, valid, w);
        } else {
            h.load(P, Wd, p, lq0);
            strip_apply<R>(c, r, h, w);
        }
        float gn = 0.f, dn = 0.f;
#pragma unroll
        for (int k = 0; k < R; ++k) {
            gn = fmaf(r[k], r[k], gn);
            dn = fmaf(r[k], w[k], dn);
        }
        cluster_sum2(gn, dn, (it & 1) ? redB : redA, L);
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

// Shared memory of one CTA of a cluster: the plane(s) for the largest share
// of strips, four reduction buffers of G x 32 float4, and (sc) the couplings
// of the CTA's rows.
static size_t cluster_smem_bytes(int n1, int R, int G, bool sc, bool pipe) {
    const int ns = strip_rows(n1, R), smax = (ns + G - 1) / G;
    const size_t W = (size_t)strip_stride(n1, R), H = (size_t)smax * R + 2;
    size_t off = ((pipe ? 2 : 1) * W * H * sizeof(float) + 15) & ~(size_t)15;
    off += 4 * (size_t)G * 32 * sizeof(float4);
    if (sc) off += 2 * (size_t)n1 * smax * R * sizeof(float4);
    return off;
}
static int cluster_threads(int n1, int R, int G) {
    const int ns = strip_rows(n1, R), smax = (ns + G - 1) / G;
    return (n1 * smax + 31) / 32 * 32;
}

template <int R, bool SC, bool PIPE>
__device__ __forceinline__ void cluster_body(const MicroArgs& a) {
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ __align__(16) unsigned char smem[];
    const int G = (int)cl.num_blocks(), g = (int)cl.block_rank();
    const int n1 = a.n1, Wd = strip_stride(n1, R), ns = strip_rows(n1, R);
    const int s0 = cl_strip_begin(ns, G, g), s1 = cl_strip_begin(ns, G, g + 1);
    const int smax = (ns + G - 1) / G, Hd = smax * R + 2, pw = Wd * Hd;
    float* P = reinterpret_cast<float*>(smem);
    float* P2 = P + pw;
    size_t off = ((size_t)(PIPE ? 2 : 1) * pw * sizeof(float) + 15) & ~(size_t)15;
    float4* red4 = reinterpret_cast<float4*>(smem + off);  // 4 buffers of G x 32 float4
    float2* redA = reinterpret_cast<float2*>(red4);
    float2* redB = reinterpret_cast<float2*>(red4 + G * 32);
    float2* redC = reinterpret_cast<float2*>(red4 + 2 * G * 32);
    float4* redD = red4 + 3 * G * 32;
    off += 4 * (size_t)G * 32 * sizeof(float4);
    float4* cA = reinterpret_cast<float4*>(smem + off);
    float4* cB = cA + n1 * smax * R;

    const int i = blockIdx.x / G, tid = threadIdx.x;
    const int nst = s1 - s0;
    const bool active = tid < n1 * nst;
    const int p = active ? tid % n1 : 0;
    const int sl = active ? tid / n1 : 0;  // local strip
    const int lq0 = sl * R;                // local row of the strip's first node (plane row lq0 + 1)
    const int q0 = (s0 + sl) * R;          // its grid row
    const size_t pl = (size_t)a.nmp, io = (size_t)i * pl;
    const double* re = a.redge + (size_t)i * n1;
    const bool edge = p == n1 - 1;
    bool valid[R];
#pragma unroll
    for (int k = 0; k < R; ++k) valid[k] = active && (q0 + k) < n1;
    ClusterLink L;
    L.g = g;
    L.G = G;
    L.Pdn = g > 0 ? cl.map_shared_rank(P, g - 1) : nullptr;
    L.Pup = g + 1 < G ? cl.map_shared_rank(P, g + 1) : nullptr;
    L.P2dn = g > 0 ? cl.map_shared_rank(P2, g - 1) : nullptr;
    L.P2up = g + 1 < G ? cl.map_shared_rank(P2, g + 1) : nullptr;
    L.rowDn = g > 0 ? (s0 - cl_strip_begin(ns, G, g - 1)) * R + 1 : 0;
    L.first = active && sl == 0;
    L.last = active && sl == nst - 1;
    // zero planes (the halo rows of the mesh boundary stay zero), then make
    // sure no CTA stores into a neighbour's plane before it is zeroed
    for (int e = tid; e < (PIPE ? 2 : 1) * pw; e += blockDim.x) P[e] = 0.f;
    cl.sync();

    float2 r[R];
    float s = 1.f, si = 1.f;
    double s64 = 1.0;
    float rr = 0.f, stop2 = 0.f;
    bool zero_rhs = false;
    double ui = 0.0, kdu = 0.0;
    float2 uo2 = make_float2(0.f, 0.f);
    if constexpr (PIPE) {
        uo2 = a.u_old2[i];
        float cv[R];
        float m = 0.f, rs = 0.f, cs = 0.f;
#pragma unroll
        for (int k = 0; k < R; ++k) {
            r[k] = make_float2(0.f, 0.f);
            cv[k] = 0.f;
            if (valid[k]) {
                const size_t j = io + p + n1 * (q0 + k);
                const float2 t = ff_mul(a.mq2[j], uo2);
                r[k] = ff_add(a.res2[j], t);
                cv[k] = a.mw2[j].x + t.x;
                m = fmaxf(m, fmaxf(fabsf(cv[k]), fabsf(r[k].x)));
                rs = fmaf(r[k].x, r[k].x, rs);
                cs = fmaf(cv[k], cv[k], cs);
            }
        }
        cluster_sum2_max(rs, cs, m, redD, L);
        if (!(m >= 0x1p-16f && m <= 0x1p+40f) && m > 0.f && m <= 3.0e38f) {
            const int e = ilogbf(m);
            s = pow2f(-e);
            si = pow2f(e);
            rs = 0.f;
            cs = 0.f;
#pragma unroll
            for (int k = 0; k < R; ++k) {
                const float x = r[k].x * s, c = cv[k] * s;
                rs = fmaf(x, x, rs);
                cs = fmaf(c, c, cs);
            }
            cluster_sum2(rs, cs, redC, L);
        }
        rr = rs;
        zero_rhs = cs == 0.f;
        stop2 = a.tol2f * cs;
        if (s > 0x1p+100f) {
            const float f = 0x1p-149f * s;
            stop2 = fmaxf(stop2, 16.f * (float)a.nm * f * f);
        }
        if (zero_rhs) {
#pragma unroll
            for (int k = 0; k < R; ++k) r[k] = make_float2(0.f, 0.f);
        }
    } else {
        ui = a.u[i];
        kdu = a.kappa * (ui - a.u_used[i]);
        const double* bn = a.bnorm + (size_t)i * 3;
        const double ku = a.kappa * ui;
        const double bn2 = fma(ku * ku, bn[2], fma(2.0 * ku, bn[1], bn[0]));
        zero_rhs = !(bn2 > 0.0);
        s64 = pow2_scale_of_norm2(bn2);
        const double* res = a.res + io;
        double r64[R];
#pragma unroll
        for (int k = 0; k < R; ++k) {
            r64[k] = 0.0;
            r[k] = make_float2(0.f, 0.f);
            if (valid[k]) {
                const int q = q0 + k;
                double x = res[p + n1 * q];
                if (edge) x = fma(kdu, re[q], x);
                r64[k] = x * s64;
                r[k].x = __double2float_rn(r64[k]);
                rr = fmaf(r[k].x, r[k].x, rr);
            }
        }
        float dummy = 0.f;
        cluster_sum2(rr, dummy, redC, L);
        stop2 = (float)(a.tol * a.tol * bn2 * s64 * s64);
        if (!zero_rhs && rr > stop2) {
#pragma unroll
            for (int k = 0; k < R; ++k) r[k].y = __double2float_rn(r64[k] - (double)r[k].x);
        }
    }

    int inner = 0, sweeps = 0, flag = 0;
    bool solved = false;
    float2 dv[R];
#pragma unroll
    for (int k = 0; k < R; ++k) dv[k] = make_float2(0.f, 0.f);
    if (!(rr == rr)) {
        flag = kNaN;
    } else if (zero_rhs) {
        solved = true;
    } else if (rr > stop2) {
        solved = true;
        const float4* ch = a.chat + (size_t)i * 2 * pl;
        RegCouplings<R> creg;
        float sch[R];
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const int j = p + n1 * (q0 + k);
            Couple8 c8{0, 0, 0, 0, 0, 0, 0, 0};
            sch[k] = 0.f;
            if (valid[k]) {
                c8 = couple8(ch[j], ch[pl + j]);
                sch[k] = a.dsc[io + j].x;
            }
            if constexpr (SC) {
                if (active) {
                    const int jl = p + n1 * (lq0 + k);  // node of the CTA's rows
                    cA[jl] = make_float4(c8.E, c8.W, c8.N, c8.S);
                    cB[jl] = make_float4(c8.NE, c8.NW, c8.SE, c8.SW);
                }
            } else {
                creg.c[k] = c8;
            }
        }
        __syncthreads();
        const SmemCouplings cs{cA, cB, p + n1 * lq0, n1};
        const float4* clo = a.chatlo + (size_t)i * 2 * pl;
        for (;;) {
            if (sweeps >= a.max_sweeps || inner >= a.maxit) {
                flag = kNotConverged;
                break;
            }
            const int et = ilogbf(sqrtf(rr));
            const float t = pow2f(-et), ti = pow2f(et);
            float y[R], rhs[R];
#pragma unroll
            for (int k = 0; k < R; ++k) {
                y[k] = 0.f;
                rhs[k] = sch[k] * ((PIPE ? r[k].x * s : r[k].x) * t);
            }
            const float rel2 = fmaxf(a.inner2f, kInnerMargin2 * stop2 / rr);
            if constexpr (SC)
                inner += cluster_cg<R>(cs, valid, y, rhs, P, L, Wd, p, lq0, rel2, a.maxit - inner, redA, redB, &flag);
            else
                inner += cluster_cg<R>(creg, valid, y, rhs, P, L, Wd, p, lq0, rel2, a.maxit - inner, redA, redB,
                                       &flag);
            if (flag == kNaN) break;
            flag = 0;
            cl_store<R>(P, L.Pdn, L.Pup, L, Wd, p, lq0, valid, y);
            cl.sync();
            StripHalo<R> h;
            h.load(P, Wd, p, lq0);
            float rs = 0.f;
#pragma unroll
            for (int k = 0; k < R; ++k) {
                if (!valid[k]) continue;
                const int j = p + n1 * (q0 + k);
                Couple8 c;
                if constexpr (SC)
                    c = cs.get(k);
                else
                    c = creg.get(k);
                const float4 la = clo[j], lb = clo[pl + j];
                const float4 ds = a.dsc[io + j];
                const float up = (k + 1 < R) ? y[k + 1] : h.xp;
                const float dn = (k > 0) ? y[k - 1] : h.xm;
                float ts = y[k], tc = 0.f;
                ff_acc(ts, tc, c.E, la.x, h.Rt[k + 1]);
                ff_acc(ts, tc, c.W, la.y, h.L[k + 1]);
                ff_acc(ts, tc, c.N, la.z, up);
                ff_acc(ts, tc, c.S, la.w, dn);
                ff_acc(ts, tc, c.NE, lb.x, h.Rt[k + 2]);
                ff_acc(ts, tc, c.NW, lb.y, h.L[k + 2]);
                ff_acc(ts, tc, c.SE, lb.z, h.Rt[k]);
                ff_acc(ts, tc, c.SW, lb.w, h.L[k]);
                float2 sd = ff_mul(make_float2(ds.z, ds.w), fast_two_sum_f(ts, tc));
                float2 d = ff_mul(make_float2(ds.x, ds.y), make_float2(y[k], 0.f));
                sd = make_float2(sd.x * ti, sd.y * ti);
                d = make_float2(d.x * ti, d.y * ti);
                if constexpr (PIPE) {
                    sd = make_float2(sd.x * si, sd.y * si);
                    d = make_float2(d.x * si, d.y * si);
                }
                r[k] = ff_sub(r[k], sd);
                dv[k] = ff_add(dv[k], d);
                const float x = PIPE ? r[k].x * s : r[k].x;
                rs = fmaf(x, x, rs);
            }
            float dummy = 0.f;
            cluster_sum2(rs, dummy, (sweeps & 1) ? redB : redA, L);
            rr = rs;
            ++sweeps;
            if (!(rr == rr)) {
                flag = kNaN;
                break;
            }
            if (rr <= stop2) break;
        }
    }

    if constexpr (!PIPE) {
        double* v = a.v + io;
        double* res = a.res + io;
        const double sinv = 1.0 / s64;
#pragma unroll
        for (int k = 0; k < R; ++k) {
            if (!valid[k]) continue;
            const int q = q0 + k, j = p + n1 * q;
            if (zero_rhs) {
                v[j] = 0.0;
                res[j] = 0.0;
            } else if (solved) {
                v[j] += ff_to_double(dv[k]) * sinv;
                res[j] = ff_to_double(r[k]) * sinv;
            } else if (edge && kdu != 0.0) {
                res[j] = fma(kdu, re[q], res[j]);
            }
        }
        __syncthreads();
        // rho_i = r_i^T v_i: each CTA sums its rows' Robin-edge nodes (one warp,
        // compensated FP64), rank 0 adds the G partial pairs in rank order
        double2* part = reinterpret_cast<double2*>(redD);  // G entries in rank 0's buffer
        if (tid < 32) {
            double sm = 0.0, cp = 0.0;
            const int qa = s0 * R, qb = min(s1 * R, n1);
            for (int q = qa + tid; q < qb; q += 32) {
                double su, er;
                two_sum(sm, re[q] * v[(n1 - 1) + n1 * q], su, er);
                sm = su;
                cp += er;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                double su, er;
                two_sum(sm, __shfl_xor_sync(0xffffffffu, sm, o), su, er);
                sm = su;
                cp += __shfl_xor_sync(0xffffffffu, cp, o) + er;
            }
            if (tid == 0) cl.map_shared_rank(part, 0)[g] = make_double2(sm, cp);
        }
        cl.sync();
        if (g == 0 && tid == 0) {
            double sm = 0.0, cp = 0.0;
            for (int k = 0; k < G; ++k) {
                double su, er;
                two_sum(sm, part[k].x, su, er);
                sm = su;
                cp += er + part[k].y;
            }
            a.u_used[i] = ui;
            a.rho[i] = sm + cp;
        }
    } else {
        const int st = a.ctl->hist_step, level = a.ctl->hist_level;
        const size_t slot = (size_t)a.nM * pl;
        float2* hc = a.hist2 + (size_t)(st % 3) * slot + io;
        const float2* h1 = a.hist2 + (size_t)((st + 2) % 3) * slot + io;
        const float2* h2 = a.hist2 + (size_t)((st + 1) % 3) * slot + io;
        float2* yc = a.yhist2 + (size_t)(st % 3) * slot + io;
        const float2* y1 = a.yhist2 + (size_t)((st + 2) % 3) * slot + io;
        const float2* y2 = a.yhist2 + (size_t)((st + 1) % 3) * slot + io;
        float2 w[R];
        float wh[R], wl[R];
#pragma unroll
        for (int k = 0; k < R; ++k) {
            w[k] = make_float2(0.f, 0.f);
            if (valid[k] && !zero_rhs) {
                const float2 gg = a.w2[io + p + n1 * (q0 + k)];
                w[k] = solved ? ff_add(gg, dv[k]) : gg;
            }
            wh[k] = w[k].x;
            wl[k] = w[k].y;
        }
        // (every CTA has finished reading its planes: the last reduction
        // ended with a cluster barrier, and the stores below only replace
        // values at owned or halo positions of the same planes)
        cl.sync();
        cl_store<R>(P, L.Pdn, L.Pup, L, Wd, p, lq0, valid, wh);
        cl_store<R>(P2, L.P2dn, L.P2up, L, Wd, p, lq0, valid, wl);
        cl.sync();
        StripHalo<R> hh, hl;
        hh.load(P, Wd, p, lq0);
        hl.load(P2, Wd, p, lq0);
        const float* Mh = a.Mh + (size_t)i * kPlanes * pl;
        const float* Ml = a.Ml + (size_t)i * kPlanes * pl;
#pragma unroll
        for (int k = 0; k < R; ++k) {
            if (!valid[k]) continue;
            const int q = q0 + k, j = p + n1 * q;
            const bool ww = p > 0, ee = p + 1 < n1, sd = q > 0;
            const float uph = (k + 1 < R) ? wh[k + 1] : hh.xp, upl = (k + 1 < R) ? wl[k + 1] : hl.xp;
            const float dnh = (k > 0) ? wh[k - 1] : hh.xm, dnl = (k > 0) ? wl[k - 1] : hl.xm;
            float ms = 0.f, mc = 0.f;
            ff_acc2(ms, mc, Mh[j], Ml[j], wh[k], wl[k]);
            ff_acc2(ms, mc, Mh[pl + j], Ml[pl + j], hh.Rt[k + 1], hl.Rt[k + 1]);
            ff_acc2(ms, mc, Mh[2 * pl + j], Ml[2 * pl + j], uph, upl);
            ff_acc2(ms, mc, Mh[3 * pl + j], Ml[3 * pl + j], hh.Rt[k + 2], hl.Rt[k + 2]);
            ff_acc2(ms, mc, Mh[4 * pl + j], Ml[4 * pl + j], hh.L[k + 2], hl.L[k + 2]);
            if (ww) ff_acc2(ms, mc, Mh[pl + j - 1], Ml[pl + j - 1], hh.L[k + 1], hl.L[k + 1]);
            if (sd) {
                ff_acc2(ms, mc, Mh[2 * pl + j - n1], Ml[2 * pl + j - n1], dnh, dnl);
                if (ww) ff_acc2(ms, mc, Mh[3 * pl + j - n1 - 1], Ml[3 * pl + j - n1 - 1], hh.L[k], hl.L[k]);
                if (ee) ff_acc2(ms, mc, Mh[4 * pl + j - n1 + 1], Ml[4 * pl + j - n1 + 1], hh.Rt[k], hl.Rt[k]);
            }
            const float2 mwn = fast_two_sum_f(ms, mc);
            const float2 c = ff_add(a.mw2[io + j], ff_mul(a.mq2[io + j], uo2));
            const float2 sw = ff_sub(c, r[k]);
            float2 gn = w[k], sg = sw;
            if (level >= 2) {
                gn = ff_add(ff_scale(ff_sub(w[k], h1[j]), 3.f), h2[j]);
                sg = ff_add(ff_scale(ff_sub(sw, y1[j]), 3.f), y2[j]);
            } else if (level == 1) {
                gn = ff_sub(ff_scale(w[k], 2.f), h1[j]);
                sg = ff_sub(ff_scale(sw, 2.f), y1[j]);
            }
            hc[j] = w[k];
            yc[j] = sw;
            a.mw2[io + j] = mwn;
            a.res2[io + j] = ff_sub(mwn, sg);
            a.w2[io + j] = gn;
        }
        if (i == 0 && g == 0 && tid == 0) a.ctl->pushed = 1;
        cl.sync();  // no CTA leaves while a neighbour may still read its planes
    }
    if (g == 0 && tid == 0) {
        a.inst_iters[i] = inner;
        atomicAdd(&a.ctl->inner_iters, (unsigned long long)inner);
        atomicAdd(&a.ctl->sweeps, (unsigned long long)sweeps);
        atomicAdd(&a.ctl->micro_solves, 1ull);
        atomicMax(&a.ctl->max_inner, inner);
        if (flag) set_status(a.ctl, flag);
    }
}

// Cluster variants: R = 5 (couplings in registers) and R = 9 (couplings in
// shared memory), G CTAs per micro problem set at launch.
template <int R, bool PIPE>
__global__ void __launch_bounds__(512, 1) k_micro_cluster(MicroArgs a) {
    cluster_body<R, false, PIPE>(a);
}
template <int R, bool PIPE>
__global__ void __maxnreg__(kTallStripRegs) k_micro_cluster_tall(MicroArgs a) {
    cluster_body<R, true, PIPE>(a);
}

// (R, G) of the cluster tilings, in tiling order
static const int kClusterR[kNumClusterTilings] = {5, 5, 9, 9};
static const int kClusterG[kNumClusterTilings] = {2, 4, 4, 8};

bool cluster_fits(int c, int n1, int smem_optin) {
    if (c < 0 || c >= kNumClusterTilings) return false;
    const int R = kClusterR[c], G = kClusterG[c];
    if (strip_rows(n1, R) < G) return false;  // every CTA needs a strip
    const int maxT = R >= 9 ? 384 : 512;
    return cluster_threads(n1, R, G) <= maxT &&
           cluster_smem_bytes(n1, R, G, R >= 9, true) <= (size_t)smem_optin;
}

template <int R, bool SC, bool PIPE>
static cudaError_t launch_cluster_kernel(const MicroArgs& a, int G, cudaStream_t s) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)a.nM * G);
    cfg.blockDim = dim3(cluster_threads(a.n1, R, G));
    cfg.dynamicSmemBytes = cluster_smem_bytes(a.n1, R, G, SC, PIPE);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = G;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if constexpr (SC) return cudaLaunchKernelEx(&cfg, k_micro_cluster_tall<R, PIPE>, a);
    else return cudaLaunchKernelEx(&cfg, k_micro_cluster<R, PIPE>, a);
}

cudaError_t launch_cluster_solve(const MicroArgs& a, int c, cudaStream_t s) {
    if (c < 0 || c >= kNumClusterTilings) return cudaErrorInvalidValue;
    const int R = kClusterR[c], G = kClusterG[c];
    if (R == 5) return a.pipe ? launch_cluster_kernel<5, false, true>(a, G, s) : launch_cluster_kernel<5, false, false>(a, G, s);
    return a.pipe ? launch_cluster_kernel<9, true, true>(a, G, s) : launch_cluster_kernel<9, true, false>(a, G, s);
}

bool strip_fits(int n1, int R, int smem_optin) {
    const bool sc = R >= 9;
    const int maxT = R == 3 ? 384 : (R == 5 ? 512 : 384);
    return strip_threads(n1, R) <= maxT && strip_smem_bytes(n1, R, sc, true, false) <= (size_t)smem_optin &&
           strip_smem_bytes(n1, R, sc, false, false) <= (size_t)smem_optin;
}

// Allow every strip kernel the device's opt-in shared memory (done once,
// outside any stream capture).
cudaError_t configure_strip_kernels(int smem_optin) {
    const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
    // (k_micro_batch, which also has static shared memory, gets its limit when
    // a persistent batch step is captured)
    const void* cfns[8] = {(const void*)k_micro_cluster<5, false>,      (const void*)k_micro_cluster<5, true>,
                           (const void*)k_micro_cluster_tall<9, false>, (const void*)k_micro_cluster_tall<9, true>,
                           (const void*)k_micro_warp<3, false>,         (const void*)k_micro_warp<3, true>,
                           (const void*)k_micro_warp<5, false>,         (const void*)k_micro_warp<5, true>};
    for (int k = 0; k < 8; ++k) {
        const cudaError_t e = cudaFuncSetAttribute(cfns[k], at, smem_optin);
        if (e != cudaSuccess) return e;
    }
    const void* fns[18] = {
        (const void*)k_micro_strip<3, false, false>, (const void*)k_micro_strip<5, false, false>,
        (const void*)k_micro_strip<7, false, false>, (const void*)k_micro_strip<3, true, false>,
        (const void*)k_micro_strip<5, true, false>,  (const void*)k_micro_strip<7, true, false>,
        (const void*)k_micro_strip<3, false, true>,  (const void*)k_micro_strip<5, false, true>,
        (const void*)k_micro_strip<7, false, true>,  (const void*)k_micro_strip<3, true, true>,
        (const void*)k_micro_strip<5, true, true>,   (const void*)k_micro_strip<7, true, true>,
        (const void*)k_micro_strip_tall<9, false>,   (const void*)k_micro_strip_tall<11, false>,
        (const void*)k_micro_strip_tall<13, false>,  (const void*)k_micro_strip_tall<9, true>,
        (const void*)k_micro_strip_tall<11, true>,   (const void*)k_micro_strip_tall<13, true>};
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 18 && e == cudaSuccess; ++k) e = cudaFuncSetAttribute(fns[k], at, smem_optin);
    return e;
}

}  // namespace tsf
