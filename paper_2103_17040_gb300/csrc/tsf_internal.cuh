// tsf_internal.cuh -- device-side structures and helpers shared by the
// kernels of the GB300 two-scale library (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace tsf {

// Stencil planes of a Q1 operator on an (n1 x n1) node grid.  The operator is
// symmetric, so only the couplings of node (p,q) to itself and to its
// "forward" neighbours are stored:
//   0: C (p,q)   1: E (p+1,q)   2: N (p,q+1)   3: NE (p+1,q+1)   4: NW (p-1,q+1)
// The remaining four couplings are read from the neighbour that stores them:
//   W = E(p-1,q), S = N(p,q-1), SW = NE(p-1,q-1), SE = NW(p+1,q-1).
// Couplings to nodes outside the mesh are stored as zero.
constexpr int kPlanes = 5;

// Device status codes (same values as tsf_status).
enum : int { kOk = 0, kNotConverged = 4, kNaN = 5, kBreakdown = 8, kBadJacobian = 3, kTimeout = 9 };

// Control and statistics block living in device memory.
struct DevCtl {
    unsigned long long inner_iters;   // inner CG iterations, summed over instances
    unsigned long long sweeps;        // FP64 residual evaluations of micro problems
    unsigned long long micro_solves;
    unsigned long long macro_iters;
    int coupling_iter;                // coupling iterations of the current step
    int coupling_iters_total;
    int coupling_iters_last;
    int max_inner;
    int status;                       // first device-side error, 0 if none
    int steps;
    int geom_error;                   // set by the geometry kernel on det F <= 0
    int cont;                         // 1 while the coupling loop must go on
    double change;                    // last relative change of u
    double gamma_bar;                 // preconditioner value of |Gamma| (macro)
    // exact elimination: history of past v0 fields for the warm start
    int hist_level;                   // number of valid past fields (0..2); reset with the state
    int hist_step;                    // ring position: the latest solve's w goes to slot hist_step % 3
    int pushed;                       // 1: k_elim_pre pushed a w the next k_elim_start must count
};

__device__ __forceinline__ void set_status(DevCtl* ctl, int code) {
    atomicCAS(&ctl->status, 0, code);
}

// ---------------------------------------------------------------------------
// Block-wide all-reduce of NV values.  blockDim.x must be a multiple of 32 and
// at most 1024.  buf must hold NV*32 elements and must not be reused by the
// block until every thread has returned from this call and passed one more
// __syncthreads (callers alternate two buffers).  The summation order is
// fixed (warp tree, then the warp partials in warp order through a second
// warp tree), so every thread gets the same, reproducible value.
// ---------------------------------------------------------------------------
template <typename T, int NV>
__device__ __forceinline__ void block_allreduce(T (&v)[NV], T* buf) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
    }
    if (lane == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) buf[i * 32 + warp] = v[i];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        T s = lane < nw ? buf[i * 32 + lane] : T(0);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        v[i] = s;
    }
}

// Error-free transformation a + b = s + e (Knuth's TwoSum).
__device__ __forceinline__ void two_sum(double a, double b, double& s, double& e) {
    s = a + b;
    double bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// Compensated block sum of one double per thread (sum and running error
// carried through the warp tree), result broadcast to all threads.
__device__ __forceinline__ double block_sum_compensated(double x, double* buf /* 64 */) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    double s = x, c = 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        double so = __shfl_xor_sync(0xffffffffu, s, o);
        double co = __shfl_xor_sync(0xffffffffu, c, o);
        double t, e;
        two_sum(s, so, t, e);
        s = t;
        c = c + co + e;
    }
    if (lane == 0) {
        buf[warp] = s;
        buf[32 + warp] = c;
    }
    __syncthreads();
    s = lane < nw ? buf[lane] : 0.0;
    c = lane < nw ? buf[32 + lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        double so = __shfl_xor_sync(0xffffffffu, s, o);
        double co = __shfl_xor_sync(0xffffffffu, c, o);
        double t, e;
        two_sum(s, so, t, e);
        s = t;
        c = c + co + e;
    }
    return s + c;
}

// y_j = (A x)_j for the symmetric 5-plane stencil A (planes of stride pl) on
// an n1 x n1 node grid, node j = (p, q), FP64.
__device__ __forceinline__ double plane_apply(const double* __restrict__ A, size_t pl, const double* __restrict__ x,
                                              int j, int p, int q, int n1) {
    double y = A[j] * x[j];
    const bool e = p + 1 < n1, w = p > 0;
    if (e) y = fma(A[pl + j], x[j + 1], y);
    if (w) y = fma(A[pl + j - 1], x[j - 1], y);
    if (q + 1 < n1) {
        y = fma(A[2 * pl + j], x[j + n1], y);
        if (e) y = fma(A[3 * pl + j], x[j + n1 + 1], y);
        if (w) y = fma(A[4 * pl + j], x[j + n1 - 1], y);
    }
    if (q > 0) {
        y = fma(A[2 * pl + j - n1], x[j - n1], y);
        if (w) y = fma(A[3 * pl + j - n1 - 1], x[j - n1 - 1], y);
        if (e) y = fma(A[4 * pl + j - n1 + 1], x[j - n1 + 1], y);
    }
    return y;
}


// ---------------------------------------------------------------------------
// Kernel argument blocks
// ---------------------------------------------------------------------------
struct GeomArgs {
    int Nm, n1, nm, nmp, nM;
    int affine;             // 1: every map has b = 0 (identity and affine families)
    const double* prm5;     // [nM][5] general form (A11, A12, A21, A22, b)
    double D11, D12, D22, kappa, dt;
    double* M64;            // [nM][5][nmp] mass planes
    double* S64;            // [nM][5][nmp] M/dt + A + kappa R planes
    float* S32;             // [nM][5][nmp] S64 rounded to FP32
    float* S32lo;           // [nM][5][nmp] S64 - S32 rounded to FP32, or nullptr
    double* lm;             // [nM][nmp]    row sums of M (lumped mass)
    double* redge;          // [nM][n1]     r = R 1 on the Robin edge nodes
    double* Rd;             // [nM][n1]     diagonal of R on the edge
    double* Ru;             // [nM][n1]     coupling of edge node q to q+1
    DevCtl* ctl;
};

struct MicroArgs {
    int n1, nm, nmp, W;     // W = n1 + 2: width of the zero-haloed shared-memory grid
    int nM;
    const float* S32;       // [nM][5][nmp] S64 rounded to FP32 (one-block-per-problem variants)
    const double* S64;
    const double* c;        // [nM][nmp] right-hand side without the u term
    double* v;              // [nM][nmp] in: initial guess, out: solution
    const double* u;        // [nM] macro iterate
    const double* redge;    // [nM][n1]
    double kappa;
    double tol;             // ||b - S v|| <= tol ||b|| (FP64-accurate residual)
    double inner_tol;       // mixed: relative tolerance of the FP32 inner solve
    float tol2f, inner2f;   // tol^2 and inner_tol^2 in FP32, set by the launchers (with_fp32_tols):
                            // an FP64 -> FP32 conversion in every thread costs the slow conversion pipe
    int maxit;              // cap on inner iterations per solve
    int max_sweeps;         // mixed: cap on refinement sweeps
    double* rho;            // [nM] out: r_i^T v_i
    int* inst_iters;        // [nM] out: inner iterations of this solve
    DevCtl* ctl;
    // stored-residual protocol of the column-strip kernels:
    double* res;            // [nM][nmp] FP64 residual b(u_used) - S v of the current iterate
    double* u_used;         // [nM] macro value the stored residual belongs to
    const double* bnorm;    // [nM][3] ||c||^2, c^T r, ||r||^2 (so ||b(u)||^2 is a quadratic in u)
    // column-strip kernels: the Jacobi-scaled operator S^ = D^-1/2 S D^-1/2
    // (unit diagonal) and the diagonal scalings, as FP32 pairs hi + lo
    const float4* chat;     // [nM][2][nmp] couplings of S^, high parts: (E, W, N, S), (NE, NW, SE, SW)
    const float4* chatlo;   // [nM][2][nmp] the low parts (S^ to about 2^-48)
    const float4* dsc;      // [nM][nmp] (1/sqrt(S_jj) hi, lo, sqrt(S_jj) hi, lo)
    // column-strip kernels, pipelined elimination (pipe = 1).  The solve of w
    // takes its right-hand side as c = mw + u_old mq and its residual as
    // res2 + u_old mq, starting from the warm start in w2; its epilogue pushes
    // w and S w = c - e into the rings at slot hist_step, leaves the
    // extrapolated warm start in w2, M w / dt in mw2 and the u-independent
    // part M w / dt - S g of the next residual in res2.  Every array of the
    // pipeline holds float pairs (hi, lo).
    int pipe;
    const float2* u_old2;   // [nM] macro values of the right-hand side as float pairs (zeros for the first w)
    float2* w2;             // [nM][nmp]
    float2* res2;           // [nM][nmp]
    float2* mw2;            // [nM][nmp]
    const float2* mq2;      // [nM][nmp] M psi / dt
    float2* hist2;          // [3][nM][nmp] ring of w
    float2* yhist2;         // [3][nM][nmp] ring of S w
    const float* Mh;        // [nM][5][nmp] M / dt split as Mh + Ml (FP32 pairs)
    const float* Ml;
};

// Per (geometry, dt) set-up of the column-strip kernels' operator data.
// The FP32 copies of the squared tolerances the column-strip kernels test
// against (set on the host, once per launch).
inline MicroArgs with_fp32_tols(MicroArgs a) {
    a.tol2f = (float)(a.tol * a.tol);
    a.inner2f = (float)(a.inner_tol * a.inner_tol);
    return a;
}

struct StripSetupArgs {
    int n1, nm, nmp, nM;
    const double* S64;      // [nM][5][nmp]
    const double* M64;      // [nM][5][nmp] (only with Mh)
    double idt;             // 1 / dt (only with Mh)
    double* rs;             // [nM][nmp] scratch: 1 / sqrt(S_jj)
    float4* chat;
    float4* chatlo;
    float4* dsc;
    float* Mh;              // [nM][5][nmp] or nullptr
    float* Ml;
};

struct PrologueArgs {
    int n1, nm, nmp, nM;
    double dt, kappa;
    const double* M64;
    const double* S64;
    double* v;              // [nM][nmp] state v^n (replaced by the warm start of v0 under elimination)
    const double* fv;       // [nM][nmp] or nullptr
    const double* g;        // [nM][n1] or nullptr
    const double* redge;
    const double* Rd;
    const double* Ru;
    const double* u;        // [nM] initial macro iterate of the step
    double* c;              // [nM][nmp] out: M (v/dt + fv) + R g
    double* res;            // [nM][nmp] out: c + kappa u r - S v
    double* u_used;         // [nM] out: u
    double* bnorm;          // [nM][3] out
    // exact elimination (nullptr otherwise): v is replaced in place by the
    // warm start v - uw phi of v0, and res = c - S v, u_used = 0
    const double* phi;      // [nM][nmp] S^-1 kappa r
    const double* uw;       // [nM] macro values of the state v
};

// One-off set-up of the solve S phi = kappa r with the stored-residual
// protocol (c = 0, u = 1, phi = 0): res = kappa r on the Robin edge,
// u_used = 1, bnorm = (0, 0, ||r||^2); zeroes phi and cz.
struct PhiSetupArgs {
    int n1, nm, nmp, nM;
    double kappa;
    const double* redge;
    double* phi;
    double* cz;             // [nM][nmp] zero right-hand side for the variants that read c
    double* res;
    double* u_used;
    double* bnorm;
};

struct MacroArgs {
    int NM, N1, nM, bc;
    double H, dt, Du, kappa;
    const double* gam;      // [nM] |Gamma_i|
    const double* cH;       // [nM] macro right-hand side without the coupling term
    const double* rho;      // [nM]
    double* uk;             // [nM] macro iterate (in: previous, out: new)
    double* u;              // [nM] committed state (written when the loop ends)
    double* x; double* r; double* z; double* zo; double* p; double* q;  // [nM] scratch
    double tol;
    int maxit;
    double coupling_tol;
    int coupling_maxit;
    int use_dct;            // fast-diagonalisation preconditioner (else Jacobi)
    int set_cond;           // call cudaGraphSetConditional
    cudaGraphConditionalHandle cond;
    DevCtl* ctl;
    int ncta;               // 1 (or 0): one thread block; kMacroCluster: one thread-block cluster
};
// CTAs of the cluster variant of the macro solve
constexpr int kMacroCluster = 8;

struct MacroPrologueArgs {
    int NM, N1, nM, bc, n1m;  // n1m: micro nodes per side (Robin edge length in nodes)
    double H, dt;
    const double* u;        // committed state u^n
    const double* fu;       // [nM] or nullptr
    const double* ud;       // [nM] or nullptr
    const double* g;        // [nM][n1m] Robin data or nullptr
    const double* redge;    // [nM][n1m]
    double* G;              // out: r_i^T g_i (compensated; 0 without g)
    double* cH;             // out
    double* uk;             // out: initial iterate (Dirichlet values applied)
    // pipelined elimination: rho_eff = rho_w + u gam_psi (fluxes of z = w + u psi)
    const double* rho_w;    // [nM] r^T w, or nullptr
    // column-strip kernels: rho_w is summed here from the ring of w (float
    // pairs) at slot (hist_step + 2) mod 3, the w the last solve pushed
    const float2* ring2;    // [3][nM][nmp] or nullptr
    int nmp;
    const double* gam_psi;  // [nM] r^T psi
    double* rho_eff;        // [nM] out
    DevCtl* ctl;
};

// ---------------------------------------------------------------------------
// Launchers (defined in the .cu files; all enqueue on `stream`)
// ---------------------------------------------------------------------------
// map32: [nM][8] FP32 copy of the whole map (A11, A12, A21, A22, b, c1, c2, 0) for the push-forward
cudaError_t launch_expand_params(int family, int nparam, const double* in, double* prm5, float* map32, int nM,
                                 cudaStream_t s);
// x_i = x0 + H (p, q); centre_mode 0: X = x_i + scale (chi - 1/2), 1: X = x_i + scale (chi - chi(1/2, 1/2))
cudaError_t launch_pushforward(int Nm, int n1, int nm, int nmp, int NM, int nM, const float* map32, const double* v,
                               float x0, float H, float scale, int centre_mode, float* out, cudaStream_t s);
cudaError_t launch_geometry(const GeomArgs& a, cudaStream_t s);
cudaError_t launch_instance_sums(int n1, int nm, int nmp, int nM, const double* lm, const double* redge,
                                 double* gam, double* vol, cudaStream_t s);
cudaError_t launch_micro_prologue(const PrologueArgs& a, cudaStream_t s);
cudaError_t launch_phi_setup(const PhiSetupArgs& a, cudaStream_t s);
// v_i += u_i phi_i on every micro DoF
cudaError_t launch_commit(int nm, int nmp, int nM, const double* u, const double* phi, double* v, cudaStream_t s);
// out = a - b elementwise
cudaError_t launch_sub(const double* a, const double* b, double* out, int n, cudaStream_t s);
// Micro-solve variants ("tilings"):
//   0..3   shared-memory stencil, K = 1, 2, 4, 8 nodes per thread (strided), FP64 or mixed
//   4..6   column strips of R = 3, 5, 7 nodes with register stencils, mixed only
//   7..9   column strips of R = 9, 11, 13 nodes with the stencil in shared memory, mixed only
//   10     the three-field system's direct micro solve (banded Cholesky, tsf_band.cu)
//   11..14 one micro problem per thread-block cluster of G CTAs, column strips of R rows,
//          (R, G) = (5, 2), (5, 4) with register stencils, (9, 4), (9, 8) with the stencil in
//          shared memory; mixed only
//   15, 16 one warp per micro problem (several per block), column strips of R = 3, 5 rows,
//          register stencils, for micro meshes whose strips fit 32 threads; mixed only
constexpr int kNumTilings = 17;
constexpr int kTilingDirect = 10;
constexpr int kFirstClusterTiling = 11;
constexpr int kNumClusterTilings = 4;
constexpr int kFirstWarpTiling = 15;
bool tiling_fits(int tiling, int precision, int n1, int smem_optin);
// column-strip kernels (tsf_strip.cu): strips of R = 3, 5, 7 (registers) or 9, 11, 13 (shared memory)
cudaError_t launch_strip_setup(const StripSetupArgs& a, cudaStream_t s);
cudaError_t launch_strip_solve(const MicroArgs& a, int R, cudaStream_t s);
bool strip_fits(int n1, int R, int smem_optin);
// cluster variants c = tiling - kFirstClusterTiling
cudaError_t launch_cluster_solve(const MicroArgs& a, int c, cudaStream_t s);
bool cluster_fits(int c, int n1, int smem_optin);
// Persistent micro solve of a batch of two-scale problems (pipelined
// elimination, column strips of R = 3 rows, or 5 where strips of 3 need more
// than 384 threads): per class of micro mesh (strip height, threads, staging)
// one launch of as many blocks as fit the GPU at once, each block one team of
// the column-strip solve; every block takes work items from its class's
// atomic queue, largest micro problems first.  An item is `count`
// consecutive micro problems of one problem instance.
constexpr int kBatchChunk = 4;             // micro problems per work item, before the last waves
constexpr size_t kBatchStaticSmem = 1024;  // bound on k_micro_batch's static shared memory
constexpr int kBatchMaxProblems = 64;      // problem instances of one persistent batch
constexpr int kBatchMaxClasses = 32;       // launches (classes of micro mesh) of one persistent step
struct BatchSolveArgs {
    // per-instance arguments (pipe = 1), in the kernel's parameter space: the
    // solves read them through the constant cache, as read-only data
    MicroArgs args[kBatchMaxProblems];
    const int4* items;                     // [nitems] (instance, first problem, count, 0)
    int nitems;
    int* counter;                          // queue head, zero before the launch
};
int batch_strip_R(int n1);                 // strip height for micro meshes of n1^2 nodes (3, 5; 0: too large)
int batch_threads(int n1, int R);          // threads of the block that solves one micro problem
bool batch_stages(int n1, int R);          // with the bulk-copy staging (as the single-problem kernel)
size_t batch_smem(int n1, int R, bool pref);  // dynamic shared memory of that block
cudaError_t launch_batch_solve(const BatchSolveArgs& b, int R, bool pref, int threads, size_t smem_bytes, int blocks,
                               int priority, cudaStream_t s);
const void* k_micro_batch_entry(int R, bool pref);  // the kernel, for its attributes and occupancy
// one-warp variants (R = 3, 5)
cudaError_t launch_warp_solve(const MicroArgs& a, int R, cudaStream_t s);
bool warp_fits(int n1, int R, int smem_optin);
cudaError_t configure_strip_kernels(int smem_optin);
// out[k] = the float pair nearest to in[k]
cudaError_t launch_split_pairs(const double* in, float2* out, size_t n, cudaStream_t s);
cudaError_t launch_micro_solve(const MicroArgs& a, int precision, int tiling, cudaStream_t s);
bool tiling_uses_stored_residual(int tiling);
cudaError_t launch_macro_prologue(const MacroPrologueArgs& a, cudaStream_t s);
// priority: 0 = the stream's; otherwise a launch priority (lower value = higher
// priority).  reserve_smem: dynamic shared memory to reserve (at least what
// the solve needs), so that a large value keeps other kernels' blocks off
// the macro solve's SM while it runs concurrently with them.
cudaError_t launch_macro_solve(const MacroArgs& a, cudaStream_t s, int priority = 0, size_t reserve_smem = 0);
size_t macro_smem_bytes(int N1, int bc, int use_dct);
bool macro_cluster_ok(int N1, int bc, int use_dct);
cudaError_t launch_vbar(int nm, int nmp, int nM, const double* lm, const double* vol, const double* v,
                        double* vbar, cudaStream_t s);
// flux_i = kappa (|Gam_i| u_i - rho_i) + r_i^T g_i and rho_i = r_i^T v_i (compensated); either output may be null
cudaError_t launch_flux(int n1, int nm, int nmp, int nM, double kappa, const double* gam, const double* u,
                        const double* v, const double* redge, const double* g, double* flux, double* rho,
                        cudaStream_t s);
cudaError_t configure_micro_kernels(int smem_optin);
cudaError_t configure_macro_kernels(int smem_optin);

// Pipelined exact elimination (tsf_elim.cu): the micro unknown of a step is
// split as z = w + u psi with psi = S^-1 (M phi / dt), so the micro solve for
// w of step k+1 needs only u^k and runs beside the macro solve of step k.
struct ElimArgs {
    int n1, nm, nmp, nM;
    double dt;
    const double* M64;
    const double* S64;
    const double* redge;
    const double* phi;      // [nM][nmp] S^-1 kappa r
    const double* psi;      // [nM][nmp] S^-1 mphi
    const double* mphi;     // [nM][nmp] M phi / dt
    const double* mpsi;     // [nM][nmp] M psi / dt
    const double* u;        // [nM] committed macro state
    double* u_old;          // [nM] the macro state the prepared w belongs to
    float2* u_old2;         // [nM] the same as float pairs (column-strip kernels)
    double* v;              // [nM][nmp] committed micro state
    double* W;              // [nM][nmp] unknown of the micro solve (warm start on entry)
    double* c;              // [nM][nmp] right-hand side of the w solve
    double* cnext;          // [nM][nmp] scratch: the next right-hand side
    double* res;            // [nM][nmp] stored residual of W
    double* u_used;         // [nM]
    double* bnorm;          // [nM][3]
    double* hist;           // [3][nM][nmp] ring of the last solves' w
    int commit_off;         // ring slot of w_k for the commit: (hist_step + commit_off) mod 3 (0: pushed
                            // by k_elim_pre in this step; 2: pushed by the previous solve's epilogue)
    // column-strip kernels (f2 = 1): the pipeline's arrays are float pairs
    int f2;
    float2* w2;             // [nM][nmp] warm start of the first w (head)
    float2* res2;           // [nM][nmp] its residual (head)
    float2* mw2;            // [nM][nmp] the first right-hand side (head)
    const float2* hist2;    // [3][nM][nmp] ring of w (commit)
    double* gtmp;           // [nM][nmp] scratch: the FP64 value of the warm-start pair (head)
    DevCtl* ctl;
};
cudaError_t launch_elim_head(const ElimArgs& a, cudaStream_t s);
cudaError_t launch_elim_start(const ElimArgs& a, cudaStream_t s);
cudaError_t launch_elim_pre(const ElimArgs& a, cudaStream_t s, int priority = 0);
cudaError_t launch_elim_commit(const ElimArgs& a, cudaStream_t s);
// out = M x / dt with x an [nM][nmp] field (norms of out: ||out||^2, out^T r, ||r||^2 into nrm)
cudaError_t launch_mass_dt(const ElimArgs& a, const double* x, double* out, double* nrm, cudaStream_t s);
// set-up of the solve S psi = mphi with the stored-residual protocol
cudaError_t launch_psi_setup(const ElimArgs& a, double* psi, double* cz, const double* mnorm, cudaStream_t s);

// Direct micro solves (tsf_band.cu): FP32 banded Cholesky factor of every
// micro operator, column k of instance i at L + (i nm + k)(n1 + 2):
// [1 / L_kk, L_{k+1,k}, ..., L_{k+n1+1,k}].
struct BandArgs {
    int n1, nm, nmp, nM;
    const float* S32;
    float* L;               // [nM][nm][n1 + 2]
    int* flag;              // set to 1 on a non-positive pivot
};
struct BandSolveArgs {      // x_t += L^-T L^-1 r_t for the right-hand sides not done
    int n1, nm, nmp, nM;
    const float* L;
    const double* r[3];     // [nM][nmp] residuals
    double* x[3];           // [nM][nmp] solutions, updated
    float* y[3];            // [nM][nmp] scratch
    const int* done[3];     // [nM] 1 = converged
};
struct BandResidualArgs {   // r_t = c_t - S x_t, done_t = ||r_t|| <= tol ||c_t||
    int n1, nm, nmp, nM, nrhs;
    double tol;
    const double* S64;
    const double* c[3];
    const double* x[3];
    double* r[3];
    const double* bnorm[3]; // [nM][3], ||c||^2 first
    int* done[3];
    int* open_count;        // += right-hand sides still open after this residual
    DevCtl* ctl;
};
size_t band_factor_smem(int n1);
cudaError_t launch_band_factor(const BandArgs& a, cudaStream_t s);
cudaError_t launch_band_solve(const BandSolveArgs& a, int nrhs, cudaStream_t s);
cudaError_t launch_band_residual(const BandResidualArgs& a, cudaStream_t s);

// discrete adjoint (tsf_adjoint.cu)
struct AdjAccArgs {
    int Nm, n1, nmp, nM;
    const double* nu;       // [nM][nmp] scaled adjoint micro state at step n+1
    const double* mu;       // [nM]      scaled adjoint macro state at step n+1
    const double* v1;       // [nM][nmp] forward micro state X^{n+1}
    const double* v0;       // [nM][nmp] forward micro state X^n
    const double* u1;       // [nM]      forward macro state at n+1
    double inv_dt;
    double* acc;            // [nM][Nm*Nm][4 qp][4]: s, T11, T12+T21, T22
    double* eacc;           // [nM][Nm][2 edge qp]
};
struct AdjGradArgs {
    int Nm, nM, NM, family, nparam;
    const double* prm5;
    double D11, D12, D22, kappa;
    const double* acc;
    const double* eacc;
    double* grad;           // [nM][nparam]
};
cudaError_t launch_adj_accumulate(const AdjAccArgs& a, cudaStream_t s);
cudaError_t launch_adj_gradient(const AdjGradArgs& a, cudaStream_t s);
cudaError_t launch_mean_u(const double* u, int nM, int NM, double* J, cudaStream_t s);
cudaError_t launch_fill(double* x, double val, size_t n, cudaStream_t s);

}  // namespace tsf
