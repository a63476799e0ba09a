// tsf_api.cu -- C ABI and host runtime of the GB300 two-scale library.
//
// Host responsibilities: validation of the inputs, one device workspace
// (caller-bound or self-allocated) carved into all arrays, rebuilding the
// pulled-back operators when the geometry, the physics or dt change, the
// choice of the micro-kernel tiling (measured on the actual problem), and the
// time step itself: a CUDA graph per dt whose coupling loop is a
// device-controlled conditional WHILE node (the macro kernel decides whether
// the Sec. 3.3 fixed-point iteration goes on), so one step costs one graph
// launch and no host round trip.
#include "tsfem.h"
#include "tsf_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

using namespace tsf;

namespace {

constexpr int kMaxNm = 128;    // micro cells per side (up to 64: one thread block per micro problem;
                               // beyond: one thread-block cluster per micro problem)
constexpr int kMaxNM = 1023;   // macro cells per side
constexpr size_t kAlign = 256;

struct Arena {
    size_t total = 0;
    size_t take(size_t bytes) {
        size_t o = total;
        total += (bytes + kAlign - 1) / kAlign * kAlign;
        return o;
    }
};

}  // namespace

struct tsf_ctx {
    tsf_options opt{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0;
    int smem_optin = 0;
    // meshes
    int Nm = 0, n1 = 0, nm = 0, nmp = 0;
    int NM = 0, N1 = 0, nM = 0, bc = 0;
    bool micro_set = false, macro_set = false;
    std::vector<double> dir_vals;
    // physics
    double D[3] = {1.0, 0.0, 1.0};
    double kappa = 1.0, Du = 1.0;
    // workspace
    unsigned char* ws = nullptr;
    size_t ws_bytes = 0;
    bool own_ws = false, ws_valid = false;
    // device arrays
    double *prm5 = nullptr, *M64 = nullptr, *S64 = nullptr, *lm = nullptr, *redge = nullptr, *Rd = nullptr,
           *Ru = nullptr, *gam = nullptr, *vol = nullptr;
    float* S32 = nullptr;
    // column-strip kernels: scaled operator, diagonal scalings, M/dt as FP32 pairs
    float4 *chat = nullptr, *chatlo = nullptr, *dsc = nullptr;
    float *Mh = nullptr, *Ml = nullptr;
    float2* mq2 = nullptr;       // [nM][nmp] M psi / dt as float pairs
    float2 *u_old2 = nullptr, *uzero2 = nullptr;  // [nM] u_old and zeros as float pairs
    double *v = nullptr, *c = nullptr, *vtmp = nullptr, *fv = nullptr, *g = nullptr, *G = nullptr;
    double *u = nullptr, *uk = nullptr, *cH = nullptr, *fu = nullptr, *ud = nullptr, *rho = nullptr,
           *out = nullptr;
    double *mx = nullptr, *mr = nullptr, *mz = nullptr, *mzo = nullptr, *mp = nullptr, *mq = nullptr;
    int macro_ncta = 1;          // CTAs of the macro solve (1 or kMacroCluster)
    double *res = nullptr, *res2 = nullptr, *u_used = nullptr, *uu2 = nullptr, *bnorm = nullptr;
    // exact elimination: phi_i = S_i^-1 kappa r_i, beta_i = r_i^T phi_i,
    // gam_eff = |Gam| - beta, constant macro vectors 0 and 1
    double *phi = nullptr, *beta = nullptr, *gam_eff = nullptr, *uzero = nullptr, *uone = nullptr;
    bool phi_valid = false;
    double* hist = nullptr;      // [3][nM][nmp] ring of the last solves' z (warm-start extrapolation)
    float* map32 = nullptr;      // [nM][8] FP32 copy of the deformation maps (push-forward)
    // pipelined elimination (tsf_elim.cu): z = w + u psi
    double *W = nullptr, *cnext = nullptr, *mphi = nullptr, *psi = nullptr, *mpsi = nullptr;  // [nM][nmp]
    double* yhist = nullptr;     // [3][nM][nmp] ring of S w of the last solves
    double *mnorm = nullptr;     // [nM][3] norms of M phi / dt
    double *u_old = nullptr, *gam_psi = nullptr, *rho_eff = nullptr;  // [nM]
    bool w_valid = false;        // W holds the solved w of the committed state
    bool extrap = true;          // pipelined elimination with extrapolated warm starts; off while the
                                 // adjoint replays states out of order
    cudaStream_t side = nullptr; // second stream of the pipelined step (prepares the next step)
    int prio_hi = 0, prio_lo = 0; // launch priorities: macro solve first, preparation after
    cudaEvent_t fork_ev = nullptr, join_ev = nullptr, mp_ev = nullptr, pre_ev = nullptr;
    int* inst_iters = nullptr;
    DevCtl* ctl = nullptr;
    DevCtl* ctl_host = nullptr;  // pinned
    // status of the contents
    bool geom_set = false, state_set = false;
    int family = 0;
    double ops_dt = -1.0;
    bool ops_valid = false;
    bool has_fv = false, has_g = false, has_fu = false, has_ud = false;
    int tiling = -1;             // micro-solve variant in use, -1 = not chosen
    int tiling_prec = -1;        // precision it was chosen for
    float tune_ms[kNumTilings] = {0};
    bool use_dct = false;
    // graph of one step; under the pipelined elimination a second one without
    // the commit of v (steps whose v nobody reads: all but the last of a call)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    cudaGraph_t graph_nc = nullptr;
    cudaGraphExec_t gexec_nc = nullptr;
    bool graph_valid = false;
    double graph_dt = -1.0;
    uint64_t graph_gen = 0;      // bumped whenever a captured step would go stale
    // per-launch CUDA-event timing of the plain-launch path (options.profile)
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    int64_t prof_micro_n = 0, prof_macro_n = 0;
    double prof_micro_ms = 0.0, prof_macro_ms = 0.0;
    std::string err;
};

static tsf_status fail(tsf_ctx* ctx, tsf_status st, const char* fmt, ...) {
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

#define CU(call)                                                                                         \
    do {                                                                                                 \
        cudaError_t e_ = (call);                                                                         \
        if (e_ != cudaSuccess)                                                                           \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? TSF_E_OOM : TSF_E_CUDA, "%s: %s (%s:%d)", \
                        #call, cudaGetErrorString(e_), __FILE__, __LINE__);                              \
    } while (0)

// Forget the warm-start history and the prepared w (after a new state, new
// sources or new operators).
static cudaError_t reset_history(tsf_ctx* ctx) {
    ctx->w_valid = false;
    cudaError_t e = cudaMemsetAsync(&ctx->ctl->hist_level, 0, sizeof(int), ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(&ctx->ctl->pushed, 0, sizeof(int), ctx->stream);
    return e;
}

static void invalidate_graph(tsf_ctx* ctx) {
    ctx->graph_gen++;
    if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
    if (ctx->graph) cudaGraphDestroy(ctx->graph);
    if (ctx->gexec_nc) cudaGraphExecDestroy(ctx->gexec_nc);
    if (ctx->graph_nc) cudaGraphDestroy(ctx->graph_nc);
    ctx->gexec = nullptr;
    ctx->graph = nullptr;
    ctx->gexec_nc = nullptr;
    ctx->graph_nc = nullptr;
    ctx->graph_valid = false;
}

static bool options_ok(const tsf_options* o) {
    return o && (o->precision == TSF_FP64 || o->precision == TSF_MIXED) && o->cg_tol >= 0 && o->inner_tol > 0 &&
           o->inner_tol < 1 && o->macro_tol >= 0 && o->coupling_tol >= 0 && o->cg_maxit > 0 && o->max_sweeps > 0 &&
           o->macro_maxit > 0 && o->coupling_maxit > 0 &&
           (o->coupling == TSF_COUPLING_PARTITIONED || o->coupling == TSF_COUPLING_ELIMINATION) &&
           (o->tiling == -1 || (o->tiling >= 0 && o->tiling < kNumTilings));
}

extern "C" {

int tsf_version(void) { return 100; }

void tsf_default_options(tsf_options* opt) {
    if (!opt) return;
    memset(opt, 0, sizeof *opt);
    opt->precision = TSF_MIXED;
    opt->cg_tol = 1e-8;
    opt->inner_tol = 1e-5;
    opt->macro_tol = 1e-12;
    opt->coupling_tol = 1e-10;
    opt->cg_maxit = 5000;
    opt->max_sweeps = 20;
    opt->macro_maxit = 500;
    opt->coupling_maxit = 50;
    opt->tiling = -1;
    opt->use_graph = 1;
    opt->cuda_stream = nullptr;
}

const char* tsf_last_error(const tsf_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

tsf_status tsf_create(tsf_ctx** out, const tsf_options* opt) {
    if (!out) return TSF_E_ARG;
    *out = nullptr;
    tsf_options o;
    tsf_default_options(&o);
    if (opt) o = *opt;
    if (!options_ok(&o)) return TSF_E_ARG;
    tsf_ctx* ctx = new (std::nothrow) tsf_ctx();
    if (!ctx) return TSF_E_OOM;
    ctx->opt = o;
    cudaError_t e = cudaGetDevice(&ctx->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device);
    if (e == cudaSuccess) {
        if (o.cuda_stream) {
            ctx->stream = (cudaStream_t)o.cuda_stream;
        } else {
            e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
            ctx->own_stream = (e == cudaSuccess);
        }
    }
    if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&ctx->prio_lo, &ctx->prio_hi);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&ctx->side, cudaStreamNonBlocking, ctx->prio_lo);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->fork_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->join_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->mp_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->pre_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = configure_micro_kernels(ctx->smem_optin);
    if (e == cudaSuccess) e = configure_macro_kernels(ctx->smem_optin);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&ctx->ctl_host, sizeof(DevCtl));
    if (e != cudaSuccess) {
        if (ctx->fork_ev) cudaEventDestroy(ctx->fork_ev);
        if (ctx->join_ev) cudaEventDestroy(ctx->join_ev);
        if (ctx->mp_ev) cudaEventDestroy(ctx->mp_ev);
        if (ctx->pre_ev) cudaEventDestroy(ctx->pre_ev);
        if (ctx->side) cudaStreamDestroy(ctx->side);
        if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
        delete ctx;
        return TSF_E_CUDA;
    }
    memset(ctx->ctl_host, 0, sizeof(DevCtl));
    *out = ctx;
    return TSF_OK;
}

tsf_status tsf_set_options(tsf_ctx* ctx, const tsf_options* opt) {
    if (!ctx) return TSF_E_ARG;
    if (!options_ok(opt)) return fail(ctx, TSF_E_ARG, "invalid options");
    void* keep = ctx->opt.cuda_stream;
    const bool prec_changed = opt->precision != ctx->opt.precision;
    ctx->opt = *opt;
    ctx->opt.cuda_stream = keep;
    if (prec_changed || opt->tiling >= 0) ctx->tiling = -1;
    ctx->phi_valid = false;
    invalidate_graph(ctx);
    return TSF_OK;
}

void tsf_destroy(tsf_ctx* ctx) {
    if (!ctx) return;
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    if (ctx->side) cudaStreamSynchronize(ctx->side);
    invalidate_graph(ctx);
    for (int k = 0; k < 4; ++k)
        if (ctx->ev[k]) cudaEventDestroy(ctx->ev[k]);
    if (ctx->fork_ev) cudaEventDestroy(ctx->fork_ev);
    if (ctx->join_ev) cudaEventDestroy(ctx->join_ev);
    if (ctx->mp_ev) cudaEventDestroy(ctx->mp_ev);
    if (ctx->pre_ev) cudaEventDestroy(ctx->pre_ev);
    if (ctx->side) cudaStreamDestroy(ctx->side);
    if (ctx->own_ws && ctx->ws) cudaFree(ctx->ws);
    if (ctx->ctl_host) cudaFreeHost(ctx->ctl_host);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

tsf_status tsf_set_micro_mesh(tsf_ctx* ctx, int nx, int ny, int robin_edge) {
    if (!ctx) return TSF_E_ARG;
    if (nx != ny || nx < 1 || nx > kMaxNm)
        return fail(ctx, TSF_E_ARG, "micro mesh must be square with 1..%d cells per side (got %d x %d)", kMaxNm, nx, ny);
    if (robin_edge != 0) return fail(ctx, TSF_E_ARG, "only robin_edge 0 (yhat_1 = 1) is supported");
    ctx->Nm = nx;
    ctx->n1 = nx + 1;
    ctx->nm = ctx->n1 * ctx->n1;
    ctx->nmp = (ctx->nm + 31) / 32 * 32;
    ctx->micro_set = true;
    ctx->ws_valid = false;
    ctx->geom_set = ctx->state_set = ctx->ops_valid = false;
    ctx->tiling = -1;
    invalidate_graph(ctx);
    return TSF_OK;
}

tsf_status tsf_set_macro_mesh(tsf_ctx* ctx, int nx, int ny, int bc, const double* dirichlet_vals) {
    if (!ctx) return TSF_E_ARG;
    if (nx != ny || nx < 1 || nx > kMaxNM)
        return fail(ctx, TSF_E_ARG, "macro mesh must be square with 1..%d cells per side (got %d x %d)", kMaxNM, nx, ny);
    if (bc != TSF_BC_NEUMANN && bc != TSF_BC_DIRICHLET) return fail(ctx, TSF_E_ARG, "bc must be 0 or 1");
    ctx->NM = nx;
    ctx->N1 = nx + 1;
    ctx->nM = ctx->N1 * ctx->N1;
    ctx->bc = bc;
    ctx->dir_vals.clear();
    if (dirichlet_vals) ctx->dir_vals.assign(dirichlet_vals, dirichlet_vals + ctx->nM);
    ctx->macro_set = true;
    ctx->ws_valid = false;
    ctx->geom_set = ctx->state_set = ctx->ops_valid = false;
    invalidate_graph(ctx);
    return TSF_OK;
}

tsf_status tsf_set_physics(tsf_ctx* ctx, const double D[3], double kappa, double macro_diff) {
    if (!ctx || !D) return TSF_E_ARG;
    if (!(D[0] > 0 && D[2] > 0 && D[0] * D[2] - D[1] * D[1] > 0))
        return fail(ctx, TSF_E_ARG, "D must be symmetric positive definite");
    if (!(kappa >= 0) || !(macro_diff > 0) || !std::isfinite(kappa) || !std::isfinite(macro_diff))
        return fail(ctx, TSF_E_ARG, "need kappa >= 0 and macro_diff > 0");
    ctx->D[0] = D[0];
    ctx->D[1] = D[1];
    ctx->D[2] = D[2];
    ctx->kappa = kappa;
    ctx->Du = macro_diff;
    ctx->ops_valid = false;
    invalidate_graph(ctx);
    return TSF_OK;
}

static void layout(tsf_ctx* ctx, Arena& A, size_t* off) {
    const size_t nM = ctx->nM, pl = ctx->nmp, n1 = ctx->n1;
    int k = 0;
    off[k++] = A.take(nM * 5 * sizeof(double));                  // prm5
    off[k++] = A.take(nM * kPlanes * pl * sizeof(double));       // M64
    off[k++] = A.take(nM * kPlanes * pl * sizeof(double));       // S64
    off[k++] = A.take(nM * kPlanes * pl * sizeof(float));        // S32
    off[k++] = A.take(nM * 2 * pl * sizeof(float4));             // chat
    off[k++] = A.take(nM * 2 * pl * sizeof(float4));             // chatlo
    off[k++] = A.take(nM * pl * sizeof(float4));                 // dsc
    off[k++] = A.take(nM * kPlanes * pl * sizeof(float));        // Mh
    off[k++] = A.take(nM * kPlanes * pl * sizeof(float));        // Ml
    off[k++] = A.take(nM * pl * sizeof(float2));                 // mq2
    off[k++] = A.take(nM * sizeof(float2));                      // u_old2
    off[k++] = A.take(nM * sizeof(float2));                      // uzero2
    off[k++] = A.take(nM * pl * sizeof(double));                 // lm
    off[k++] = A.take(nM * n1 * sizeof(double));                 // redge
    off[k++] = A.take(nM * n1 * sizeof(double));                 // Rd
    off[k++] = A.take(nM * n1 * sizeof(double));                 // Ru
    off[k++] = A.take(nM * sizeof(double));                      // gam
    off[k++] = A.take(nM * sizeof(double));                      // vol
    off[k++] = A.take(nM * pl * sizeof(double));                 // v
    off[k++] = A.take(nM * pl * sizeof(double));                 // c
    off[k++] = A.take(nM * pl * sizeof(double));                 // vtmp
    off[k++] = A.take(nM * pl * sizeof(double));                 // fv
    off[k++] = A.take(nM * n1 * sizeof(double));                 // g
    off[k++] = A.take(nM * sizeof(double));                      // G
    for (int r = 0; r < 13; ++r) off[k++] = A.take(nM * sizeof(double));  // u uk cH fu ud rho out mx mr mz mzo mp mq
    off[k++] = A.take(nM * pl * sizeof(double));                 // res
    off[k++] = A.take(nM * pl * sizeof(double));                 // res2 (tuning scratch)
    off[k++] = A.take(nM * sizeof(double));                      // u_used
    off[k++] = A.take(nM * sizeof(double));                      // uu2 (tuning scratch)
    off[k++] = A.take(nM * 3 * sizeof(double));                  // bnorm
    off[k++] = A.take(nM * sizeof(int));                         // inst_iters
    off[k++] = A.take(sizeof(DevCtl));                           // ctl
    off[k++] = A.take(nM * pl * sizeof(double));                 // phi
    for (int r = 0; r < 4; ++r) off[k++] = A.take(nM * sizeof(double));  // beta gam_eff uzero uone
    off[k++] = A.take(3 * nM * pl * sizeof(double));             // hist
    for (int r = 0; r < 5; ++r) off[k++] = A.take(nM * pl * sizeof(double));  // W cnext mphi psi mpsi
    off[k++] = A.take(3 * nM * pl * sizeof(double));             // yhist
    off[k++] = A.take(nM * 3 * sizeof(double));                  // mnorm
    off[k++] = A.take(nM * 8 * sizeof(float));                   // map32
    for (int r = 0; r < 3; ++r) off[k++] = A.take(nM * sizeof(double));  // u_old gam_psi rho_eff
}

static void assign(tsf_ctx* ctx, const size_t* off) {
    unsigned char* b = ctx->ws;
    int k = 0;
    ctx->prm5 = (double*)(b + off[k++]);
    ctx->M64 = (double*)(b + off[k++]);
    ctx->S64 = (double*)(b + off[k++]);
    ctx->S32 = (float*)(b + off[k++]);
    ctx->chat = (float4*)(b + off[k++]);
    ctx->chatlo = (float4*)(b + off[k++]);
    ctx->dsc = (float4*)(b + off[k++]);
    ctx->Mh = (float*)(b + off[k++]);
    ctx->Ml = (float*)(b + off[k++]);
    ctx->mq2 = (float2*)(b + off[k++]);
    ctx->u_old2 = (float2*)(b + off[k++]);
    ctx->uzero2 = (float2*)(b + off[k++]);
    ctx->lm = (double*)(b + off[k++]);
    ctx->redge = (double*)(b + off[k++]);
    ctx->Rd = (double*)(b + off[k++]);
    ctx->Ru = (double*)(b + off[k++]);
    ctx->gam = (double*)(b + off[k++]);
    ctx->vol = (double*)(b + off[k++]);
    ctx->v = (double*)(b + off[k++]);
    ctx->c = (double*)(b + off[k++]);
    ctx->vtmp = (double*)(b + off[k++]);
    ctx->fv = (double*)(b + off[k++]);
    ctx->g = (double*)(b + off[k++]);
    ctx->G = (double*)(b + off[k++]);
    double** r[13] = {&ctx->u, &ctx->uk, &ctx->cH, &ctx->fu, &ctx->ud, &ctx->rho, &ctx->out,
                      &ctx->mx, &ctx->mr, &ctx->mz, &ctx->mzo, &ctx->mp, &ctx->mq};
    for (int i = 0; i < 13; ++i) *r[i] = (double*)(b + off[k++]);
    ctx->res = (double*)(b + off[k++]);
    ctx->res2 = (double*)(b + off[k++]);
    ctx->u_used = (double*)(b + off[k++]);
    ctx->uu2 = (double*)(b + off[k++]);
    ctx->bnorm = (double*)(b + off[k++]);
    ctx->inst_iters = (int*)(b + off[k++]);
    ctx->ctl = (DevCtl*)(b + off[k++]);
    ctx->phi = (double*)(b + off[k++]);
    ctx->beta = (double*)(b + off[k++]);
    ctx->gam_eff = (double*)(b + off[k++]);
    ctx->uzero = (double*)(b + off[k++]);
    ctx->uone = (double*)(b + off[k++]);
    ctx->hist = (double*)(b + off[k++]);
    ctx->W = (double*)(b + off[k++]);
    ctx->cnext = (double*)(b + off[k++]);
    ctx->mphi = (double*)(b + off[k++]);
    ctx->psi = (double*)(b + off[k++]);
    ctx->mpsi = (double*)(b + off[k++]);
    ctx->yhist = (double*)(b + off[k++]);
    ctx->mnorm = (double*)(b + off[k++]);
    ctx->map32 = (float*)(b + off[k++]);
    ctx->u_old = (double*)(b + off[k++]);
    ctx->gam_psi = (double*)(b + off[k++]);
    ctx->rho_eff = (double*)(b + off[k++]);
}

static constexpr int kNumBuffers = 17 + 13 + 5 + 2 + 5 + 1 + 5 + 1 + 1 + 3 + 1 + 5 + 2;

tsf_status tsf_workspace_bytes(tsf_ctx* ctx, size_t* bytes) {
    if (!ctx || !bytes) return TSF_E_ARG;
    if (!ctx->micro_set || !ctx->macro_set) return fail(ctx, TSF_E_STATE, "set both meshes first");
    Arena A;
    size_t off[kNumBuffers];
    layout(ctx, A, off);
    *bytes = A.total;
    return TSF_OK;
}

static tsf_status init_workspace(tsf_ctx* ctx) {
    Arena A;
    size_t off[kNumBuffers];
    layout(ctx, A, off);
    assign(ctx, off);
    CU(cudaMemsetAsync(ctx->ctl, 0, sizeof(DevCtl), ctx->stream));
    CU(cudaMemsetAsync(ctx->u, 0, (size_t)ctx->nM * sizeof(double), ctx->stream));
    CU(cudaMemsetAsync(ctx->v, 0, (size_t)ctx->nM * ctx->nmp * sizeof(double), ctx->stream));
    CU(cudaMemsetAsync(ctx->G, 0, (size_t)ctx->nM * sizeof(double), ctx->stream));
    CU(launch_fill(ctx->uzero, 0.0, ctx->nM, ctx->stream));
    CU(launch_fill(ctx->uone, 1.0, ctx->nM, ctx->stream));
    CU(cudaMemsetAsync(ctx->uzero2, 0, (size_t)ctx->nM * sizeof(float2), ctx->stream));
    ctx->phi_valid = false;
    if (!ctx->dir_vals.empty())
        CU(cudaMemcpyAsync(ctx->ud, ctx->dir_vals.data(), ctx->nM * sizeof(double), cudaMemcpyHostToDevice,
                           ctx->stream));
    ctx->has_ud = !ctx->dir_vals.empty();
    ctx->has_fv = ctx->has_g = ctx->has_fu = false;
    ctx->geom_set = ctx->state_set = ctx->ops_valid = false;
    ctx->w_valid = false;
    ctx->ws_valid = true;
    invalidate_graph(ctx);
    return TSF_OK;
}

tsf_status tsf_bind_workspace(tsf_ctx* ctx, void* device_ptr, size_t bytes) {
    if (!ctx || !device_ptr) return TSF_E_ARG;
    size_t need = 0;
    tsf_status st = tsf_workspace_bytes(ctx, &need);
    if (st) return st;
    if (bytes < need) return fail(ctx, TSF_E_OOM, "workspace of %zu bytes < %zu needed", bytes, need);
    if (((uintptr_t)device_ptr) % kAlign) return fail(ctx, TSF_E_ARG, "workspace must be 256-byte aligned");
    cudaStreamSynchronize(ctx->stream);
    if (ctx->own_ws && ctx->ws) cudaFree(ctx->ws);
    ctx->ws = (unsigned char*)device_ptr;
    ctx->ws_bytes = bytes;
    ctx->own_ws = false;
    return init_workspace(ctx);
}

static tsf_status ensure_workspace(tsf_ctx* ctx) {
    if (!ctx->micro_set || !ctx->macro_set) return fail(ctx, TSF_E_STATE, "set both meshes first");
    if (ctx->ws_valid) return TSF_OK;
    size_t need = 0;
    tsf_workspace_bytes(ctx, &need);
    if (!ctx->ws || ctx->ws_bytes < need || !ctx->own_ws) {
        if (ctx->own_ws && ctx->ws) {
            cudaStreamSynchronize(ctx->stream);
            cudaFree(ctx->ws);
        }
        ctx->ws = nullptr;
        ctx->own_ws = false;
        cudaError_t e = cudaMalloc((void**)&ctx->ws, need);
        if (e != cudaSuccess) {
            ctx->ws = nullptr;
            cudaGetLastError();
            return fail(ctx, TSF_E_OOM, "cudaMalloc of %zu bytes failed: %s", need, cudaGetErrorString(e));
        }
        ctx->ws_bytes = need;
        ctx->own_ws = true;
    }
    return init_workspace(ctx);
}

static tsf_status copy_in(tsf_ctx* ctx, double* dst, const double* src, size_t n, int on_device) {
    CU(cudaMemcpyAsync(dst, src, n * sizeof(double), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                       ctx->stream));
    return TSF_OK;
}

// rows of nm values (caller, contiguous) <-> rows of nmp values (device, padded)
static tsf_status copy_field_in(tsf_ctx* ctx, double* dst, const double* src, int on_device) {
    CU(cudaMemcpy2DAsync(dst, ctx->nmp * sizeof(double), src, ctx->nm * sizeof(double), ctx->nm * sizeof(double),
                         ctx->nM, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->stream));
    return TSF_OK;
}

static tsf_status build_operators(tsf_ctx* ctx, double dt) {
    GeomArgs a{};
    a.affine = ctx->family == TSF_FAMILY_IDENTITY || ctx->family == TSF_FAMILY_AFFINE;
    a.Nm = ctx->Nm;
    a.n1 = ctx->n1;
    a.nm = ctx->nm;
    a.nmp = ctx->nmp;
    a.nM = ctx->nM;
    a.prm5 = ctx->prm5;
    a.D11 = ctx->D[0];
    a.D12 = ctx->D[1];
    a.D22 = ctx->D[2];
    a.kappa = ctx->kappa;
    a.dt = dt;
    a.M64 = ctx->M64;
    a.S64 = ctx->S64;
    a.S32 = ctx->S32;
    a.S32lo = nullptr;
    a.lm = ctx->lm;
    a.redge = ctx->redge;
    a.Rd = ctx->Rd;
    a.Ru = ctx->Ru;
    a.ctl = ctx->ctl;
    CU(launch_geometry(a, ctx->stream));
    CU(launch_instance_sums(ctx->n1, ctx->nm, ctx->nmp, ctx->nM, ctx->lm, ctx->redge, ctx->gam, ctx->vol,
                            ctx->stream));
    StripSetupArgs ss{};
    ss.n1 = ctx->n1;
    ss.nm = ctx->nm;
    ss.nmp = ctx->nmp;
    ss.nM = ctx->nM;
    ss.S64 = ctx->S64;
    ss.M64 = ctx->M64;
    ss.idt = 1.0 / dt;
    ss.rs = ctx->vtmp;  // scratch
    ss.chat = ctx->chat;
    ss.chatlo = ctx->chatlo;
    ss.dsc = ctx->dsc;
    ss.Mh = ctx->Mh;
    ss.Ml = ctx->Ml;
    CU(launch_strip_setup(ss, ctx->stream));
    ctx->ops_dt = dt;
    ctx->ops_valid = true;
    ctx->phi_valid = false;
    return TSF_OK;
}

tsf_status tsf_set_deformation(tsf_ctx* ctx, int family, int nparam, const double* params, int params_on_device) {
    if (!ctx) return TSF_E_ARG;
    static const int np_of[5] = {0, 1, 2, 6, 5};
    if (family < 0 || family > 4) return fail(ctx, TSF_E_ARG, "unknown deformation family %d", family);
    if (nparam != np_of[family])
        return fail(ctx, TSF_E_ARG, "family %d takes %d parameters per node (got %d)", family, np_of[family], nparam);
    if (nparam > 0 && !params) return fail(ctx, TSF_E_ARG, "params is NULL");
    tsf_status st = ensure_workspace(ctx);
    if (st) return st;
    if (nparam > 0) {
        // stage the raw parameters in the scratch field, then expand on the device
        st = copy_in(ctx, ctx->vtmp, params, (size_t)ctx->nM * nparam, params_on_device);
        if (st) return st;
    }
    CU(launch_expand_params(family, nparam, ctx->vtmp, ctx->prm5, ctx->map32, ctx->nM, ctx->stream));
    CU(cudaMemsetAsync(&ctx->ctl->geom_error, 0, sizeof(int), ctx->stream));
    ctx->family = family;   // before the operators: it selects the geometry kernel
    st = build_operators(ctx, 1.0);
    if (st) return st;
    int gerr = 0;
    CU(cudaMemcpyAsync(&gerr, &ctx->ctl->geom_error, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    invalidate_graph(ctx);
    if (gerr) {
        ctx->geom_set = false;
        ctx->ops_valid = false;
        return fail(ctx, TSF_E_BAD_JACOBIAN, "det F <= 0 at a quadrature point of some micro problem");
    }
    ctx->geom_set = true;
    return TSF_OK;
}

tsf_status tsf_set_state(tsf_ctx* ctx, const double* u, const double* v, int on_device) {
    if (!ctx || !u) return TSF_E_ARG;
    tsf_status st = ensure_workspace(ctx);
    if (st) return st;
    st = copy_in(ctx, ctx->u, u, ctx->nM, on_device);
    if (st) return st;
    if (v) {
        st = copy_field_in(ctx, ctx->v, v, on_device);
        if (st) return st;
    } else {
        CU(cudaMemsetAsync(ctx->v, 0, (size_t)ctx->nM * ctx->nmp * sizeof(double), ctx->stream));
    }
    CU(reset_history(ctx));
    ctx->state_set = true;
    return TSF_OK;
}

tsf_status tsf_set_sources(tsf_ctx* ctx, const double* fv, const double* g, const double* fu, const double* ud,
                           int on_device) {
    if (!ctx) return TSF_E_ARG;
    tsf_status st = ensure_workspace(ctx);
    if (st) return st;
    const bool before[4] = {ctx->has_fv, ctx->has_g, ctx->has_fu, ctx->has_ud};
    if (fv && (st = copy_field_in(ctx, ctx->fv, fv, on_device))) return st;
    if (g && (st = copy_in(ctx, ctx->g, g, (size_t)ctx->nM * ctx->n1, on_device))) return st;
    if (fu && (st = copy_in(ctx, ctx->fu, fu, ctx->nM, on_device))) return st;
    if (ud && (st = copy_in(ctx, ctx->ud, ud, ctx->nM, on_device))) return st;
    ctx->has_fv = fv != nullptr;
    ctx->has_g = g != nullptr;
    ctx->has_fu = fu != nullptr;
    ctx->has_ud = ud != nullptr;
    if (!ud && !ctx->dir_vals.empty()) {
        // no new values: fall back to the ones given with the macro mesh
        if ((st = copy_in(ctx, ctx->ud, ctx->dir_vals.data(), ctx->nM, 0))) return st;
        ctx->has_ud = true;
    }
    if (before[0] != ctx->has_fv || before[1] != ctx->has_g || before[2] != ctx->has_fu || before[3] != ctx->has_ud)
        invalidate_graph(ctx);
    if (before[0] != ctx->has_fv || before[1] != ctx->has_g) CU(reset_history(ctx));  // pipelining on or off
    return TSF_OK;
}

// ---------------------------------------------------------------------------
// the step
// ---------------------------------------------------------------------------
static MicroArgs micro_args(tsf_ctx* ctx, double* v) {
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
    a.c = ctx->c;
    a.v = v;
    a.u = ctx->uk;
    a.redge = ctx->redge;
    a.kappa = ctx->kappa;
    a.tol = ctx->opt.cg_tol;
    a.inner_tol = ctx->opt.inner_tol;
    a.maxit = ctx->opt.cg_maxit;
    a.max_sweeps = ctx->opt.max_sweeps;
    a.rho = ctx->rho;
    a.inst_iters = ctx->inst_iters;
    a.ctl = ctx->ctl;
    a.res = ctx->res;
    a.u_used = ctx->u_used;
    a.bnorm = ctx->bnorm;
    return a;
}

static MacroArgs macro_args(tsf_ctx* ctx, double dt, bool set_cond, cudaGraphConditionalHandle cond) {
    MacroArgs a{};
    a.NM = ctx->NM;
    a.N1 = ctx->N1;
    a.nM = ctx->nM;
    a.bc = ctx->bc;
    a.H = 1.0 / ctx->NM;
    a.dt = dt;
    a.Du = ctx->Du;
    a.kappa = ctx->kappa;
    a.gam = ctx->gam;
    a.cH = ctx->cH;
    a.rho = ctx->rho;
    a.uk = ctx->uk;
    a.u = ctx->u;
    a.x = ctx->mx;
    a.r = ctx->mr;
    a.z = ctx->mz;
    a.zo = ctx->mzo;
    a.p = ctx->mp;
    a.q = ctx->mq;
    a.tol = ctx->opt.macro_tol;
    a.maxit = ctx->opt.macro_maxit;
    a.coupling_tol = ctx->opt.coupling_tol;
    a.coupling_maxit = ctx->opt.coupling_maxit;
    a.use_dct = ctx->use_dct ? 1 : 0;
    a.set_cond = set_cond ? 1 : 0;
    a.cond = cond;
    a.ctl = ctx->ctl;
    a.ncta = ctx->macro_ncta;
    return a;
}

static bool eliminating(const tsf_ctx* ctx) { return ctx->opt.coupling == TSF_COUPLING_ELIMINATION; }

static tsf_status enqueue_macro_prologue(tsf_ctx* ctx, double dt, bool pipelined = false,
                                         cudaStream_t stream = nullptr) {
    MacroPrologueArgs m{};
    m.NM = ctx->NM;
    m.N1 = ctx->N1;
    m.nM = ctx->nM;
    m.bc = ctx->bc;
    m.n1m = ctx->n1;
    m.H = 1.0 / ctx->NM;
    m.dt = dt;
    m.u = ctx->u;
    m.fu = ctx->has_fu ? ctx->fu : nullptr;
    m.ud = ctx->has_ud ? ctx->ud : nullptr;
    m.g = ctx->has_g ? ctx->g : nullptr;
    m.redge = ctx->redge;
    m.G = ctx->G;
    m.cH = ctx->cH;
    m.uk = ctx->uk;
    m.ctl = ctx->ctl;
    if (pipelined) {
        m.rho_w = ctx->rho;
        m.gam_psi = ctx->gam_psi;
        m.rho_eff = ctx->rho_eff;
        if (tiling_uses_stored_residual(ctx->tiling)) {  // r^T w from the ring of the strip kernels
            m.ring2 = reinterpret_cast<const float2*>(ctx->hist);
            m.nmp = ctx->nmp;
        }
    }
    CU(launch_macro_prologue(m, stream ? stream : ctx->stream));
    return TSF_OK;
}

// Macro and micro prologues of a step.  With elim the micro prologue also
// replaces v by the warm start v - u phi of v0 (exact elimination).
static tsf_status enqueue_prologue(tsf_ctx* ctx, double dt, bool elim) {
    tsf_status st = enqueue_macro_prologue(ctx, dt);
    if (st) return st;
    PrologueArgs p{};
    p.n1 = ctx->n1;
    p.nm = ctx->nm;
    p.nmp = ctx->nmp;
    p.nM = ctx->nM;
    p.dt = dt;
    p.kappa = ctx->kappa;
    p.M64 = ctx->M64;
    p.S64 = ctx->S64;
    p.v = ctx->v;
    p.fv = ctx->has_fv ? ctx->fv : nullptr;
    p.g = ctx->has_g ? ctx->g : nullptr;
    p.redge = ctx->redge;
    p.Rd = ctx->Rd;
    p.Ru = ctx->Ru;
    p.u = ctx->uk;
    p.c = ctx->c;
    p.res = ctx->res;
    p.u_used = ctx->u_used;
    p.bnorm = ctx->bnorm;
    p.phi = elim ? ctx->phi : nullptr;
    p.uw = elim ? ctx->u : nullptr;
    CU(launch_micro_prologue(p, ctx->stream));
    return TSF_OK;
}

// One step by exact elimination: micro solve S v0 = c (u = 0 in the
// right-hand side), macro solve with the diagonal kappa m (|Gam| - beta) and
// the fluxes alpha = r^T v0, then v = v0 + u phi.  ev: optional events around
// the micro and macro solves.
static tsf_status enqueue_elimination_step(tsf_ctx* ctx, double dt, cudaEvent_t* ev) {
    tsf_status st = enqueue_prologue(ctx, dt, true);
    if (st) return st;
    if (ev) CU(cudaEventRecord(ev[0], ctx->stream));
    MicroArgs ma = micro_args(ctx, ctx->v);
    ma.u = ctx->uzero;
    CU(launch_micro_solve(ma, ctx->opt.precision, ctx->tiling, ctx->stream));
    if (ev) CU(cudaEventRecord(ev[1], ctx->stream));
    cudaGraphConditionalHandle none{};
    MacroArgs mg = macro_args(ctx, dt, false, none);
    mg.gam = ctx->gam_eff;
    mg.coupling_tol = HUGE_VAL;  // one macro solve ends the step
    mg.coupling_maxit = 1;
    CU(launch_macro_solve(mg, ctx->stream));
    if (ev) CU(cudaEventRecord(ev[2], ctx->stream));
    CU(launch_commit(ctx->nm, ctx->nmp, ctx->nM, ctx->u, ctx->phi, ctx->v, ctx->stream));
    return TSF_OK;
}

static ElimArgs elim_args(tsf_ctx* ctx, double dt) {
    ElimArgs a{};
    a.n1 = ctx->n1;
    a.nm = ctx->nm;
    a.nmp = ctx->nmp;
    a.nM = ctx->nM;
    a.dt = dt;
    a.M64 = ctx->M64;
    a.S64 = ctx->S64;
    a.redge = ctx->redge;
    a.phi = ctx->phi;
    a.psi = ctx->psi;
    a.mphi = ctx->mphi;
    a.mpsi = ctx->mpsi;
    a.u = ctx->u;
    a.u_old = ctx->u_old;
    a.u_old2 = tiling_uses_stored_residual(ctx->tiling) ? ctx->u_old2 : nullptr;
    a.v = ctx->v;
    a.W = ctx->W;
    a.c = ctx->c;
    a.cnext = ctx->cnext;
    a.res = ctx->res;
    a.u_used = ctx->u_used;
    a.bnorm = ctx->bnorm;
    a.hist = ctx->hist;
    a.commit_off = tiling_uses_stored_residual(ctx->tiling) ? 2 : 0;
    a.f2 = tiling_uses_stored_residual(ctx->tiling) ? 1 : 0;
    a.w2 = reinterpret_cast<float2*>(ctx->W);
    a.res2 = reinterpret_cast<float2*>(ctx->res);
    a.mw2 = reinterpret_cast<float2*>(ctx->cnext);
    a.hist2 = reinterpret_cast<const float2*>(ctx->hist);
    a.gtmp = ctx->vtmp;
    a.ctl = ctx->ctl;
    return a;
}

// The micro solve of w: u = 0 in the right-hand side.  The strip kernels run
// it pipelined (MicroArgs::pipe): they add u_old M psi / dt to the right-hand
// side and residual the previous solve left (zeros for the first w, whose
// right-hand side k_elim_head writes whole) and prepare the next step in
// their epilogue, in place of k_elim_pre.
static MicroArgs w_solve_args(tsf_ctx* ctx, double dt, bool head = false) {
    MicroArgs ma = micro_args(ctx, ctx->W);
    ma.u = ctx->uzero;
    (void)dt;
    if (tiling_uses_stored_residual(ctx->tiling)) {
        // the pipeline's arrays as float pairs (same 8 bytes per value as the
        // FP64 arrays they share memory with; k_elim_head writes them)
        ma.pipe = 1;
        ma.u_old2 = head ? ctx->uzero2 : ctx->u_old2;
        ma.w2 = reinterpret_cast<float2*>(ctx->W);
        ma.res2 = reinterpret_cast<float2*>(ctx->res);
        ma.mw2 = reinterpret_cast<float2*>(ctx->cnext);
        ma.mq2 = ctx->mq2;
        ma.hist2 = reinterpret_cast<float2*>(ctx->hist);
        ma.yhist2 = reinterpret_cast<float2*>(ctx->yhist);
        ma.Mh = ctx->Mh;
        ma.Ml = ctx->Ml;
    }
    return ma;
}

// Steps by pipelined elimination (tsf_elim.cu): eliminating, with warm-start
// history, and without volume or Robin sources (whose next values are not
// known one step ahead).
static bool pipelined(const tsf_ctx* ctx) {
    return eliminating(ctx) && ctx->extrap && !ctx->has_fv && !ctx->has_g;
}

// The first w from the committed state: k_elim_head and one micro solve.
static tsf_status enqueue_head(tsf_ctx* ctx, double dt) {
    const ElimArgs ea = elim_args(ctx, dt);
    CU(launch_elim_head(ea, ctx->stream));
    CU(launch_micro_solve(w_solve_args(ctx, dt, true), ctx->opt.precision, ctx->tiling, ctx->stream));
    return TSF_OK;
}

// One pipelined step (needs the solved w of the committed state):
//   k_elim_start
//   -> macro branch (this stream): macro prologue, macro solve, [after pre] commit
//   -> micro branch (side stream): k_elim_pre (not with the strip kernels),
//      [after the macro prologue] micro solve of the next w
//   -> join.
// ev: optional events around the micro solve (ev[0], ev[1], side stream) and
// the macro solve (ev[2], ev[3], this stream).
// commit = false leaves v as it was: within a run of pipelined steps nothing
// reads v (the micro solves work on w, the macro branch on the ring of w), so
// only the last step of a call has to write it.
static tsf_status enqueue_steady(tsf_ctx* ctx, double dt, cudaEvent_t* ev, bool commit = true) {
    const ElimArgs ea = elim_args(ctx, dt);
    CU(launch_elim_start(ea, ctx->stream));
    CU(cudaEventRecord(ctx->fork_ev, ctx->stream));
    CU(cudaStreamWaitEvent(ctx->side, ctx->fork_ev, 0));
    // micro branch (the strip kernels do k_elim_pre's work in the previous solve's epilogue)
    const bool fused = tiling_uses_stored_residual(ctx->tiling);
    if (!fused) {
        CU(launch_elim_pre(ea, ctx->side, ctx->prio_lo));
        CU(cudaEventRecord(ctx->pre_ev, ctx->side));
    }
    // macro branch: its prologue reads r^T w before the next solve rewrites it
    // (the strip kernels leave w in a ring slot the next solve does not touch,
    // and the prologue sums r^T w itself: their solve starts at once)
    tsf_status st = enqueue_macro_prologue(ctx, dt, true);
    if (st) return st;
    if (!fused) {
        CU(cudaEventRecord(ctx->mp_ev, ctx->stream));
        CU(cudaStreamWaitEvent(ctx->side, ctx->mp_ev, 0));
    }
    if (ev) CU(cudaEventRecord(ev[0], ctx->side));
    CU(launch_micro_solve(w_solve_args(ctx, dt), ctx->opt.precision, ctx->tiling, ctx->side));
    if (ev) CU(cudaEventRecord(ev[1], ctx->side));
    CU(cudaEventRecord(ctx->join_ev, ctx->side));
    cudaGraphConditionalHandle none{};
    MacroArgs mg = macro_args(ctx, dt, false, none);
    mg.gam = ctx->gam_eff;
    mg.rho = ctx->rho_eff;
    mg.coupling_tol = HUGE_VAL;  // one macro solve ends the step
    mg.coupling_maxit = 1;
    if (ev) CU(cudaEventRecord(ev[2], ctx->stream));
    // high priority: the one-block solve is scheduled beside the micro solve
    CU(launch_macro_solve(mg, ctx->stream, ctx->prio_hi));
    if (ev) CU(cudaEventRecord(ev[3], ctx->stream));
    if (!fused) CU(cudaStreamWaitEvent(ctx->stream, ctx->pre_ev, 0));
    if (commit) CU(launch_elim_commit(ea, ctx->stream));
    CU(cudaStreamWaitEvent(ctx->stream, ctx->join_ev, 0));
    return TSF_OK;
}

// the step of the elimination mode in use
static tsf_status enqueue_elim(tsf_ctx* ctx, double dt, cudaEvent_t* ev, bool commit = true) {
    return pipelined(ctx) ? enqueue_steady(ctx, dt, ev, commit) : enqueue_elimination_step(ctx, dt, ev);
}

static double phi_tol(double cg_tol) { return std::max(1e-3 * cg_tol, 1e-13); }

// phi_i = S_i^-1 kappa r_i for every micro problem (with the variant in use),
// beta_i = r_i^T phi_i and gam_eff = |Gam| - beta.  The counters of the
// control block are left as they were.
static tsf_status compute_phi(tsf_ctx* ctx) {
    DevCtl saved;
    CU(cudaMemcpyAsync(&saved, ctx->ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    PhiSetupArgs ps{};
    ps.n1 = ctx->n1;
    ps.nm = ctx->nm;
    ps.nmp = ctx->nmp;
    ps.nM = ctx->nM;
    ps.kappa = ctx->kappa;
    ps.redge = ctx->redge;
    ps.phi = ctx->phi;
    ps.cz = ctx->vtmp;
    ps.res = ctx->res;
    ps.u_used = ctx->u_used;
    ps.bnorm = ctx->bnorm;
    CU(launch_phi_setup(ps, ctx->stream));
    CU(cudaMemsetAsync(&ctx->ctl->status, 0, sizeof(int), ctx->stream));
    MicroArgs a = micro_args(ctx, ctx->phi);
    a.c = ctx->vtmp;
    a.u = ctx->uone;
    a.tol = phi_tol(ctx->opt.cg_tol);
    a.rho = ctx->beta;
    CU(launch_micro_solve(a, ctx->opt.precision, ctx->tiling, ctx->stream));
    CU(launch_sub(ctx->gam, ctx->beta, ctx->gam_eff, ctx->nM, ctx->stream));
    int status = 0;
    CU(cudaMemcpyAsync(&status, &ctx->ctl->status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    CU(cudaMemcpyAsync(ctx->ctl, &saved, sizeof(DevCtl), cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    if (status)
        return fail(ctx, (tsf_status)status, "solving for the elimination vectors S phi = kappa r failed (status %d)",
                    status);
    // psi = S^-1 (M phi / dt) for the pipelined steps, and M psi / dt
    const ElimArgs ea = elim_args(ctx, ctx->ops_dt);
    CU(launch_mass_dt(ea, ctx->phi, ctx->mphi, ctx->mnorm, ctx->stream));
    CU(launch_psi_setup(ea, ctx->psi, ctx->vtmp, ctx->mnorm, ctx->stream));
    MicroArgs b = micro_args(ctx, ctx->psi);
    b.c = ctx->vtmp;
    b.u = ctx->uzero;
    b.tol = phi_tol(ctx->opt.cg_tol);
    b.rho = ctx->gam_psi;
    CU(launch_micro_solve(b, ctx->opt.precision, ctx->tiling, ctx->stream));
    CU(launch_mass_dt(ea, ctx->psi, ctx->mpsi, nullptr, ctx->stream));
    CU(launch_split_pairs(ctx->mpsi, ctx->mq2, (size_t)ctx->nM * ctx->nmp, ctx->stream));
    CU(cudaMemcpyAsync(&status, &ctx->ctl->status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    CU(cudaMemcpyAsync(ctx->ctl, &saved, sizeof(DevCtl), cudaMemcpyHostToDevice, ctx->stream));
    if (status)
        return fail(ctx, (tsf_status)status, "solving for the elimination vectors S psi = M phi / dt failed (status %d)",
                    status);
    CU(reset_history(ctx));  // past w fields belong to the old phi and psi
    CU(cudaStreamSynchronize(ctx->stream));
    ctx->phi_valid = true;
    return TSF_OK;
}

// Choose the micro-solve variant by timing one solve of every admissible
// variant on the actual problem (right-hand side of the current step, warm
// start from the current state, results written to scratch copies).
static tsf_status autotune(tsf_ctx* ctx, double dt) {
    const int prec = ctx->opt.precision;
    if (ctx->opt.tiling >= 0) {
        if (!tiling_fits(ctx->opt.tiling, prec, ctx->n1, ctx->smem_optin))
            return fail(ctx, TSF_E_ARG, "tiling %d does not fit this micro mesh / precision", ctx->opt.tiling);
        ctx->tiling = ctx->opt.tiling;
        ctx->tiling_prec = prec;
        return TSF_OK;
    }
    DevCtl saved;
    CU(cudaMemcpyAsync(&saved, ctx->ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, ctx->stream));
    tsf_status st = enqueue_prologue(ctx, dt, false);
    if (st) return st;
    cudaEvent_t e0, e1;
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    float best = 1e30f;
    int best_t = -1;
    const size_t bytes = (size_t)ctx->nM * ctx->nmp * sizeof(double);
    for (int t = 0; t < kNumTilings; ++t) {
        if (!tiling_fits(t, prec, ctx->n1, ctx->smem_optin)) continue;
        MicroArgs a = micro_args(ctx, ctx->vtmp);
        a.res = ctx->res2;
        a.u_used = ctx->uu2;
        float ms = 0.f;
        for (int rep = 0; rep < 2; ++rep) {
            CU(cudaMemcpyAsync(ctx->vtmp, ctx->v, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
            CU(cudaMemcpyAsync(ctx->res2, ctx->res, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
            CU(cudaMemcpyAsync(ctx->uu2, ctx->u_used, ctx->nM * sizeof(double), cudaMemcpyDeviceToDevice,
                               ctx->stream));
            CU(cudaEventRecord(e0, ctx->stream));
            CU(launch_micro_solve(a, prec, t, ctx->stream));
            CU(cudaEventRecord(e1, ctx->stream));
            CU(cudaEventSynchronize(e1));
            CU(cudaEventElapsedTime(&ms, e0, e1));
        }
        ctx->tune_ms[t] = ms;
        if (ms < best) {
            best = ms;
            best_t = t;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CU(cudaMemcpyAsync(ctx->ctl, &saved, sizeof(DevCtl), cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    if (best_t < 0) return fail(ctx, TSF_E_ARG, "no micro-solve variant fits this mesh");
    // The variants are timed without the pipelined elimination's epilogue,
    // whose per-thread work grows with the strip height.  Eliminating, the
    // lowest short strip that fits is taken when a short strip won: with the
    // epilogue, R = 5 solves 48x48 micro cells 10 % faster than R = 7, and
    // R = 3 16x16 cells faster than R = 5 (on 32x32 cells R = 3 and R = 5
    // are within a few per cent of each other).
    if (eliminating(ctx) && best_t >= 4 && best_t <= 6) {
        for (int t = 4; t < best_t; ++t)
            if (tiling_fits(t, prec, ctx->n1, ctx->smem_optin)) {
                best_t = t;
                break;
            }
    }
    ctx->tiling = best_t;
    ctx->tiling_prec = prec;
    return TSF_OK;
}

// A capture that fails part-way can leave the graph (and the conditional
// node's body) in a state the runtime does not promise to destroy cleanly, so
// a failed capture abandons its graph instead of destroying it.
static tsf_status capture_failed(tsf_ctx* ctx, tsf_status st, cudaError_t e, const char* what) {
    ctx->graph = nullptr;
    ctx->gexec = nullptr;
    ctx->graph_nc = nullptr;
    ctx->gexec_nc = nullptr;
    ctx->graph_valid = false;
    cudaGetLastError();
    if (st) return st;
    return fail(ctx, TSF_E_CUDA, "graph capture failed at %s: %s", what, cudaGetErrorString(e));
}

// Appends one step of ctx to graph G as a branch that starts after the nodes
// dep[0..ndep) (none: a root branch): the macro and micro prologues, then a
// WHILE conditional node whose body is one coupling iteration (micro solve,
// macro solve; the macro kernel clears the condition when the coupling test
// passes), or the eliminated step (without the commit of v when commit is
// false and the steps are pipelined).  The branch's last nodes are appended to
// *tails when given.  On failure *what names the stage; the caller abandons G.
static cudaError_t capture_step_into(tsf_ctx* ctx, cudaGraph_t G, double dt, tsf_status* st, const char** what,
                                     const cudaGraphNode_t* dep = nullptr, size_t ndep = 0,
                                     std::vector<cudaGraphNode_t>* tails = nullptr, bool commit = true) {
    *st = TSF_OK;
    cudaError_t e;
    if (eliminating(ctx)) {  // the eliminated step: no coupling loop
        *what = "begin capture";
        e = cudaStreamBeginCaptureToGraph(ctx->stream, G, dep, nullptr, ndep, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return e;
        *st = enqueue_elim(ctx, dt, nullptr, commit);
        if (!*st && tails) {
            cudaStreamCaptureStatus cs;
            const cudaGraphNode_t* last = nullptr;
            size_t nlast = 0;
            e = cudaStreamGetCaptureInfo(ctx->stream, &cs, nullptr, nullptr, &last, nullptr, &nlast);
            if (e == cudaSuccess) tails->insert(tails->end(), last, last + nlast);
        }
        cudaGraph_t endg = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(ctx->stream, &endg);
        *what = "elimination step";
        if (*st) return cudaErrorUnknown;
        return e != cudaSuccess ? e : e2;
    }
    // (a conditional handle must belong to a conditional node of G)
    cudaGraphConditionalHandle cond;
    *what = "conditional handle";
    e = cudaGraphConditionalHandleCreate(&cond, G, 1, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) return e;
    *what = "begin capture";
    e = cudaStreamBeginCaptureToGraph(ctx->stream, G, dep, nullptr, ndep, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    *st = enqueue_prologue(ctx, dt, false);
    cudaStreamCaptureStatus cs;
    cudaGraph_t capg = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    e = cudaStreamGetCaptureInfo(ctx->stream, &cs, nullptr, &capg, &deps, nullptr, &ndeps);
    cudaGraphNode_t cnode = nullptr;
    cudaGraph_t body = nullptr;
    if (!*st && e == cudaSuccess) {
        alignas(cudaGraphNodeParams) unsigned char cpbuf[sizeof(cudaGraphNodeParams)];
        memset(cpbuf, 0, sizeof cpbuf);
        cudaGraphNodeParams& cp = *reinterpret_cast<cudaGraphNodeParams*>(cpbuf);
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = cond;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        e = cudaGraphAddNode(&cnode, capg, deps, nullptr, ndeps, &cp);
        if (e == cudaSuccess) {
            body = cp.conditional.phGraph_out[0];
            e = cudaStreamUpdateCaptureDependencies(ctx->stream, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies);
            if (tails) tails->push_back(cnode);
        }
    }
    cudaGraph_t endg = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(ctx->stream, &endg);
    *what = "prologue / conditional node";
    if (*st) return cudaErrorUnknown;
    if (e != cudaSuccess || e2 != cudaSuccess) return e != cudaSuccess ? e : e2;
    *what = "begin body capture";
    e = cudaStreamBeginCaptureToGraph(ctx->stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    MicroArgs ma = micro_args(ctx, ctx->v);
    e = launch_micro_solve(ma, ctx->opt.precision, ctx->tiling, ctx->stream);
    if (e == cudaSuccess) e = launch_macro_solve(macro_args(ctx, dt, true, cond), ctx->stream);
    e2 = cudaStreamEndCapture(ctx->stream, &body);
    *what = "body";
    return e != cudaSuccess ? e : e2;
}

static tsf_status capture_graph(tsf_ctx* ctx, double dt) {
    invalidate_graph(ctx);
    CU(cudaGraphCreate(&ctx->graph, 0));
    tsf_status st;
    const char* what;
    cudaError_t e = capture_step_into(ctx, ctx->graph, dt, &st, &what);
    if (e != cudaSuccess) return capture_failed(ctx, st, e, what);
    e = cudaGraphInstantiate(&ctx->gexec, ctx->graph, cudaGraphInstantiateFlagUseNodePriority);
    if (e != cudaSuccess) return capture_failed(ctx, TSF_OK, e, "instantiate");
    if (pipelined(ctx)) {
        CU(cudaGraphCreate(&ctx->graph_nc, 0));
        e = capture_step_into(ctx, ctx->graph_nc, dt, &st, &what, nullptr, 0, nullptr, false);
        if (e != cudaSuccess) return capture_failed(ctx, st, e, what);
        e = cudaGraphInstantiate(&ctx->gexec_nc, ctx->graph_nc, cudaGraphInstantiateFlagUseNodePriority);
        if (e != cudaSuccess) return capture_failed(ctx, TSF_OK, e, "instantiate");
    }
    ctx->graph_valid = true;
    ctx->graph_dt = dt;
    return TSF_OK;
}

// Operators for dt, macro preconditioner choice, micro variant (autotuned on
// first use): everything a step needs besides the state.
static tsf_status prepare_step(tsf_ctx* ctx, double dt) {
    if (!ctx->ops_valid || ctx->ops_dt != dt) {
        tsf_status st = build_operators(ctx, dt);
        if (st) return st;
        invalidate_graph(ctx);
    }
    ctx->use_dct = macro_smem_bytes(ctx->N1, ctx->bc, 1) <= (size_t)ctx->smem_optin;
    // The macro solve runs on one SM unless a cluster of kMacroCluster CTAs
    // pays: when it is on the step's critical path (the partitioned loop, the
    // unpipelined elimination, and pipelined steps whose micro solve is too
    // short to hide it).  Beside a long pipelined micro solve one block is
    // better: it takes one SM as soon as one frees, where a cluster would
    // wait for kMacroCluster of them.
    {
        const bool hidden = pipelined(ctx) && (double)ctx->nM * ctx->nm > 2e6;
        const int ncta = !hidden && macro_cluster_ok(ctx->N1, ctx->bc, ctx->use_dct) ? kMacroCluster : 1;
        if (ncta != ctx->macro_ncta) {
            ctx->macro_ncta = ncta;
            invalidate_graph(ctx);
        }
    }
    bool any = false;
    for (int t = 0; t < kNumTilings; ++t) any = any || tiling_fits(t, ctx->opt.precision, ctx->n1, ctx->smem_optin);
    if (!any)
        return fail(ctx, TSF_E_ARG, "no micro-solve variant fits %d micro cells per side in this precision%s", ctx->Nm,
                    ctx->opt.precision == TSF_FP64 && ctx->Nm > 64 ? " (above 64 cells only the mixed-precision "
                                                                      "cluster variants fit)" : "");
    if (ctx->tiling < 0 || ctx->tiling_prec != ctx->opt.precision) {
        tsf_status st = autotune(ctx, dt);
        if (st) return st;
        invalidate_graph(ctx);
    }
    if (eliminating(ctx) && !ctx->phi_valid) {
        tsf_status st = compute_phi(ctx);
        if (st) return st;
    }
    return TSF_OK;
}

// Steps with plain launches and a host-controlled coupling loop, on whatever
// arrays ctx->u / ctx->v point to.
static tsf_status run_plain_steps(tsf_ctx* ctx, double dt, int nsteps) {
    const bool prof = ctx->opt.profile != 0;
    if (prof && !ctx->ev[0])
        for (int k = 0; k < 4; ++k) CU(cudaEventCreate(&ctx->ev[k]));
    if (eliminating(ctx)) {
        const bool pipe = pipelined(ctx);
        for (int s = 0; s < nsteps; ++s) {
            tsf_status st = enqueue_elim(ctx, dt, prof ? ctx->ev : nullptr);
            if (st) return st;
            if (prof) {
                float a = 0.f, b = 0.f;
                CU(cudaStreamSynchronize(ctx->stream));
                CU(cudaEventElapsedTime(&a, ctx->ev[0], ctx->ev[1]));
                CU(cudaEventElapsedTime(&b, ctx->ev[pipe ? 2 : 1], ctx->ev[pipe ? 3 : 2]));
                ctx->prof_micro_ms += a;
                ctx->prof_macro_ms += b;
                ctx->prof_micro_n += 1;
                ctx->prof_macro_n += 1;
            }
        }
        return TSF_OK;
    }
    for (int s = 0; s < nsteps; ++s) {
        tsf_status st = enqueue_prologue(ctx, dt, false);
        if (st) return st;
        for (int it = 0; it < ctx->opt.coupling_maxit; ++it) {
            if (prof) CU(cudaEventRecord(ctx->ev[0], ctx->stream));
            CU(launch_micro_solve(micro_args(ctx, ctx->v), ctx->opt.precision, ctx->tiling, ctx->stream));
            if (prof) CU(cudaEventRecord(ctx->ev[1], ctx->stream));
            cudaGraphConditionalHandle none{};
            CU(launch_macro_solve(macro_args(ctx, dt, false, none), ctx->stream));
            if (prof) CU(cudaEventRecord(ctx->ev[2], ctx->stream));
            CU(cudaMemcpyAsync(&ctx->ctl_host->cont, &ctx->ctl->cont, sizeof(int), cudaMemcpyDeviceToHost,
                               ctx->stream));
            CU(cudaStreamSynchronize(ctx->stream));
            if (prof) {
                float a = 0.f, b = 0.f;
                CU(cudaEventElapsedTime(&a, ctx->ev[0], ctx->ev[1]));
                CU(cudaEventElapsedTime(&b, ctx->ev[1], ctx->ev[2]));
                ctx->prof_micro_ms += a;
                ctx->prof_macro_ms += b;
                ctx->prof_micro_n += 1;
                ctx->prof_macro_n += 1;
            }
            if (!ctx->ctl_host->cont) break;
        }
    }
    return TSF_OK;
}

tsf_status tsf_step(tsf_ctx* ctx, double dt, int nsteps) {
    if (!ctx) return TSF_E_ARG;
    if (!(dt > 0) || !std::isfinite(dt) || nsteps < 0) return fail(ctx, TSF_E_ARG, "need dt > 0 and nsteps >= 0");
    if (!ctx->ws_valid || !ctx->geom_set) return fail(ctx, TSF_E_STATE, "set meshes and deformation first");
    if (!ctx->state_set) return fail(ctx, TSF_E_STATE, "set the state first");
    if (nsteps == 0) return TSF_OK;
    tsf_status st = prepare_step(ctx, dt);
    if (st) return st;
    if (pipelined(ctx) && !ctx->w_valid) {  // the first w of this state
        if ((st = enqueue_head(ctx, dt))) return st;
        ctx->w_valid = true;
    }
    if (ctx->opt.use_graph) {
        if (!ctx->graph_valid || ctx->graph_dt != dt) {
            st = capture_graph(ctx, dt);
            if (st) return st;
        }
        for (int s = 0; s < nsteps; ++s)
            CU(cudaGraphLaunch(ctx->gexec_nc && s + 1 < nsteps ? ctx->gexec_nc : ctx->gexec, ctx->stream));
        return TSF_OK;
    }
    return run_plain_steps(ctx, dt, nsteps);
}

// ---------------------------------------------------------------------------
// Discrete adjoint of the march (kernels and derivation in tsf_adjoint.cu).
// Forward with checkpoints, then segment by segment backwards: recompute the
// segment's states from its checkpoint, step the scaled adjoint state with
// the forward solver (W A is symmetric), accumulate the gradient products.
// ---------------------------------------------------------------------------
tsf_status tsf_adjoint_mean_u(tsf_ctx* ctx, double dt, int nsteps, int ckpt_every, double* J_out, double* grad_out,
                              int on_device) {
    if (!ctx) return TSF_E_ARG;
    if (!(dt > 0) || !std::isfinite(dt) || nsteps < 1 || ckpt_every < 1)
        return fail(ctx, TSF_E_ARG, "need dt > 0, nsteps >= 1, ckpt_every >= 1");
    if (!ctx->ws_valid || !ctx->geom_set || !ctx->state_set)
        return fail(ctx, TSF_E_STATE, "set meshes, deformation and state first");
    if (ctx->bc != TSF_BC_NEUMANN) return fail(ctx, TSF_E_ARG, "the adjoint supports the Neumann macro boundary only");
    if (ctx->has_fv || ctx->has_g || ctx->has_fu)
        return fail(ctx, TSF_E_ARG, "the adjoint supports problems without sources only");
    static const int np_of[5] = {0, 1, 2, 6, 5};
    const int nparam = np_of[ctx->family];
    tsf_status st = prepare_step(ctx, dt);
    if (st) return st;
    const int K = ckpt_every, nck = (nsteps + K - 1) / K;
    const size_t nM = ctx->nM, nv = nM * ctx->nmp, ns = nM + nv;
    const size_t cells = (size_t)ctx->Nm * ctx->Nm;
    const size_t nacc = nM * cells * 16, nea = nM * (size_t)ctx->Nm * 2;
    const size_t total = (size_t)nck * ns + (size_t)(K + 1) * ns + 2 * ns + nacc + nea + nM * 6 + 8;
    double* buf = nullptr;
    cudaError_t e = cudaMalloc((void**)&buf, total * sizeof(double));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, TSF_E_OOM, "adjoint buffers (%zu bytes): %s", total * sizeof(double), cudaGetErrorString(e));
    }
    double* ck = buf;
    double* seg = ck + (size_t)nck * ns;
    double* lam = seg + (size_t)(K + 1) * ns;
    double* xN = lam + ns;
    double* acc = xN + ns;
    double* eacc = acc + nacc;
    double* grad = eacc + nea;
    double* Jd = grad + nM * 6;
    const int saved_graph = ctx->opt.use_graph;
    ctx->opt.use_graph = 0;
    ctx->extrap = false;  // the replayed steps start from checkpoints: no warm-start history
    invalidate_graph(ctx);
    double* const u_state = ctx->u;
    double* const v_state = ctx->v;
    auto save = [&](double* dst) -> tsf_status {
        CU(cudaMemcpyAsync(dst, ctx->u, nM * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
        CU(cudaMemcpyAsync(dst + nM, ctx->v, nv * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
        return TSF_OK;
    };
    auto load = [&](const double* src) -> tsf_status {
        CU(cudaMemcpyAsync(ctx->u, src, nM * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
        CU(cudaMemcpyAsync(ctx->v, src + nM, nv * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
        return TSF_OK;
    };
    auto adjoint_step = [&]() -> tsf_status {  // lam <- forward step of lam
        ctx->u = lam;
        ctx->v = lam + nM;
        tsf_status s2 = run_plain_steps(ctx, dt, 1);
        ctx->u = u_state;
        ctx->v = v_state;
        return s2;
    };
    auto body = [&]() -> tsf_status {
        // forward march with checkpoints
        for (int s = 0; s < nck; ++s) {
            tsf_status s2 = save(ck + (size_t)s * ns);
            if (s2) return s2;
            if ((s2 = run_plain_steps(ctx, dt, std::min(K, nsteps - s * K)))) return s2;
        }
        tsf_status s2 = save(xN);
        if (s2) return s2;
        CU(launch_mean_u(ctx->u, ctx->nM, ctx->NM, Jd, ctx->stream));
        // terminal adjoint: A lam~ = (m, 0) = B (dt 1, 0)
        CU(launch_fill(lam, dt, nM, ctx->stream));
        CU(launch_fill(lam + nM, 0.0, nv, ctx->stream));
        if ((s2 = adjoint_step())) return s2;
        CU(cudaMemsetAsync(acc, 0, (nacc + nea) * sizeof(double), ctx->stream));
        for (int s = nck - 1; s >= 0; --s) {
            const int n0 = s * K, nsg = std::min(K, nsteps - n0);
            CU(cudaMemcpyAsync(seg, ck + (size_t)s * ns, ns * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
            if ((s2 = load(seg))) return s2;
            for (int j = 1; j <= nsg; ++j) {
                if ((s2 = run_plain_steps(ctx, dt, 1))) return s2;
                if ((s2 = save(seg + (size_t)j * ns))) return s2;
            }
            for (int j = nsg - 1; j >= 0; --j) {
                if (n0 + j != nsteps - 1 && (s2 = adjoint_step())) return s2;
                AdjAccArgs aa{};
                aa.Nm = ctx->Nm;
                aa.n1 = ctx->n1;
                aa.nmp = ctx->nmp;
                aa.nM = ctx->nM;
                aa.nu = lam + nM;
                aa.mu = lam;
                aa.v1 = seg + (size_t)(j + 1) * ns + nM;
                aa.v0 = seg + (size_t)j * ns + nM;
                aa.u1 = seg + (size_t)(j + 1) * ns;
                aa.inv_dt = 1.0 / dt;
                aa.acc = acc;
                aa.eacc = eacc;
                CU(launch_adj_accumulate(aa, ctx->stream));
            }
        }
        if ((s2 = load(xN))) return s2;
        AdjGradArgs ga{};
        ga.Nm = ctx->Nm;
        ga.nM = ctx->nM;
        ga.NM = ctx->NM;
        ga.family = ctx->family;
        ga.nparam = nparam;
        ga.prm5 = ctx->prm5;
        ga.D11 = ctx->D[0];
        ga.D12 = ctx->D[1];
        ga.D22 = ctx->D[2];
        ga.kappa = ctx->kappa;
        ga.acc = acc;
        ga.eacc = eacc;
        ga.grad = grad;
        if (nparam > 0) CU(launch_adj_gradient(ga, ctx->stream));
        if (grad_out && nparam > 0)
            CU(cudaMemcpyAsync(grad_out, grad, nM * nparam * sizeof(double),
                               on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream));
        if (J_out)
            CU(cudaMemcpyAsync(J_out, Jd, sizeof(double), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                               ctx->stream));
        CU(cudaStreamSynchronize(ctx->stream));
        return TSF_OK;
    };
    st = body();
    ctx->u = u_state;
    ctx->v = v_state;
    ctx->opt.use_graph = saved_graph;
    ctx->extrap = true;
    reset_history(ctx);
    invalidate_graph(ctx);
    cudaStreamSynchronize(ctx->stream);
    cudaFree(buf);
    return st;
}

tsf_status tsf_synchronize(tsf_ctx* ctx) {
    if (!ctx) return TSF_E_ARG;
    CU(cudaStreamSynchronize(ctx->stream));
    if (!ctx->ws_valid) return TSF_OK;
    int status = 0;
    CU(cudaMemcpy(&status, &ctx->ctl->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (status) return fail(ctx, (tsf_status)status, "device reported status %d during the steps", status);
    return TSF_OK;
}

static tsf_status copy_out(tsf_ctx* ctx, double* dst, const double* src, size_t n, int on_device) {
    CU(cudaMemcpyAsync(dst, src, n * sizeof(double), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                       ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    return TSF_OK;
}

tsf_status tsf_get_macro(tsf_ctx* ctx, double* u_out, int on_device) {
    if (!ctx || !u_out) return TSF_E_ARG;
    if (!ctx->ws_valid) return fail(ctx, TSF_E_STATE, "no state");
    return copy_out(ctx, u_out, ctx->u, ctx->nM, on_device);
}

tsf_status tsf_get_macro_async(tsf_ctx* ctx, double* u_out, int on_device) {
    if (!ctx || !u_out) return TSF_E_ARG;
    if (!ctx->ws_valid) return fail(ctx, TSF_E_STATE, "no state");
    CU(cudaMemcpyAsync(u_out, ctx->u, ctx->nM * sizeof(double),
                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream));
    return TSF_OK;
}

tsf_status tsf_get_micro_field(tsf_ctx* ctx, double* v_out, int on_device) {
    if (!ctx || !v_out) return TSF_E_ARG;
    if (!ctx->ws_valid) return fail(ctx, TSF_E_STATE, "no state");
    CU(cudaMemcpy2DAsync(v_out, ctx->nm * sizeof(double), ctx->v, ctx->nmp * sizeof(double), ctx->nm * sizeof(double),
                         ctx->nM, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    return TSF_OK;
}

tsf_status tsf_get_micro_averages(tsf_ctx* ctx, double* vbar_out, int on_device) {
    if (!ctx || !vbar_out) return TSF_E_ARG;
    if (!ctx->ws_valid || !ctx->geom_set) return fail(ctx, TSF_E_STATE, "set meshes and deformation first");
    CU(launch_vbar(ctx->nm, ctx->nmp, ctx->nM, ctx->lm, ctx->vol, ctx->v, ctx->out, ctx->stream));
    return copy_out(ctx, vbar_out, ctx->out, ctx->nM, on_device);
}

// The averages go through the context's scratch vector; the next kernel that
// writes it is later on the same stream, so the queued copy reads this step's.
tsf_status tsf_get_micro_averages_async(tsf_ctx* ctx, double* vbar_out, int on_device) {
    if (!ctx || !vbar_out) return TSF_E_ARG;
    if (!ctx->ws_valid || !ctx->geom_set) return fail(ctx, TSF_E_STATE, "set meshes and deformation first");
    CU(launch_vbar(ctx->nm, ctx->nmp, ctx->nM, ctx->lm, ctx->vol, ctx->v, ctx->out, ctx->stream));
    CU(cudaMemcpyAsync(vbar_out, ctx->out, ctx->nM * sizeof(double),
                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream));
    return TSF_OK;
}

tsf_status tsf_get_flux(tsf_ctx* ctx, double* flux_out, int on_device) {
    if (!ctx || !flux_out) return TSF_E_ARG;
    if (!ctx->ws_valid || !ctx->geom_set) return fail(ctx, TSF_E_STATE, "set meshes and deformation first");
    if (!ctx->ops_valid) {
        tsf_status st = build_operators(ctx, ctx->ops_dt > 0 ? ctx->ops_dt : 1.0);
        if (st) return st;
    }
    CU(launch_flux(ctx->n1, ctx->nm, ctx->nmp, ctx->nM, ctx->kappa, ctx->gam, ctx->u, ctx->v, ctx->redge,
                   ctx->has_g ? ctx->g : nullptr, ctx->out, nullptr, ctx->stream));
    return copy_out(ctx, flux_out, ctx->out, ctx->nM, on_device);
}

tsf_status tsf_get_rho(tsf_ctx* ctx, double* rho_out, int on_device) {
    if (!ctx || !rho_out) return TSF_E_ARG;
    if (!ctx->ws_valid || !ctx->geom_set) return fail(ctx, TSF_E_STATE, "set meshes and deformation first");
    if (!ctx->ops_valid) {
        tsf_status st = build_operators(ctx, ctx->ops_dt > 0 ? ctx->ops_dt : 1.0);
        if (st) return st;
    }
    CU(launch_flux(ctx->n1, ctx->nm, ctx->nmp, ctx->nM, ctx->kappa, ctx->gam, ctx->u, ctx->v, ctx->redge, nullptr,
                   nullptr, ctx->out, ctx->stream));
    return copy_out(ctx, rho_out, ctx->out, ctx->nM, on_device);
}

tsf_status tsf_get_geometry(tsf_ctx* ctx, double* gamma_out, double* vol_out, int on_device) {
    if (!ctx) return TSF_E_ARG;
    if (!ctx->ws_valid || !ctx->geom_set) return fail(ctx, TSF_E_STATE, "set meshes and deformation first");
    tsf_status st = TSF_OK;
    if (gamma_out && (st = copy_out(ctx, gamma_out, ctx->gam, ctx->nM, on_device))) return st;
    if (vol_out && (st = copy_out(ctx, vol_out, ctx->vol, ctx->nM, on_device))) return st;
    return TSF_OK;
}

tsf_status tsf_get_pushforward(tsf_ctx* ctx, float scale, float* out, int on_device) {
    if (!ctx || !out) return TSF_E_ARG;
    if (!(scale > 0.0f) || !std::isfinite(scale)) return fail(ctx, TSF_E_ARG, "scale must be positive");
    if (!ctx->ws_valid || !ctx->geom_set) return fail(ctx, TSF_E_STATE, "set meshes and deformation first");
    const size_t n = (size_t)ctx->nM * ctx->nm * 3;
    float* dst = out;
    if (!on_device) {
        cudaError_t e = cudaMalloc((void**)&dst, n * sizeof(float));
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(ctx, TSF_E_OOM, "cudaMalloc of %zu bytes for the push-forward failed", n * sizeof(float));
        }
    }
    cudaError_t e = launch_pushforward(ctx->Nm, ctx->n1, ctx->nm, ctx->nmp, ctx->NM, ctx->nM, ctx->map32, ctx->v,
                                       0.0f, 1.0f / ctx->NM, scale, 0, dst, ctx->stream);
    if (e == cudaSuccess && !on_device)
        e = cudaMemcpyAsync(out, dst, n * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (!on_device) cudaFree(dst);
    if (e != cudaSuccess) return fail(ctx, TSF_E_CUDA, "push-forward: %s", cudaGetErrorString(e));
    return TSF_OK;
}

tsf_status tsf_get_stats(tsf_ctx* ctx, tsf_stats* out) {
    if (!ctx || !out) return TSF_E_ARG;
    memset(out, 0, sizeof *out);
    out->tiling = ctx->tiling;
    out->micro_launches = ctx->prof_micro_n;
    out->macro_launches = ctx->prof_macro_n;
    out->micro_kernel_ms = ctx->prof_micro_ms;
    out->macro_kernel_ms = ctx->prof_macro_ms;
    if (!ctx->ws_valid) return TSF_OK;
    CU(cudaMemcpyAsync(ctx->ctl_host, ctx->ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    const DevCtl& c = *ctx->ctl_host;
    out->inner_iters = (int64_t)c.inner_iters;
    out->dof_cg_iters = (int64_t)c.inner_iters * ctx->nm;
    out->refine_sweeps = (int64_t)c.sweeps;
    out->micro_solves = (int64_t)c.micro_solves;
    out->macro_iters = (int64_t)c.macro_iters;
    out->coupling_iters_last = c.coupling_iters_last;
    out->coupling_iters_total = c.coupling_iters_total;
    out->max_inner_iters = c.max_inner;
    out->steps = c.steps;
    out->status = c.status;
    out->coupling_change = c.change;
    return TSF_OK;
}

tsf_status tsf_reset_stats(tsf_ctx* ctx) {
    if (!ctx) return TSF_E_ARG;
    ctx->prof_micro_n = ctx->prof_macro_n = 0;
    ctx->prof_micro_ms = ctx->prof_macro_ms = 0.0;
    if (!ctx->ws_valid) return TSF_OK;
    // keep geom_error, coupling_iter, cont; clear the counters and the status
    CU(cudaMemsetAsync(ctx->ctl, 0, offsetof(DevCtl, coupling_iter), ctx->stream));
    const int zero4[4] = {0, 0, 0, 0};
    CU(cudaMemcpyAsync(&ctx->ctl->coupling_iters_total, zero4, 4 * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaMemcpyAsync(&ctx->ctl->steps, zero4, sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    return TSF_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batches of independent two-scale problems.  Each instance is an ordinary
// context on the batch's stream; a batch step is one CUDA graph holding one
// independent branch per instance (prologues, then that instance's own
// device-controlled coupling loop), so the instances' micro and macro
// kernels run concurrently and small instances fill the SMs that large ones
// leave idle.
// ---------------------------------------------------------------------------
struct tsf_batch {
    std::vector<tsf_ctx*> inst;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int use_graph = 1;
    // persistent mode: per step one launch of k_micro_batch for each class
    // of micro mesh, for the micro solves of all instances (the device table
    // of the work items, the queue heads)
    int persistent = 0;
    int4* d_items = nullptr;
    int* d_counter = nullptr;          // [kBatchMaxClasses] queue heads
    size_t cap_items = 0;
    int nitems = 0;
    // the classes' launches run side by side: streams and events of the
    // fork and the join (the first path runs on the batch's stream)
    cudaStream_t kside[kBatchMaxClasses - 1] = {};
    cudaEvent_t kfork = nullptr;
    cudaEvent_t kjoin[kBatchMaxClasses - 1] = {};
    int nlaunch = 0;                   // persistent micro-solve launches of the captured step
    cudaGraph_t graph = nullptr;       // one batch step
    cudaGraphExec_t gexec = nullptr;
    cudaGraph_t graph_nc = nullptr;    // the same without the commits of v (all but a call's last step)
    cudaGraphExec_t gexec_nc = nullptr;
    bool graph_valid = false;
    double graph_dt = -1.0;
    std::vector<uint64_t> gen;   // instance graph generations the graph was captured at
    int steps = 0;
    std::string err;
};

static tsf_status bfail(tsf_batch* b, tsf_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    b->err = buf;
    return st;
}

static void batch_drop_graph(tsf_batch* b, bool destroy) {
    if (destroy) {
        if (b->gexec) cudaGraphExecDestroy(b->gexec);
        if (b->graph) cudaGraphDestroy(b->graph);
        if (b->gexec_nc) cudaGraphExecDestroy(b->gexec_nc);
        if (b->graph_nc) cudaGraphDestroy(b->graph_nc);
    }
    b->gexec = nullptr;
    b->graph = nullptr;
    b->gexec_nc = nullptr;
    b->graph_nc = nullptr;
    b->graph_valid = false;
}

// An instance error is reported with the instance's index and message.
static tsf_status inst_fail(tsf_batch* b, int i, tsf_status st) {
    return bfail(b, st, "instance %d: %s", i, b->inst[i]->err.c_str());
}

// One batch step as one graph.  Problems with the same micro mesh and
// variant run as concurrent branches; these groups run one after another,
// largest micro mesh first.  Blocks of different variants (registers, shared
// memory, threads) pack an SM badly when they run together: on the 32-problem
// uneven workload one phase per micro mesh was 5 % faster than all branches at
// once.
static tsf_status batch_capture_one(tsf_batch* b, double dt, bool commit, cudaGraph_t& G, cudaGraphExec_t& X) {
    cudaError_t e = cudaGraphCreate(&G, 0);
    if (e != cudaSuccess) return bfail(b, TSF_E_CUDA, "cudaGraphCreate: %s", cudaGetErrorString(e));
    const int n = (int)b->inst.size();
    std::vector<int> order(n);
    for (int k = 0; k < n; ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        const tsf_ctx *cx = b->inst[x], *cy = b->inst[y];
        return cx->n1 != cy->n1 ? cx->n1 > cy->n1 : cx->tiling < cy->tiling;
    });
    cudaGraphNode_t join = nullptr;  // end of the previous group
    std::vector<cudaGraphNode_t> tails;
    for (int a = 0; a < n;) {
        int z = a;
        while (z < n && b->inst[order[z]]->n1 == b->inst[order[a]]->n1 &&
               b->inst[order[z]]->tiling == b->inst[order[a]]->tiling)
            ++z;
        tails.clear();
        for (int m = a; m < z; ++m) {
            const int i = order[m];
            tsf_status st;
            const char* what;
            e = capture_step_into(b->inst[i], G, dt, &st, &what, join ? &join : nullptr, join ? 1 : 0, &tails,
                                  commit);
            if (e != cudaSuccess) {
                batch_drop_graph(b, false);  // abandoned, as for a single context
                cudaGetLastError();
                if (st) return inst_fail(b, i, st);
                return bfail(b, TSF_E_CUDA, "instance %d: graph capture failed at %s: %s", i, what,
                             cudaGetErrorString(e));
            }
        }
        if (z < n) {
            e = cudaGraphAddEmptyNode(&join, G, tails.data(), tails.size());
            if (e != cudaSuccess) {
                batch_drop_graph(b, false);
                cudaGetLastError();
                return bfail(b, TSF_E_CUDA, "batch graph: %s", cudaGetErrorString(e));
            }
        }
        a = z;
    }
    e = cudaGraphInstantiate(&X, G, cudaGraphInstantiateFlagUseNodePriority);
    if (e != cudaSuccess) {
        batch_drop_graph(b, false);
        cudaGetLastError();
        return bfail(b, TSF_E_CUDA, "batch graph instantiate: %s", cudaGetErrorString(e));
    }
    return TSF_OK;
}

// The variant whose arithmetic the persistent batch kernel runs for an
// instance: column strips of 3 rows (tiling 4), or of 5 (tiling 5) where strips
// of 3 need more than 384 threads.
static int persistent_tiling(const tsf_ctx* c) { return batch_strip_R(c->n1) == 3 ? 4 : 5; }

// Every micro solve of an instance in a persistent batch (its head solves
// and set-up solves included) runs that variant.
static void use_persistent_tiling(tsf_ctx* c) {
    const int t = persistent_tiling(c);
    if (c->opt.tiling != t) {
        c->opt.tiling = t;
        c->tiling = -1;
        c->phi_valid = false;
        invalidate_graph(c);
    }
}

static tsf_status batch_capture(tsf_batch* b, double dt) {
    batch_drop_graph(b, true);
    tsf_status st = batch_capture_one(b, dt, true, b->graph, b->gexec);
    if (!st) st = batch_capture_one(b, dt, false, b->graph_nc, b->gexec_nc);
    if (st) return st;
    b->gen.resize(b->inst.size());
    for (size_t i = 0; i < b->inst.size(); ++i) b->gen[i] = b->inst[i]->graph_gen;
    b->graph_valid = true;
    b->graph_dt = dt;
    return TSF_OK;
}

// The persistent batch step (pipelined elimination of every instance):
//   per instance, on its side stream: k_elim_start (the macro state the next w
//   belongs to), the macro prologue, then the macro solve (high priority) and,
//   in a call's last step, the commit;
//   once every prologue is done: the persistent launches of k_micro_batch,
//   one per class of micro mesh (strip height, threads, staging), side by
//   side at the lowest priority, which solve the next w of every micro problem
//   of every instance from work queues ordered largest micro problem first.
//   The micro launches wait for the prologues so that the macro solves, ready
//   at the same time or earlier and of higher priority, take their SMs first:
//   the persistent blocks leave an SM only when their queue is drained.
static tsf_status batch_capture_persistent(tsf_batch* b, double dt) {
    batch_drop_graph(b, true);
    const int n = (int)b->inst.size();
    if (n > kBatchMaxProblems)
        return bfail(b, TSF_E_ARG, "the persistent batch takes at most %d problems (%d given)", kBatchMaxProblems, n);
    std::vector<MicroArgs> args(n);
    std::vector<int> order(n);
    for (int k = 0; k < n; ++k) {
        tsf_ctx* c = b->inst[k];
        args[k] = with_fp32_tols(w_solve_args(c, dt));
        order[k] = k;
    }
    // largest micro problems first (work per problem grows with n1^2), then
    // the instances with more micro problems
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        const tsf_ctx *cx = b->inst[x], *cy = b->inst[y];
        return cx->nm != cy->nm ? cx->nm > cy->nm : cx->nM > cy->nM;
    });
    // the classes, in the order of their largest micro mesh
    struct Class {
        int R, threads;
        bool pref;
        size_t smem;
        long problems;
        int grid;
        std::vector<int4> items;
    };
    std::vector<Class> cls;
    std::vector<int> cof(n);
    tsf_ctx* c0 = b->inst[0];
    for (int k : order) {
        tsf_ctx* c = b->inst[k];
        const int R = batch_strip_R(c->n1);
        if (!R)
            return bfail(b, TSF_E_ARG, "instance %d: %d micro cells per side are too many for the persistent batch",
                         k, c->Nm);
        const int T = batch_threads(c->n1, R);
        const bool pref = batch_stages(c->n1, R);
        int q = 0;
        while (q < (int)cls.size() && !(cls[q].R == R && cls[q].threads == T && cls[q].pref == pref)) ++q;
        if (q == (int)cls.size()) {
            if (q == kBatchMaxClasses)
                return bfail(b, TSF_E_ARG, "the persistent batch takes micro meshes of at most %d classes",
                             kBatchMaxClasses);
            cls.push_back(Class{R, T, pref, 0, 0, 0, {}});
        }
        cls[q].smem = std::max(cls[q].smem, batch_smem(c->n1, R, pref));
        cls[q].problems += c->nM;
        cof[k] = q;
    }
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c0->device);
    cudaError_t e = cudaSuccess;
    // each kernel's shared-memory limit: the largest of the classes it serves
    for (const Class& q : cls) {
        if (q.smem + kBatchStaticSmem > (size_t)c0->smem_optin)
            return bfail(b, TSF_E_ARG, "persistent batch: shared memory %zu > %d", q.smem, c0->smem_optin);
        size_t most = 0;
        for (const Class& o : cls)
            if (o.R == q.R && o.pref == q.pref) most = std::max(most, o.smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_micro_batch_entry(q.R, q.pref), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)most);
    }
    for (Class& q : cls) {
        int per_sm = 0;
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_micro_batch_entry(q.R, q.pref), q.threads,
                                                              q.smem);
        q.grid = (int)std::min<long>((long)std::max(per_sm, 1) * nsm, q.problems);
    }
    // the items: kBatchChunk micro problems each, one each in the last two
    // waves of the class's queue, where long items would leave SMs idle
    for (int k : order) {
        tsf_ctx* c = b->inst[k];
        Class& q = cls[cof[k]];
        for (int i = 0; i < c->nM;) {
            const int chunk = q.problems > 2L * q.grid * kBatchChunk ? kBatchChunk : 1;
            const int cnt = std::min(chunk, c->nM - i);
            q.items.push_back(make_int4(k, i, cnt, 0));
            i += cnt;
            q.problems -= cnt;
        }
    }
    std::vector<int4> items;
    std::vector<int> koff;
    for (const Class& q : cls) {
        koff.push_back((int)items.size());
        items.insert(items.end(), q.items.begin(), q.items.end());
    }
    if (e == cudaSuccess && b->cap_items < items.size()) {
        if (b->d_items) cudaFree(b->d_items);
        e = cudaMalloc((void**)&b->d_items, items.size() * sizeof(int4));
        b->cap_items = e == cudaSuccess ? items.size() : 0;
    }
    if (e == cudaSuccess && !b->d_counter) e = cudaMalloc((void**)&b->d_counter, kBatchMaxClasses * sizeof(int));
    for (int k = 0; k + 1 < (int)cls.size() && e == cudaSuccess; ++k) {  // (kept for later captures)
        if (!b->kside[k]) e = cudaStreamCreateWithFlags(&b->kside[k], cudaStreamNonBlocking);
        if (e == cudaSuccess && !b->kjoin[k]) e = cudaEventCreateWithFlags(&b->kjoin[k], cudaEventDisableTiming);
    }
    if (e == cudaSuccess && !b->kfork) e = cudaEventCreateWithFlags(&b->kfork, cudaEventDisableTiming);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_items, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return bfail(b, e == cudaErrorMemoryAllocation ? TSF_E_OOM : TSF_E_CUDA, "persistent batch set-up: %s",
                     cudaGetErrorString(e));
    }
    b->nitems = (int)items.size();
    b->nlaunch = (int)cls.size();

    cudaStream_t s = b->stream;
    // capture one batch step into G (with or without the commits of v)
    auto capture = [&](bool commit, cudaGraph_t& G, cudaGraphExec_t& X) -> tsf_status {
        cudaError_t er = cudaGraphCreate(&G, 0);
        if (er != cudaSuccess) return bfail(b, TSF_E_CUDA, "cudaGraphCreate: %s", cudaGetErrorString(er));
        tsf_status st = TSF_OK;
        er = cudaStreamBeginCaptureToGraph(s, G, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (er == cudaSuccess) {
            er = cudaEventRecord(c0->fork_ev, s);
            for (int k = 0; k < n && er == cudaSuccess; ++k) {
                tsf_ctx* c = b->inst[k];
                er = cudaStreamWaitEvent(c->side, c0->fork_ev, 0);
                if (er == cudaSuccess) er = launch_elim_start(elim_args(c, dt), c->side);
                if (er != cudaSuccess) break;
                if ((st = enqueue_macro_prologue(c, dt, true, c->side))) {
                    er = cudaErrorUnknown;  // (the capture is still ended below)
                    break;
                }
                er = cudaEventRecord(c->pre_ev, c->side);
                cudaGraphConditionalHandle none{};
                MacroArgs mg = macro_args(c, dt, false, none);
                mg.gam = c->gam_eff;
                mg.rho = c->rho_eff;
                mg.coupling_tol = HUGE_VAL;
                mg.coupling_maxit = 1;
                if (er == cudaSuccess) er = launch_macro_solve(mg, c->side, c->prio_hi);
                if (er == cudaSuccess && commit) er = launch_elim_commit(elim_args(c, dt), c->side);
                if (er == cudaSuccess) er = cudaEventRecord(c->join_ev, c->side);
            }
            for (int k = 0; k < n && er == cudaSuccess; ++k) er = cudaStreamWaitEvent(s, b->inst[k]->pre_ev, 0);
            if (er == cudaSuccess) er = cudaMemsetAsync(b->d_counter, 0, cls.size() * sizeof(int), s);
            if (er == cudaSuccess) er = cudaEventRecord(b->kfork, s);
            for (int q = 0; q < (int)cls.size() && er == cudaSuccess; ++q) {
                cudaStream_t qs = q == 0 ? s : b->kside[q - 1];
                if (q) er = cudaStreamWaitEvent(qs, b->kfork, 0);
                BatchSolveArgs ba{};
                for (int k = 0; k < n; ++k) ba.args[k] = args[k];
                ba.items = b->d_items + koff[q];
                ba.nitems = (int)cls[q].items.size();
                ba.counter = b->d_counter + q;
                if (er == cudaSuccess)
                    er = launch_batch_solve(ba, cls[q].R, cls[q].pref, cls[q].threads, cls[q].smem, cls[q].grid,
                                            c0->prio_lo, qs);
                if (er == cudaSuccess && q) er = cudaEventRecord(b->kjoin[q - 1], qs);
            }
            for (int q = 1; q < (int)cls.size() && er == cudaSuccess; ++q) er = cudaStreamWaitEvent(s, b->kjoin[q - 1], 0);
            for (int k = 0; k < n && er == cudaSuccess; ++k) er = cudaStreamWaitEvent(s, b->inst[k]->join_ev, 0);
            cudaGraph_t endg = nullptr;
            const cudaError_t e2 = cudaStreamEndCapture(s, &endg);
            if (er == cudaSuccess) er = e2;
        }
        if (er != cudaSuccess || st) {
            batch_drop_graph(b, false);
            cudaGetLastError();
            return st ? st : bfail(b, TSF_E_CUDA, "persistent batch capture: %s", cudaGetErrorString(er));
        }
        er = cudaGraphInstantiate(&X, G, cudaGraphInstantiateFlagUseNodePriority);
        if (er != cudaSuccess) {
            batch_drop_graph(b, false);
            cudaGetLastError();
            return bfail(b, TSF_E_CUDA, "persistent batch instantiate: %s", cudaGetErrorString(er));
        }
        return TSF_OK;
    };
    tsf_status st = capture(true, b->graph, b->gexec);
    if (!st) st = capture(false, b->graph_nc, b->gexec_nc);
    if (st) return st;
    b->gen.resize(n);
    for (int k = 0; k < n; ++k) b->gen[k] = b->inst[k]->graph_gen;
    b->graph_valid = true;
    b->graph_dt = dt;
    return TSF_OK;
}

extern "C" {

tsf_status tsf_batch_set_persistent(tsf_batch* b, int on) {
    if (!b) return TSF_E_ARG;
    if (on != 0 && on != 1) return bfail(b, TSF_E_ARG, "on must be 0 or 1");
    if (b->persistent != on) batch_drop_graph(b, true);
    b->persistent = on;
    if (on)
        for (tsf_ctx* c : b->inst) use_persistent_tiling(c);
    return TSF_OK;
}

tsf_status tsf_batch_create(tsf_batch** out, int ninst, const tsf_options* opt) {
    if (!out) return TSF_E_ARG;
    *out = nullptr;
    if (ninst < 1 || ninst > TSF_BATCH_MAX) return TSF_E_ARG;
    tsf_options o;
    tsf_default_options(&o);
    if (opt) o = *opt;
    if (!options_ok(&o)) return TSF_E_ARG;
    tsf_batch* b = new (std::nothrow) tsf_batch();
    if (!b) return TSF_E_OOM;
    b->use_graph = o.use_graph;
    if (o.cuda_stream) {
        b->stream = (cudaStream_t)o.cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete b;
            return TSF_E_CUDA;
        }
        b->own_stream = true;
    }
    o.cuda_stream = b->stream;
    for (int i = 0; i < ninst; ++i) {
        tsf_ctx* c = nullptr;
        tsf_status st = tsf_create(&c, &o);
        if (st) {
            for (tsf_ctx* x : b->inst) tsf_destroy(x);
            if (b->own_stream) cudaStreamDestroy(b->stream);
            delete b;
            return st;
        }
        b->inst.push_back(c);
    }
    *out = b;
    return TSF_OK;
}

tsf_status tsf_batch_instance(tsf_batch* b, int inst, tsf_ctx** out) {
    if (!b || !out) return TSF_E_ARG;
    *out = nullptr;
    if (inst < 0 || inst >= (int)b->inst.size()) return bfail(b, TSF_E_ARG, "instance %d out of range", inst);
    *out = b->inst[inst];
    return TSF_OK;
}

tsf_status tsf_batch_step(tsf_batch* b, double dt, int nsteps) {
    if (!b) return TSF_E_ARG;
    if (!(dt > 0) || !std::isfinite(dt) || nsteps < 0) return bfail(b, TSF_E_ARG, "need dt > 0 and nsteps >= 0");
    const int n = (int)b->inst.size();
    for (int i = 0; i < n; ++i) {
        tsf_ctx* c = b->inst[i];
        if (!c->ws_valid || !c->geom_set || !c->state_set)
            return bfail(b, TSF_E_STATE, "instance %d: set meshes, deformation and state first", i);
    }
    if (nsteps == 0) return TSF_OK;
    if (b->persistent)
        for (tsf_ctx* c : b->inst) use_persistent_tiling(c);  // (after a change of micro mesh)
    for (int i = 0; i < n; ++i) {
        tsf_ctx* c = b->inst[i];
        tsf_status st = prepare_step(c, dt);
        if (st) return inst_fail(b, i, st);
        if (pipelined(c) && !c->w_valid) {  // the first w of this state
            if ((st = enqueue_head(c, dt))) return inst_fail(b, i, st);
            c->w_valid = true;
        }
    }
    if (b->persistent) {
        for (int i = 0; i < n; ++i) {
            tsf_ctx* c = b->inst[i];
            if (c->opt.precision != TSF_MIXED || !pipelined(c) || c->tiling != persistent_tiling(c))
                return bfail(b, TSF_E_ARG, "instance %d: the persistent batch needs mixed precision and the pipelined "
                                           "elimination (coupling = elimination, no volume or Robin sources)", i);
        }
    }
    if (!b->use_graph && !b->persistent) {
        for (int s = 0; s < nsteps; ++s) {
            for (int i = 0; i < n; ++i) {
                tsf_status st = run_plain_steps(b->inst[i], dt, 1);
                if (st) return inst_fail(b, i, st);
            }
            b->steps++;
        }
        return TSF_OK;
    }
    bool stale = !b->graph_valid || b->graph_dt != dt || b->gen.size() != (size_t)n;
    for (int i = 0; i < n && !stale; ++i) stale = b->gen[i] != b->inst[i]->graph_gen;
    if (stale) {
        tsf_status st = b->persistent ? batch_capture_persistent(b, dt) : batch_capture(b, dt);
        if (st) return st;
    }
    for (int s = 0; s < nsteps; ++s) {
        cudaError_t e = cudaGraphLaunch(b->gexec_nc && s + 1 < nsteps ? b->gexec_nc : b->gexec, b->stream);
        if (e != cudaSuccess) return bfail(b, TSF_E_CUDA, "cudaGraphLaunch: %s", cudaGetErrorString(e));
        b->steps++;
    }
    return TSF_OK;
}

tsf_status tsf_batch_synchronize(tsf_batch* b) {
    if (!b) return TSF_E_ARG;
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bfail(b, TSF_E_CUDA, "cudaStreamSynchronize: %s", cudaGetErrorString(e));
    for (int i = 0; i < (int)b->inst.size(); ++i) {
        tsf_status st = tsf_synchronize(b->inst[i]);
        if (st) return inst_fail(b, i, st);
    }
    return TSF_OK;
}

tsf_status tsf_batch_persistent_launches(const tsf_batch* b, int* out) {
    if (!b || !out) return TSF_E_ARG;
    *out = b->graph_valid && b->persistent ? b->nlaunch : 0;
    return TSF_OK;
}

tsf_status tsf_batch_get_stats(tsf_batch* b, tsf_stats* out) {
    if (!b || !out) return TSF_E_ARG;
    memset(out, 0, sizeof *out);
    out->tiling = -1;
    for (int i = 0; i < (int)b->inst.size(); ++i) {
        tsf_stats s;
        tsf_status st = tsf_get_stats(b->inst[i], &s);
        if (st) return inst_fail(b, i, st);
        out->inner_iters += s.inner_iters;
        out->dof_cg_iters += s.dof_cg_iters;
        out->refine_sweeps += s.refine_sweeps;
        out->micro_solves += s.micro_solves;
        out->macro_iters += s.macro_iters;
        out->coupling_iters_last = std::max(out->coupling_iters_last, s.coupling_iters_last);
        out->coupling_iters_total += s.coupling_iters_total;
        out->max_inner_iters = std::max(out->max_inner_iters, s.max_inner_iters);
        if (!out->status) out->status = s.status;
        out->coupling_change = std::max(out->coupling_change, s.coupling_change);
        out->micro_launches += s.micro_launches;
        out->macro_launches += s.macro_launches;
        out->micro_kernel_ms += s.micro_kernel_ms;
        out->macro_kernel_ms += s.macro_kernel_ms;
    }
    out->steps = b->steps;
    return TSF_OK;
}

tsf_status tsf_batch_reset_stats(tsf_batch* b) {
    if (!b) return TSF_E_ARG;
    for (int i = 0; i < (int)b->inst.size(); ++i) {
        tsf_status st = tsf_reset_stats(b->inst[i]);
        if (st) return inst_fail(b, i, st);
    }
    b->steps = 0;
    return TSF_OK;
}

const char* tsf_batch_last_error(const tsf_batch* b) { return b ? b->err.c_str() : "null batch"; }

void tsf_batch_destroy(tsf_batch* b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    batch_drop_graph(b, true);
    if (b->d_items) cudaFree(b->d_items);
    if (b->d_counter) cudaFree(b->d_counter);
    for (int k = 0; k < kBatchMaxClasses - 1; ++k) {
        if (b->kside[k]) cudaStreamDestroy(b->kside[k]);
        if (b->kjoin[k]) cudaEventDestroy(b->kjoin[k]);
    }
    if (b->kfork) cudaEventDestroy(b->kfork);
    for (tsf_ctx* c : b->inst) tsf_destroy(c);
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
}

}  // extern "C"
