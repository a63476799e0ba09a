// tsf_noalloc.cu -- the macro solve for callers that cannot allocate device
// memory.
//
// Some programs cannot call cudaMalloc at the point where they need a solve:
// a host application that hands all device memory to its own pool at start-up
// (so a library allocation would fail or fragment the pool), or code running
// in a latency-critical loop (cudaMalloc may synchronise the whole device).
// For them this file offers tsf_macro_solve_noalloc: the same macro-solve
// kernel the coupled step uses, but its scratch vectors and control block live
// in a fixed file-scope device array instead of a workspace.  The array is
// part of the loaded library, so every GPU that loads the library holds it
// (about 0.8 MB) until the process exits.  The call reads its status back and
// waits for the stream before it returns.
#include "tsfem.h"
#include "tsf_internal.cuh"

#include <cmath>
#include <mutex>

using namespace tsf;

namespace {

constexpr int kNoAllocMaxNM = TSF_NOALLOC_MAX_NM;
constexpr size_t kNoAllocMaxNodes = (size_t)(kNoAllocMaxNM + 1) * (kNoAllocMaxNM + 1);
constexpr size_t kCtlDoubles = (sizeof(DevCtl) + sizeof(double) - 1) / sizeof(double);
// six FP64 vectors of the macro PCG (x, r, z, z_old, p, q) and the control block
constexpr size_t kScratchDoubles = 6 * kNoAllocMaxNodes + kCtlDoubles;

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double* g_scratch_addr[kMaxDevices] = {nullptr};  // device address of the array, per device
int g_smem_optin[kMaxDevices] = {0};                // opt-in shared memory per block, per device
bool g_setup_done[kMaxDevices] = {false};

}  // namespace

// The scratch itself.  In host code this name is only a stand-in for the
// symbol; the device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

// Once per device, with that device current: the array's device address and
// the kernel's shared-memory limit (*optin receives the device's opt-in
// shared memory per block, kept for the later calls).  Returns the address or
// nullptr.
static double* noalloc_setup(int dev, int* optin_out, cudaError_t* err) {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (g_setup_done[dev]) {
        *err = cudaSuccess;
        *optin_out = g_smem_optin[dev];
        return g_scratch_addr[dev];
    }
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    int optin = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = configure_macro_kernels(optin);
    *err = e;
    if (e != cudaSuccess) return nullptr;
    g_scratch_addr[dev] = static_cast<double*>(ptr);
    g_smem_optin[dev] = optin;
    g_setup_done[dev] = true;
    *optin_out = optin;
    return g_scratch_addr[dev];
}

extern "C" tsf_status tsf_macro_solve_noalloc(int NM, int bc, double dt, double macro_diff, double kappa,
                                              const double* gam, const double* cH, const double* rho,
                                              const double* u0, double* u_out, double tol, int maxit,
                                              void* cuda_stream, int* iters_out) {
    if (NM < 1 || NM > kNoAllocMaxNM) return TSF_E_ARG;  // beyond the fixed scratch array
    if (bc != TSF_BC_NEUMANN && bc != TSF_BC_DIRICHLET) return TSF_E_ARG;
    if (!(dt > 0) || !(macro_diff > 0) || !(kappa >= 0) || !(tol >= 0) || maxit < 1) return TSF_E_ARG;
    if (!gam || !cH || !rho || !u0 || !u_out) return TSF_E_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return TSF_E_CUDA;
    cudaError_t e;
    int optin = 0;
    double* scratch = noalloc_setup(dev, &optin, &e);
    if (!scratch) return TSF_E_CUDA;
    const int N1 = NM + 1, nM = N1 * N1;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    DevCtl* ctl = reinterpret_cast<DevCtl*>(scratch + 6 * kNoAllocMaxNodes);

    // The array keeps the previous call's contents: the control block (status,
    // counters, coupling counter) must start from zero; the six vectors are
    // fully written by the kernel before they are read.
    if (cudaMemsetAsync(ctl, 0, sizeof(DevCtl), s) != cudaSuccess) return TSF_E_CUDA;
    if (u_out != u0 && cudaMemcpyAsync(u_out, u0, nM * sizeof(double), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return TSF_E_CUDA;

    MacroArgs a{};
    a.NM = NM;
    a.N1 = N1;
    a.nM = nM;
    a.bc = bc;
    a.H = 1.0 / NM;
    a.dt = dt;
    a.Du = macro_diff;
    a.kappa = kappa;
    a.gam = gam;
    a.cH = cH;
    a.rho = rho;
    a.uk = u_out;  // initial guess and Dirichlet values, overwritten by the solution
    a.u = u_out;
    a.x = scratch;
    a.r = scratch + kNoAllocMaxNodes;
    a.z = scratch + 2 * kNoAllocMaxNodes;
    a.zo = scratch + 3 * kNoAllocMaxNodes;
    a.p = scratch + 4 * kNoAllocMaxNodes;
    a.q = scratch + 5 * kNoAllocMaxNodes;
    a.tol = tol;
    a.maxit = maxit;
    a.coupling_tol = HUGE_VAL;  // one pass: the solve itself is the whole job
    a.coupling_maxit = 1;
    a.use_dct = macro_smem_bytes(N1, bc, 1) <= (size_t)optin ? 1 : 0;
    a.set_cond = 0;
    a.ctl = ctl;
    if (launch_macro_solve(a, s) != cudaSuccess) return TSF_E_CUDA;

    DevCtl out;
    if (cudaMemcpyAsync(&out, ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, s) != cudaSuccess) return TSF_E_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return TSF_E_CUDA;
    if (iters_out) *iters_out = (int)out.macro_iters;
    if (out.status) return (tsf_status)out.status;
    return TSF_OK;
}
