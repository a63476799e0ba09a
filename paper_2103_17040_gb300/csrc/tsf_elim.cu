// tsf_elim.cu -- steps by exact elimination of the coupling, pipelined across
// steps.
//
// Given u_i the micro solution is affine in u_i (Eq. (17), micro rows):
//     z_i = S_i^-1 c_i,  c = M v/dt,  v' = z + u' phi,  S phi = kappa r,
// and the fluxes r^T z close one macro solve for u'.  Writing
//     c_{k+1} = M v^{k+1}/dt = M z_k/dt + u^{k+1} mphi,      mphi = M phi/dt,
//     z_{k+1} = w_{k+1} + u^{k+1} psi,   S w_{k+1} = M z_k/dt,   S psi = mphi,
// the micro solve of step k+1 (for w) needs z_k = w_k + u^k psi only, i.e. the
// macro values of the step before.  So one graph launch per step runs
//     k_elim_start: u_old = u^k
//     macro branch: macro prologue (fluxes r^T w_k + u^k r^T psi), macro
//                   solve for u^{k+1}, k_elim_commit v^{k+1} = w_k + u^k psi +
//                   u^{k+1} phi
//     micro branch: k_elim_pre (right-hand side M z_k/dt, warm start), micro
//                   solve for w_{k+1}
// and the one-block macro solve runs beside the micro solve.  At the end of
// the launch the state (u^{k+1}, v^{k+1}) is committed and w_{k+1} is ready
// for the next step.  k_elim_head computes the first w from a state:
//     S w = M v/dt - u mphi   (= c - u mphi, so z = w + u psi).
//
// Warm start of w: extrapolated from the last three solves (quadratic
// 3 w_k - 3 w_{k-1} + w_{k-2}, linear with two, w_k with one), kept in a ring.
// Without volume or Robin sources only (those are stepped by the unpipelined
// elimination).
//
// The column-strip micro kernels, which keep their residual between solves,
// do k_elim_pre's work themselves, so their step has no k_elim_pre: the solve
// of w_k ends by computing M w_k / dt, pushing w_k, and leaving the warm start
// g and the u-independent part M w_k / dt - S g of the next residual; the
// next solve adds u^k M psi / dt to both its right-hand side and that
// residual.  S g needs no second stencil product: the solve leaves its
// residual e = c - S w, so S w = c - e is kept in a second ring and S g is
// the same combination of it.  For these kernels every array of the pipeline
// holds float pairs (hi, lo) instead of FP64 values (ElimArgs::f2): on GB300
// FP64 arithmetic runs at about 1/70 of the FP32 rate, and the pairs keep the
// values to about 2^-44 with FP32 instructions only.  The push happens one
// step earlier, so the commit finds w_k at ring slot hist_step + 2 instead of
// hist_step (ElimArgs::commit_off).  k_elim_pre remains for the
// one-block-per-problem variants, which form their residual from scratch.
#include "tsf_internal.cuh"

namespace tsf {

// One block per micro problem: right-hand side c = M v/dt - u mphi of the
// first w (also into cnext, where the pipelined strip solve reads it with
// u_old = 0), warm start W = v - u (phi + psi), residual and norms.  For the
// column-strip kernels (f2) the warm start, its residual and the right-hand
// side go to the float-pair arrays instead; the residual is that of the pair
// itself (its FP64 value goes through gtmp), so the solve starts consistent.
__global__ void __launch_bounds__(256) k_elim_head(ElimArgs a) {
    __shared__ double buf[3 * 32];
    const int i = blockIdx.x, n1 = a.n1, nm = a.nm;
    const size_t pl = (size_t)a.nmp, io = (size_t)i * pl;
    const double* M = a.M64 + (size_t)i * kPlanes * pl;
    const double* S = a.S64 + (size_t)i * kPlanes * pl;
    const double* v = a.v + io;
    const double* ph = a.phi + io;
    const double* ps = a.psi + io;
    const double* mp = a.mphi + io;
    const double* re = a.redge + (size_t)i * n1;
    double* c = a.c + io;
    double* W = a.f2 ? a.gtmp + io : a.W + io;
    double* res = a.res + io;
    const double ui = a.u[i], idt = 1.0 / a.dt;
    double cc = 0.0, cr = 0.0, rr = 0.0;
    for (int j = threadIdx.x; j < nm; j += blockDim.x) {
        const int p = j % n1, q = j / n1;
        const double cj = fma(plane_apply(M, pl, v, j, p, q, n1), idt, -ui * mp[j]);
        c[j] = cj;
        const double g = fma(-ui, ph[j] + ps[j], v[j]);
        if (a.f2) {
            const float gh = __double2float_rn(g), gl = __double2float_rn(g - (double)gh);
            a.w2[io + j] = make_float2(gh, gl);
            W[j] = (double)gh + (double)gl;
            const float ch = __double2float_rn(cj);
            a.mw2[io + j] = make_float2(ch, __double2float_rn(cj - (double)ch));
        } else {
            a.cnext[io + j] = cj;
            W[j] = g;
        }
        cc = fma(cj, cj, cc);
        if (p == n1 - 1) {
            cr = fma(cj, re[q], cr);
            rr = fma(re[q], re[q], rr);
        }
    }
    double t[3] = {cc, cr, rr};
    block_allreduce<double, 3>(t, buf);  // (also: every thread has written W)
    __syncthreads();
    for (int j = threadIdx.x; j < nm; j += blockDim.x) {
        const double rj = c[j] - plane_apply(S, pl, W, j, j % n1, j / n1, n1);
        if (a.f2) {
            const float rh = __double2float_rn(rj);
            a.res2[io + j] = make_float2(rh, __double2float_rn(rj - (double)rh));
        } else {
            res[j] = rj;
        }
    }
    if (threadIdx.x == 0) {
        double* bn = a.bnorm + (size_t)i * 3;
        bn[0] = t[0];
        bn[1] = t[1];
        bn[2] = t[2];
        a.u_used[i] = 0.0;
    }
}

// u_old = u (the macro state the prepared w belongs to), and the w pushed by
// the previous step's k_elim_pre becomes history.
__global__ void __launch_bounds__(256) k_elim_start(ElimArgs a) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < a.nM) {
        const double u = a.u[k];
        a.u_old[k] = u;
        if (a.u_old2) {
            const float h = __double2float_rn(u);
            a.u_old2[k] = make_float2(h, __double2float_rn(u - (double)h));
        }
    }
    if (k == 0 && a.ctl->pushed) {
        a.ctl->pushed = 0;
        a.ctl->hist_step += 1;
        if (a.ctl->hist_level < 2) a.ctl->hist_level += 1;
    }
}

// One block per micro problem, after the solve of w_k (in W) by a
// one-block-per-problem variant, which forms its residual and ||b|| itself:
// c_{k+1} = M (w_k + u^k psi)/dt = M w_k/dt + u^k mpsi, w_k pushed into the
// ring, W = the extrapolated warm start.  (The strip kernels do this in their
// pipelined epilogue, with the stored residual.)
__global__ void __launch_bounds__(256) k_elim_pre(ElimArgs a) {
    const int i = blockIdx.x, n1 = a.n1, nm = a.nm;
    const size_t pl = (size_t)a.nmp, slot = (size_t)a.nM * pl;
    const double* M = a.M64 + (size_t)i * kPlanes * pl;
    const double* mq = a.mpsi + (size_t)i * pl;
    double* W = a.W + (size_t)i * pl;
    double* c = a.c + (size_t)i * pl;
    const int st = a.ctl->hist_step, level = a.ctl->hist_level;
    double* hc = a.hist + (size_t)(st % 3) * slot + (size_t)i * pl;
    const double* h1 = a.hist + (size_t)((st + 2) % 3) * slot + (size_t)i * pl;
    const double* h2 = a.hist + (size_t)((st + 1) % 3) * slot + (size_t)i * pl;
    const double uo = a.u_old[i], idt = 1.0 / a.dt;
    for (int j = threadIdx.x; j < nm; j += blockDim.x)
        c[j] = fma(uo, mq[j], plane_apply(M, pl, W, j, j % n1, j / n1, n1) * idt);
    __syncthreads();  // every read of w_k at neighbours is done
    for (int j = threadIdx.x; j < nm; j += blockDim.x) {
        const double w = W[j];
        double g = w;
        if (level >= 2)
            g = fma(3.0, w - h1[j], h2[j]);
        else if (level == 1)
            g = fma(2.0, w, -h1[j]);
        hc[j] = w;
        W[j] = g;
    }
    if (i == 0 && threadIdx.x == 0) a.ctl->pushed = 1;
}

// v^{k+1} = w_k + u^k psi + u^{k+1} phi, w_k from its ring slot (pushed by
// k_elim_pre in this step, or by the previous step's strip-solve epilogue).
__global__ void __launch_bounds__(256) k_elim_commit(ElimArgs a) {
    const int i = blockIdx.x;
    const int j = blockIdx.y * blockDim.x + threadIdx.x;
    if (j >= a.nm) return;
    const size_t pl = (size_t)a.nmp, o = (size_t)i * pl + j;
    const size_t ring = (size_t)((a.ctl->hist_step + a.commit_off) % 3) * a.nM * pl;
    const double w = a.f2 ? (double)a.hist2[ring + o].x + (double)a.hist2[ring + o].y : a.hist[ring + o];
    a.v[o] = fma(a.u[i], a.phi[o], fma(a.u_old[i], a.psi[o], w));
}

// out = M x / dt, and ||out||^2, out^T r, ||r||^2 per instance
__global__ void __launch_bounds__(256) k_mass_dt(ElimArgs a, const double* x, double* out, double* nrm) {
    __shared__ double buf[3 * 32];
    const int i = blockIdx.x, n1 = a.n1;
    const size_t pl = (size_t)a.nmp;
    const double* M = a.M64 + (size_t)i * kPlanes * pl;
    const double* xi = x + (size_t)i * pl;
    const double* re = a.redge + (size_t)i * n1;
    double* oi = out + (size_t)i * pl;
    const double idt = 1.0 / a.dt;
    double n0 = 0.0, n1m = 0.0, n2 = 0.0;
    for (int j = threadIdx.x; j < a.nm; j += blockDim.x) {
        const double y = plane_apply(M, pl, xi, j, j % n1, j / n1, n1) * idt;
        oi[j] = y;
        n0 = fma(y, y, n0);
        if (j % n1 == n1 - 1) {
            n1m = fma(y, re[j / n1], n1m);
            n2 = fma(re[j / n1], re[j / n1], n2);
        }
    }
    double t[3] = {n0, n1m, n2};
    block_allreduce<double, 3>(t, buf);
    if (threadIdx.x == 0 && nrm) {
        nrm[(size_t)i * 3] = t[0];
        nrm[(size_t)i * 3 + 1] = t[1];
        nrm[(size_t)i * 3 + 2] = t[2];
    }
}

// psi = 0, cz = mphi (right-hand side for the variants that read c),
// res = mphi, u_used = 0, bnorm = the norms of mphi
__global__ void __launch_bounds__(256) k_psi_setup(ElimArgs a, double* psi, double* cz, const double* mnorm) {
    const int i = blockIdx.x;
    const size_t pl = (size_t)a.nmp;
    for (int j = threadIdx.x; j < a.nmp; j += blockDim.x) {
        const size_t o = (size_t)i * pl + j;
        const double m = j < a.nm ? a.mphi[o] : 0.0;
        psi[o] = 0.0;
        cz[o] = m;
        a.res[o] = m;
    }
    if (threadIdx.x < 3) a.bnorm[(size_t)i * 3 + threadIdx.x] = mnorm[(size_t)i * 3 + threadIdx.x];
    if (threadIdx.x == 0) a.u_used[i] = 0.0;
}

cudaError_t launch_elim_head(const ElimArgs& a, cudaStream_t s) {
    k_elim_head<<<a.nM, 256, 0, s>>>(a);
    return cudaGetLastError();
}
cudaError_t launch_elim_start(const ElimArgs& a, cudaStream_t s) {
    k_elim_start<<<(a.nM + 255) / 256, 256, 0, s>>>(a);
    return cudaGetLastError();
}
cudaError_t launch_elim_pre(const ElimArgs& a, cudaStream_t s, int priority) {
    if (priority == 0) {
        k_elim_pre<<<a.nM, 256, 0, s>>>(a);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(a.nM);
    cfg.blockDim = dim3(256);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributePriority;
    at[0].val.priority = priority;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_elim_pre, a);
}
cudaError_t launch_elim_commit(const ElimArgs& a, cudaStream_t s) {
    dim3 grid(a.nM, (a.nm + 255) / 256);
    k_elim_commit<<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}
cudaError_t launch_mass_dt(const ElimArgs& a, const double* x, double* out, double* nrm, cudaStream_t s) {
    k_mass_dt<<<a.nM, 256, 0, s>>>(a, x, out, nrm);
    return cudaGetLastError();
}
cudaError_t launch_psi_setup(const ElimArgs& a, double* psi, double* cz, const double* mnorm, cudaStream_t s) {
    k_psi_setup<<<a.nM, 256, 0, s>>>(a, psi, cz, mnorm);
    return cudaGetLastError();
}

}  // namespace tsf
