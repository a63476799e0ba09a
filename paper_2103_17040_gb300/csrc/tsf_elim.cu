// tsf_elim.cu -- pipelined steps by exact elimination of the coupling.
//
// Given u_i the micro solution is affine in u_i (Eq. (17), micro rows):
//     v_i = z_i + u_i phi_i,   S_i z_i = c_i,   S_i phi_i = kappa r_i,
// so one micro solve for z and one macro solve for u close a step.  The next
// step's right-hand side is
//     c' = M v'/dt + src = M z/dt + u' (M phi/dt) + src,
// whose only dependence on the new macro values u' is the scalar multiple of
// the precomputed M phi/dt.  So right after the micro solve, while the
// one-block macro solve runs, k_elim_pre computes on the other SMs
//     cpre = M z/dt,   g = warm start of the next z,   res = cpre - S g,
// and the next step's k_elim_front only adds u' M phi/dt and the sources
// (elementwise, plus M fv when a volume source is set).
//
// The residual of the warm start needs S g: the solve leaves its residual
// e = c - S z behind, so S z = c - e is kept in a second ring and S g is the
// same extrapolation of those (no second stencil product).
//
// Warm start: the next z is extrapolated from the last three solves,
// g = 3 z_n - 3 z_{n-1} + z_{n-2} (quadratic), 2 z_n - z_{n-1} with two, z_n
// with one; the z's are kept in a ring of three fields.  The first step after
// a new state (or new operators) has no prepared data and computes
// everything from the state: c = M v/dt + src, g = v - u phi, res = c - S g.
//
// Ring bookkeeping (device counters, so the same kernels serve every graph
// launch): k_elim_pre pushes z_n into slot hist_step % 3 and reads the
// hist_level older slots; k_elim_commit reads z_n from that slot; the next
// k_elim_front (prepared path) advances hist_step and hist_level.
#include "tsf_internal.cuh"

namespace tsf {

// M fv + R g at node j = (p, q) of instance i (0 without sources)
__device__ __forceinline__ double elim_source(const ElimArgs& a, int i, int j, int p, int q, const double* M,
                                              size_t pl) {
    double y = 0.0;
    if (a.fv) y = plane_apply(M, pl, a.fv + (size_t)i * pl, j, p, q, a.n1);
    if (a.g && p == a.n1 - 1) {
        const int n1 = a.n1;
        const double* g = a.g + (size_t)i * n1;
        const double* Rd = a.Rd + (size_t)i * n1;
        const double* Ru = a.Ru + (size_t)i * n1;
        y = fma(Rd[q], g[q], y);
        if (q + 1 < n1) y = fma(Ru[q], g[q + 1], y);
        if (q > 0) y = fma(Ru[q - 1], g[q - 1], y);
    }
    return y;
}

// One block per micro problem: the right-hand side, the residual of the warm
// start in Z, and the norms that scale the tolerance.
__global__ void __launch_bounds__(256) k_elim_front(ElimArgs a) {
    __shared__ double buf[3 * 32];
    const int i = blockIdx.x, n1 = a.n1, nm = a.nm;
    const size_t pl = (size_t)a.nmp;
    const double* M = a.M64 + (size_t)i * kPlanes * pl;
    const double* S = a.S64 + (size_t)i * kPlanes * pl;
    const double* re = a.redge + (size_t)i * n1;
    double* c = a.c + (size_t)i * pl;
    double* res = a.res + (size_t)i * pl;
    double* Z = a.Z + (size_t)i * pl;
    const double ui = a.u[i], idt = 1.0 / a.dt;
    const bool prep = a.ctl->prep_ok != 0;
    const bool sources = a.fv || a.g;
    double cc = 0.0, cr = 0.0, rr = 0.0;
    if (prep && !sources) {
        // c = cpre + u mphi; its norms follow from the prepared ones (the FP64
        // pipe is the bound of this kernel: two DFMA per node)
        const double* cp = a.cpre + (size_t)i * pl;
        const double* mp = a.mphi + (size_t)i * pl;
        for (int j = threadIdx.x; j < nm; j += blockDim.x) {
            const double add = ui * mp[j];
            c[j] = cp[j] + add;
            res[j] += add;  // res = cpre - S g + (c - cpre)
        }
        if (threadIdx.x == 0) {
            const double* pn = a.pnorm + (size_t)i * 3;
            const double* mn = a.mnorm + (size_t)i * 3;
            double* bn = a.bnorm + (size_t)i * 3;
            bn[0] = fma(ui, fma(ui, mn[0], 2.0 * pn[1]), pn[0]);
            bn[1] = fma(ui, mn[1], pn[2]);
            bn[2] = mn[2];
            a.u_used[i] = 0.0;
            if (i == 0) {  // the z pushed by the last k_elim_pre becomes history
                a.ctl->hist_step += 1;
                if (a.ctl->hist_level < 2) a.ctl->hist_level += 1;
            }
        }
        return;
    }
    if (prep) {
        const double* cp = a.cpre + (size_t)i * pl;
        const double* mp = a.mphi + (size_t)i * pl;
        for (int j = threadIdx.x; j < nm; j += blockDim.x) {
            const int p = j % n1, q = j / n1;
            const double add = fma(ui, mp[j], elim_source(a, i, j, p, q, M, pl));
            const double cj = cp[j] + add;
            c[j] = cj;
            res[j] += add;  // res = cpre - S g + (c - cpre)
            const double rj = p == n1 - 1 ? re[q] : 0.0;
            cc = fma(cj, cj, cc);
            cr = fma(cj, rj, cr);
            rr = fma(rj, rj, rr);
        }
    } else {
        const double* v = a.v + (size_t)i * pl;
        const double* ph = a.phi + (size_t)i * pl;
        for (int j = threadIdx.x; j < nm; j += blockDim.x) {
            const int p = j % n1, q = j / n1;
            const double cj = fma(plane_apply(M, pl, v, j, p, q, n1), idt, elim_source(a, i, j, p, q, M, pl));
            c[j] = cj;
            Z[j] = fma(-ui, ph[j], v[j]);
            const double rj = p == n1 - 1 ? re[q] : 0.0;
            cc = fma(cj, cj, cc);
            cr = fma(cj, rj, cr);
            rr = fma(rj, rj, rr);
        }
        __syncthreads();
        for (int j = threadIdx.x; j < nm; j += blockDim.x) res[j] = c[j] - plane_apply(S, pl, Z, j, j % n1, j / n1, n1);
    }
    double t[3] = {cc, cr, rr};
    block_allreduce<double, 3>(t, buf);
    if (threadIdx.x == 0) {
        double* bn = a.bnorm + (size_t)i * 3;
        bn[0] = t[0];
        bn[1] = t[1];
        bn[2] = t[2];
        a.u_used[i] = 0.0;
        if (prep && i == 0) {  // the z pushed by the last k_elim_pre becomes history
            a.ctl->hist_step += 1;
            if (a.ctl->hist_level < 2) a.ctl->hist_level += 1;
        }
    }
}

// One block per micro problem, right after the micro solve (Z = z_n):
// cpre = M z/dt, push z into the ring, Z = extrapolated warm start,
// res = cpre - S Z.
__global__ void __launch_bounds__(256) k_elim_pre(ElimArgs a) {
    __shared__ double buf[3 * 32];
    const int i = blockIdx.x, n1 = a.n1, nm = a.nm;
    const size_t pl = (size_t)a.nmp, slot = (size_t)a.nM * pl;
    const double* M = a.M64 + (size_t)i * kPlanes * pl;
    const double* S = a.S64 + (size_t)i * kPlanes * pl;
    double* Z = a.Z + (size_t)i * pl;
    double* cp = a.cpre + (size_t)i * pl;
    double* res = a.res + (size_t)i * pl;
    const int st = a.ctl->hist_step, level = a.ctl->hist_level;
    double* hc = a.hist + (size_t)(st % 3) * slot + (size_t)i * pl;
    const double* h1 = a.hist + (size_t)((st + 2) % 3) * slot + (size_t)i * pl;
    const double* h2 = a.hist + (size_t)((st + 1) % 3) * slot + (size_t)i * pl;
    const double idt = 1.0 / a.dt;
    const double* mp = a.mphi + (size_t)i * pl;
    const double* re = a.redge + (size_t)i * n1;
    double n0 = 0.0, n1m = 0.0, n2 = 0.0;
    for (int j = threadIdx.x; j < nm; j += blockDim.x) {
        const double y = plane_apply(M, pl, Z, j, j % n1, j / n1, n1) * idt;
        cp[j] = y;
        n0 = fma(y, y, n0);
        n1m = fma(y, mp[j], n1m);
        if (j % n1 == n1 - 1) n2 = fma(y, re[j / n1], n2);
    }
    {   // norms of cpre for the next front (also orders every read of z_n at
        // neighbours before Z is overwritten: the reduction synchronises)
        double t[3] = {n0, n1m, n2};
        block_allreduce<double, 3>(t, buf);
        if (threadIdx.x == 0) {
            double* pn = a.pnorm + (size_t)i * 3;
            pn[0] = t[0];
            pn[1] = t[1];
            pn[2] = t[2];
        }
    }
    __syncthreads();
    if (a.yhist) {
        // S z_k = c_k - e_k with e_k the residual the solve left behind, so
        // S g is the same combination of the stored S z as g of the z: no
        // second stencil product
        const double* c = a.c + (size_t)i * pl;
        double* yc = a.yhist + (size_t)(st % 3) * slot + (size_t)i * pl;
        const double* y1 = a.yhist + (size_t)((st + 2) % 3) * slot + (size_t)i * pl;
        const double* y2 = a.yhist + (size_t)((st + 1) % 3) * slot + (size_t)i * pl;
        for (int j = threadIdx.x; j < nm; j += blockDim.x) {
            const double z = Z[j], y = c[j] - res[j];
            double g = z, sg = y;
            if (level >= 2) {
                g = fma(3.0, z - h1[j], h2[j]);
                sg = fma(3.0, y - y1[j], y2[j]);
            } else if (level == 1) {
                g = fma(2.0, z, -h1[j]);
                sg = fma(2.0, y, -y1[j]);
            }
            hc[j] = z;
            yc[j] = y;
            Z[j] = g;
            res[j] = cp[j] - sg;
        }
    } else {
        for (int j = threadIdx.x; j < nm; j += blockDim.x) {
            const double z = Z[j];
            double g = z;
            if (level >= 2)
                g = fma(3.0, z - h1[j], h2[j]);
            else if (level == 1)
                g = fma(2.0, z, -h1[j]);
            hc[j] = z;
            Z[j] = g;
        }
        __syncthreads();
        for (int j = threadIdx.x; j < nm; j += blockDim.x)
            res[j] = cp[j] - plane_apply(S, pl, Z, j, j % n1, j / n1, n1);
    }
    if (i == 0 && threadIdx.x == 0) a.ctl->prep_ok = 1;
}

// v = z_n + u phi with z_n from the ring slot the last k_elim_pre wrote.
__global__ void __launch_bounds__(256) k_elim_commit(ElimArgs a) {
    const int i = blockIdx.x;
    const int j = blockIdx.y * blockDim.x + threadIdx.x;
    if (j >= a.nm) return;
    const size_t pl = (size_t)a.nmp, o = (size_t)i * pl + j;
    const double* z = a.hist + (size_t)(a.ctl->hist_step % 3) * a.nM * pl;
    a.v[o] = fma(a.u[i], a.phi[o], z[o]);
}

// mphi = M phi / dt (once per geometry and dt)
__global__ void __launch_bounds__(256) k_mphi(ElimArgs a) {
    __shared__ double buf[3 * 32];
    const int i = blockIdx.x, n1 = a.n1;
    const size_t pl = (size_t)a.nmp;
    const double* M = a.M64 + (size_t)i * kPlanes * pl;
    const double* ph = a.phi + (size_t)i * pl;
    const double* re = a.redge + (size_t)i * n1;
    double* mp = a.mphi + (size_t)i * pl;
    const double idt = 1.0 / a.dt;
    double n0 = 0.0, n1m = 0.0, n2 = 0.0;
    for (int j = threadIdx.x; j < a.nm; j += blockDim.x) {
        const double y = plane_apply(M, pl, ph, j, j % n1, j / n1, n1) * idt;
        mp[j] = y;
        n0 = fma(y, y, n0);
        if (j % n1 == n1 - 1) {
            n1m = fma(y, re[j / n1], n1m);
            n2 = fma(re[j / n1], re[j / n1], n2);
        }
    }
    double t[3] = {n0, n1m, n2};
    block_allreduce<double, 3>(t, buf);
    if (threadIdx.x == 0) {
        double* mn = a.mnorm + (size_t)i * 3;
        mn[0] = t[0];
        mn[1] = t[1];
        mn[2] = t[2];
    }
}

cudaError_t launch_elim_front(const ElimArgs& a, cudaStream_t s) {
    k_elim_front<<<a.nM, 256, 0, s>>>(a);
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
cudaError_t launch_mphi(const ElimArgs& a, cudaStream_t s) {
    k_mphi<<<a.nM, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace tsf
