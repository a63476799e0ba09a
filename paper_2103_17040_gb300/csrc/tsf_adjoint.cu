// tsf_adjoint.cu -- kernels of the discrete adjoint of the two-scale march.
//
// Objective J = sum_k m_k u_k^N: the integral of the macro field over
// Omega = [0,1]^2 after N steps (m = row sums of M_H).  One step is
// A(p) X^{n+1} = B(p) X^n with X = (u, v_1, .., v_nM); weighting the micro
// rows with the lumped macro masses, W = diag(1, m_i I), makes W A and W B
// symmetric (the coupling blocks are -kappa m_i r_i^T and -kappa m_i r_i), so
// the adjoint recursion A^T lam^n = B^T lam^{n+1} is the forward recursion
// for lam~ = W^-1 lam.  The host runs adjoint steps with the forward solver;
// these kernels accumulate the gradient
//   dJ/dp_i = -sum_n lam^{n+1 T} (dA/dp_i X^{n+1} - dB/dp_i X^n)
//           = -m_i sum_n [ nu~^T (dM (v^{n+1} - v^n)/dt + dA v^{n+1})
//                          + kappa (v^{n+1} - u_i^{n+1} 1)^T dR (nu~ - mu~_i 1) ]
// (macro Neumann boundary, no sources).  dM, dA, dR come from the
// derivatives of J, C = adj(F) D adj(F)^T / J and |adj(F)^T nu| at the
// quadrature points (Sec. 3.1, Eqs. (13)-(16) differentiated); those do not
// depend on time, so each step only accumulates, per quadrature point,
//   s   += nu~ (v^{n+1} - v^n)/dt,   T += sym(grad nu~ (x) grad v^{n+1}),
//   e   += (v^{n+1} - u^{n+1}) (nu~ - mu~)       (Robin-edge points),
// and one final kernel contracts them with the derivatives for every
// parameter of the deformation family.
#include "tsf_internal.cuh"

namespace tsf {

// 2-point Gauss abscissae on [0,1]
__device__ __forceinline__ double gq(int k) { return k ? 0.5 + 0.28867513459481288225 : 0.5 - 0.28867513459481288225; }

// lumped macro mass of node i on the NM x NM mesh of [0,1]^2
__device__ __forceinline__ double lumped_mass(int i, int NM) {
    const int n1 = NM + 1, p = i % n1, q = i / n1;
    const double cx = (p == 0 || p == NM) ? 1.0 : 2.0, cy = (q == 0 || q == NM) ? 1.0 : 2.0;
    return 0.25 * cx * cy / ((double)NM * NM);
}

// One thread per (instance, micro cell): adds this step's products at the
// cell's 4 quadrature points (and its 2 Robin-edge points).
__global__ void __launch_bounds__(128) k_adj_accumulate(AdjAccArgs a) {
    const int i = blockIdx.x;
    const int cell = blockIdx.y * blockDim.x + threadIdx.x;
    const int N = a.Nm, n1 = a.n1;
    if (cell >= N * N) return;
    const int ac = cell % N, b = cell / N;
    const size_t base = (size_t)i * a.nmp;
    const int j0 = ac + n1 * b, j1 = j0 + 1, j2 = j0 + n1, j3 = j2 + 1;
    const double nu[4] = {a.nu[base + j0], a.nu[base + j1], a.nu[base + j2], a.nu[base + j3]};
    const double w1[4] = {a.v1[base + j0], a.v1[base + j1], a.v1[base + j2], a.v1[base + j3]};
    const double w0[4] = {a.v0[base + j0], a.v0[base + j1], a.v0[base + j2], a.v0[base + j3]};
    double* acc = a.acc + ((size_t)i * N * N + cell) * 16;
    for (int qt = 0; qt < 2; ++qt)
        for (int qs = 0; qs < 2; ++qs) {
            const double s = gq(qs), t = gq(qt);
            const double phi[4] = {(1 - s) * (1 - t), s * (1 - t), (1 - s) * t, s * t};
            const double ds[4] = {-(1 - t), (1 - t), -t, t};
            const double dt[4] = {-(1 - s), -s, (1 - s), s};
            double nq = 0, dv = 0, ns = 0, nt = 0, vs = 0, vt = 0;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                nq = fma(phi[k], nu[k], nq);
                dv = fma(phi[k], w1[k] - w0[k], dv);
                ns = fma(ds[k], nu[k], ns);
                nt = fma(dt[k], nu[k], nt);
                vs = fma(ds[k], w1[k], vs);
                vt = fma(dt[k], w1[k], vt);
            }
            double* c = acc + 4 * (2 * qt + qs);
            c[0] = fma(nq, dv * a.inv_dt, c[0]);
            c[1] = fma(ns, vs, c[1]);
            c[2] = fma(ns, vt, fma(nt, vs, c[2]));
            c[3] = fma(nt, vt, c[3]);
        }
    if (ac == N - 1) {  // Robin edge yhat_1 = 1: local nodes 1 (t = 0) and 3 (t = 1)
        const double mu = a.mu[i], u1 = a.u1[i];
        double* e = a.eacc + ((size_t)i * N + b) * 2;
        for (int qt = 0; qt < 2; ++qt) {
            const double t = gq(qt);
            const double vq = (1 - t) * w1[1] + t * w1[3];
            const double nq = (1 - t) * nu[1] + t * nu[3];
            e[qt] = fma(vq - u1, nq - mu, e[qt]);
        }
    }
}

cudaError_t launch_adj_accumulate(const AdjAccArgs& a, cudaStream_t s) {
    dim3 grid(a.nM, (a.Nm * a.Nm + 127) / 128);
    k_adj_accumulate<<<grid, 128, 0, s>>>(a);
    return cudaGetLastError();
}

// Derivative direction of a family parameter in the general form
// F = A + b pi [[c1 s2, s1 c2], [0, 0]]: 0..3 = entries of A, 4 = b, -1 = none.
__device__ __forceinline__ int param_direction(int family, int k) {
    switch (family) {
        case 1: return 4;                    // bump a
        case 2: return k == 0 ? 1 : 4;       // shear s = A12, bump b
        case 3: return k < 4 ? k : -1;       // affine A (shift c has no effect on F)
        case 4: return k < 4 ? k : 4;        // affine A, bump b
        default: return -1;
    }
}

// dJ, dC (sym, 3), ds (|adj(F)^T e1|) for dF at F.
__device__ __forceinline__ void dpull(const double F[4], const double dF[4], double D11, double D12, double D22,
                                      double& dJ, double dC[3], double& dsg) {
    const double J = F[0] * F[3] - F[1] * F[2];
    const double G[4] = {F[3], -F[1], -F[2], F[0]};
    const double dG[4] = {dF[3], -dF[1], -dF[2], dF[0]};
    const double Dm[4] = {D11, D12, D12, D22};
    dJ = dF[0] * F[3] + F[0] * dF[3] - dF[1] * F[2] - F[1] * dF[2];
    double GD[4], dGD[4];
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 2; ++c) {
            GD[2 * r + c] = G[2 * r] * Dm[c] + G[2 * r + 1] * Dm[2 + c];
            dGD[2 * r + c] = dG[2 * r] * Dm[c] + dG[2 * r + 1] * Dm[2 + c];
        }
    double P[3], dP[3];
    const int rr[3] = {0, 0, 1}, cc[3] = {0, 1, 1};
    for (int m = 0; m < 3; ++m) {
        const int r = rr[m], c = cc[m];
        P[m] = GD[2 * r] * G[2 * c] + GD[2 * r + 1] * G[2 * c + 1];
        dP[m] = dGD[2 * r] * G[2 * c] + dGD[2 * r + 1] * G[2 * c + 1] + GD[2 * r] * dG[2 * c] +
                GD[2 * r + 1] * dG[2 * c + 1];
    }
    for (int m = 0; m < 3; ++m) dC[m] = dP[m] / J - P[m] * dJ / (J * J);
    const double w0 = G[0], w1 = G[1], dw0 = dG[0], dw1 = dG[1];  // adj(F)^T e1
    dsg = (w0 * dw0 + w1 * dw1) / sqrt(w0 * w0 + w1 * w1);
}

// One block per instance: grad[i][k] = -m_i (sum over quadrature points of the
// accumulated products contracted with the derivatives for parameter k).
__global__ void __launch_bounds__(256) k_adj_gradient(AdjGradArgs a) {
    __shared__ double buf[6 * 32];
    const int i = blockIdx.x;
    const int N = a.Nm;
    const double h = 1.0 / N;
    const double* pr = a.prm5 + (size_t)i * 5;
    const double pi = 3.14159265358979323846;
    double part[6] = {0, 0, 0, 0, 0, 0};
    int dir[6];
    for (int k = 0; k < 6; ++k) dir[k] = k < a.nparam ? param_direction(a.family, k) : -1;
    const double* acc = a.acc + (size_t)i * N * N * 16;
    for (int cell = threadIdx.x; cell < N * N; cell += blockDim.x) {
        const int ac = cell % N, b = cell / N;
        for (int qt = 0; qt < 2; ++qt)
            for (int qs = 0; qs < 2; ++qs) {
                double s1, c1, s2, c2;
                sincospi((ac + gq(qs)) * h, &s1, &c1);
                sincospi((b + gq(qt)) * h, &s2, &c2);
                const double F[4] = {fma(pr[4] * pi, c1 * s2, pr[0]), fma(pr[4] * pi, s1 * c2, pr[1]), pr[2], pr[3]};
                const double* c = acc + cell * 16 + 4 * (2 * qt + qs);
                for (int k = 0; k < 6; ++k) {
                    if (dir[k] < 0) continue;
                    double dF[4] = {0, 0, 0, 0};
                    if (dir[k] < 4) dF[dir[k]] = 1.0;
                    else {
                        dF[0] = pi * c1 * s2;
                        dF[1] = pi * s1 * c2;
                    }
                    double dJ, dC[3], dsg;
                    dpull(F, dF, a.D11, a.D12, a.D22, dJ, dC, dsg);
                    const double v = h * h * dJ * c[0] + dC[0] * c[1] + dC[1] * c[2] + dC[2] * c[3];
                    part[k] = fma(0.25, v, part[k]);
                }
            }
    }
    for (int b = threadIdx.x; b < N; b += blockDim.x) {
        for (int qt = 0; qt < 2; ++qt) {
            double s1, c1, s2, c2;
            sincospi(1.0, &s1, &c1);
            sincospi((b + gq(qt)) * h, &s2, &c2);
            const double F[4] = {fma(pr[4] * pi, c1 * s2, pr[0]), fma(pr[4] * pi, s1 * c2, pr[1]), pr[2], pr[3]};
            const double e = a.eacc[((size_t)i * N + b) * 2 + qt];
            for (int k = 0; k < 6; ++k) {
                if (dir[k] < 0) continue;
                double dF[4] = {0, 0, 0, 0};
                if (dir[k] < 4) dF[dir[k]] = 1.0;
                else {
                    dF[0] = pi * c1 * s2;
                    dF[1] = pi * s1 * c2;
                }
                double dJ, dC[3], dsg;
                dpull(F, dF, a.D11, a.D12, a.D22, dJ, dC, dsg);
                part[k] = fma(0.5 * h * a.kappa * dsg, e, part[k]);
            }
        }
    }
    block_allreduce<double, 6>(part, buf);
    if (threadIdx.x == 0) {
        const double m = lumped_mass(i, a.NM);
        for (int k = 0; k < a.nparam; ++k) a.grad[(size_t)i * a.nparam + k] = -m * part[k];
    }
}

cudaError_t launch_adj_gradient(const AdjGradArgs& a, cudaStream_t s) {
    k_adj_gradient<<<a.nM, 256, 0, s>>>(a);
    return cudaGetLastError();
}

// J = sum_k m_k u_k (compensated), one block.
__global__ void __launch_bounds__(256) k_mean_u(const double* u, int nM, int NM, double* J) {
    __shared__ double buf[64];
    double s = 0.0, c = 0.0;
    for (int k = threadIdx.x; k < nM; k += blockDim.x) {
        double t, e;
        two_sum(s, lumped_mass(k, NM) * u[k], t, e);
        s = t;
        c += e;
    }
    const double r = block_sum_compensated(s + c, buf);
    if (threadIdx.x == 0) *J = r;
}

cudaError_t launch_mean_u(const double* u, int nM, int NM, double* J, cudaStream_t s) {
    k_mean_u<<<1, 256, 0, s>>>(u, nM, NM, J);
    return cudaGetLastError();
}

__global__ void k_fill(double* x, double val, size_t n) {
    const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) x[k] = val;
}

cudaError_t launch_fill(double* x, double val, size_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_fill<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(x, val, n);
    return cudaGetLastError();
}

}  // namespace tsf
