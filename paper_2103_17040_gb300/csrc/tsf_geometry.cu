// tsf_geometry.cu -- pulled-back Q1 operators of every micro problem (K0).
//
// For node x_i of the macro mesh the micro problem lives on the reference
// cell Z = [0,1]^2 and sees the deformation chi(x_i, .) only through
// J = det F, C = J F^{-1} D F^{-T} at the quadrature points of the cells and
// s = |cof(F) nu| on the Robin edge (Sec. 3.1, Eqs. (13), (14), (16); the
// diffusion tensor D sits between F^{-1} and F^{-T}).  The paper caches J and
// J K K^T per quadrature point (Sec. 3.4); here every quadrature point is
// recomputed from the node's few deformation parameters while the stencil of
// the assembled operator is written once per (geometry, dt), so the solver
// streams 5 stencil planes per node and never touches quadrature data.
//
// All five deformation families are mapped to one general form
//     chi(yhat) = A yhat + b (sin pi y1 sin pi y2, 0),
//     F = A + b pi [[cos pi y1 sin pi y2, sin pi y1 cos pi y2], [0, 0]],
// with parameters (A11, A12, A21, A22, b).
#include "tsf_geom.cuh"

namespace tsf {

__global__ void k_expand_params(int family, int nparam, const double* __restrict__ in, double* __restrict__ prm5,
                                float* __restrict__ map32, int nM) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nM) return;
    const double* p = in + (size_t)i * nparam;
    double A11 = 1.0, A12 = 0.0, A21 = 0.0, A22 = 1.0, b = 0.0, c1 = 0.0, c2 = 0.0;
    switch (family) {
        case 1: b = p[0]; break;                                           // bump (a)
        case 2: A12 = p[0]; b = p[1]; break;                               // shear + bump (s, b)
        case 3:                                                            // affine (A, c): c drops out of F
            A11 = p[0]; A12 = p[1]; A21 = p[2]; A22 = p[3]; c1 = p[4]; c2 = p[5];
            break;
        case 4: A11 = p[0]; A12 = p[1]; A21 = p[2]; A22 = p[3]; b = p[4]; break;
        default: break;                                                    // identity
    }
    double* o = prm5 + (size_t)i * 5;
    o[0] = A11; o[1] = A12; o[2] = A21; o[3] = A22; o[4] = b;
    float* m = map32 + (size_t)i * 8;  // the whole map in FP32 for the push-forward
    m[0] = (float)A11; m[1] = (float)A12; m[2] = (float)A21; m[3] = (float)A22;
    m[4] = (float)b; m[5] = (float)c1; m[6] = (float)c2; m[7] = 0.f;
}

cudaError_t launch_expand_params(int family, int nparam, const double* in, double* prm5, float* map32, int nM,
                                 cudaStream_t s) {
    k_expand_params<<<(nM + 127) / 128, 128, 0, s>>>(family, nparam, in, prm5, map32, nM);
    return cudaGetLastError();
}

// Push-forward for visualisation (Sec. 3.6): micro node j of instance i,
// reference point yhat_j, goes to
//     X = x_i + scale (chi(x_i, yhat_j) - centre),
// chi = A yhat + b (sin pi y1 sin pi y2, 0) + c, x_i = x0 + H (p, q);
// centre = (1/2, 1/2) (centre_mode 0: cells around the reference cell
// [0,1]^2), or chi(x_i, (1/2, 1/2)) (centre_mode 1: each cell centred on its
// own image of the reference centre).  out[(i nm + j) 3 + {0,1,2}] =
// (X1, X2, v_i(yhat_j)) in FP32 (a picture needs no more, and GB300's FP64
// rate would make this streaming kernel compute-bound).  One thread per
// (instance, node); sin(pi k/Nm) of the n1 grid lines from a table.
__global__ void __launch_bounds__(256) k_pushforward(int n1, int nm, int nmp, int NM, float x0, float H, float h,
                                                     const float* __restrict__ map32, const double* __restrict__ v,
                                                     float scale, int centre_mode, float* __restrict__ out) {
    __shared__ float sinpi_tab[65];  // n1 <= 65
    for (int k = threadIdx.x; k < n1; k += blockDim.x) sinpi_tab[k] = sinpif((float)k * h);
    __syncthreads();
    const int i = blockIdx.x;
    const int j = blockIdx.y * blockDim.x + threadIdx.x;
    if (j >= nm) return;
    const int N1 = NM + 1;
    const float x1 = fmaf((float)(i % N1), H, x0), x2 = fmaf((float)(i / N1), H, x0);
    const int pj = j % n1, qj = j / n1;
    const float y1 = (float)pj * h, y2 = (float)qj * h;
    const float4 m0 = *reinterpret_cast<const float4*>(map32 + (size_t)i * 8);
    const float4 m1 = *reinterpret_cast<const float4*>(map32 + (size_t)i * 8 + 4);
    const float s12 = sinpi_tab[pj] * sinpi_tab[qj];
    const float ch1 = fmaf(m1.x, s12, fmaf(m0.x, y1, fmaf(m0.y, y2, m1.y)));
    const float ch2 = fmaf(m0.z, y1, fmaf(m0.w, y2, m1.z));
    float c1 = 0.5f, c2 = 0.5f;
    if (centre_mode == 1) {   // chi(1/2, 1/2): sin(pi/2)^2 = 1
        c1 = m1.x + fmaf(m0.x, 0.5f, fmaf(m0.y, 0.5f, m1.y));
        c2 = fmaf(m0.z, 0.5f, fmaf(m0.w, 0.5f, m1.z));
    }
    float* o = out + ((size_t)i * nm + j) * 3;
    o[0] = fmaf(scale, ch1 - c1, x1);
    o[1] = fmaf(scale, ch2 - c2, x2);
    o[2] = (float)v[(size_t)i * nmp + j];
}

cudaError_t launch_pushforward(int Nm, int n1, int nm, int nmp, int NM, int nM, const float* map32, const double* v,
                               float x0, float H, float scale, int centre_mode, float* out, cudaStream_t s) {
    dim3 grid(nM, (nm + 255) / 256);
    k_pushforward<<<grid, 256, 0, s>>>(n1, nm, nmp, NM, x0, H, 1.0f / Nm, map32, v, scale, centre_mode, out);
    return cudaGetLastError();
}

// One thread per (micro node j, instance i): the five stored couplings of
// node j in M and in S = M/dt + A + kappa R, summed over the (up to four)
// cells around the node with 2x2 Gauss points; on Robin-edge nodes also the
// boundary mass R (2-point Gauss per edge segment).  Where the node's own map
// has b = 0 (identity and affine maps, and any member of the other families
// whose bump amplitude is zero) F is constant and the element matrices come
// from the reference tables; otherwise from the quadrature points.  The
// tables are filled by the first 16 threads before any thread leaves, and the
// branch is taken on each node's own parameters, so both paths can run in one
// launch.
__global__ void __launch_bounds__(128) k_geometry(GeomArgs a) {
    __shared__ double ref[64];
    fill_reference_tables(ref);
    __syncthreads();
    const int j = blockIdx.y * blockDim.x + threadIdx.x;
    const int i = blockIdx.x;  // instances on grid.x (up to 2^31 - 1); nodes on grid.y
    if (j >= a.nmp) return;
    const size_t pl = (size_t)a.nmp;
    double* M64 = a.M64 + (size_t)i * kPlanes * pl;
    double* S64 = a.S64 + (size_t)i * kPlanes * pl;
    float* S32 = a.S32 + (size_t)i * kPlanes * pl;
    float* S32lo = a.S32lo ? a.S32lo + (size_t)i * kPlanes * pl : nullptr;
    if (j >= a.nm) {  // padding of the planes: zero couplings
        for (int k = 0; k < kPlanes; ++k) {
            M64[k * pl + j] = 0.0;
            S64[k * pl + j] = 0.0;
            S32[k * pl + j] = 0.0f;
            if (S32lo) S32lo[k * pl + j] = 0.0f;
        }
        a.lm[(size_t)i * pl + j] = 0.0;
        return;
    }
    const int N = a.Nm, n1 = a.n1;
    const int p = j % n1, q = j / n1;
    const Deform d = load_deform(a.prm5, i);
    double m[kPlanes], k[kPlanes], lump;
    bool bad;
    if (d.bpi == 0.0) node_couplings_affine(d, a.D11, a.D12, a.D22, p, q, N, ref, m, k, lump, bad);
    else node_couplings(d, a.D11, a.D12, a.D22, p, q, N, m, k, lump, bad);

    // Robin edge yhat_1 = 1: R = int s eta eta with s = |cof(F) e1| = sqrt(F22^2 + F12^2)
    double Rd = 0.0, Ru = 0.0, Rdn = 0.0;
    if (p == N) {
        edge_node_mass(d, kEdgeRight, q, N, Rd, Ru, Rdn);
        const size_t e = (size_t)i * n1 + q;
        a.Rd[e] = Rd;
        a.Ru[e] = Ru;
        a.redge[e] = Rd + Ru + Rdn;
    }

    const double idt = 1.0 / a.dt;
    double sv[kPlanes];
#pragma unroll
    for (int c = 0; c < kPlanes; ++c) sv[c] = fma(m[c], idt, k[c]);
    sv[0] += a.kappa * Rd;
    sv[2] += a.kappa * Ru;
#pragma unroll
    for (int c = 0; c < kPlanes; ++c) {
        M64[c * pl + j] = m[c];
        S64[c * pl + j] = sv[c];
        const float hi = (float)sv[c];
        S32[c * pl + j] = hi;
        if (S32lo) S32lo[c * pl + j] = (float)(sv[c] - (double)hi);  // the difference is exact in FP64
    }
    a.lm[(size_t)i * pl + j] = lump;
    if (bad) atomicOr(&a.ctl->geom_error, 1);
}

cudaError_t launch_geometry(const GeomArgs& a, cudaStream_t s) {
    dim3 grid(a.nM, (a.nmp + 127) / 128);
    k_geometry<<<grid, 128, 0, s>>>(a);
    return cudaGetLastError();
}

// |Gamma_i| = sum_q r_i(q) and |Y_x_i| = 1^T M_i 1 (one block per instance).
__global__ void __launch_bounds__(256) k_instance_sums(int n1, int nm, int nmp, const double* __restrict__ lm,
                                                       const double* __restrict__ redge, double* gam,
                                                       double* vol) {
    __shared__ double buf[64];
    const int i = blockIdx.x;
    double sv = 0.0, sg = 0.0;
    for (int j = threadIdx.x; j < nm; j += blockDim.x) sv += lm[(size_t)i * nmp + j];
    for (int qq = threadIdx.x; qq < n1; qq += blockDim.x) sg += redge[(size_t)i * n1 + qq];
    double v2[2] = {sv, sg};
    block_allreduce<double, 2>(v2, buf);
    if (threadIdx.x == 0) {
        vol[i] = v2[0];
        gam[i] = v2[1];
    }
}

cudaError_t launch_instance_sums(int n1, int nm, int nmp, int nM, const double* lm, const double* redge,
                                 double* gam, double* vol, cudaStream_t s) {
    k_instance_sums<<<nM, 256, 0, s>>>(n1, nm, nmp, lm, redge, gam, vol);
    return cudaGetLastError();
}

}  // namespace tsf
