// tsf_geom.cuh -- point-wise pull-back of one micro cell and the Q1 couplings
// of one node, shared by the geometry kernels of the two-field and the
// three-field systems (device code, not part of the public ABI).
//
// General form of every deformation family:
//     chi(yhat) = A yhat + b (sin pi y1 sin pi y2, 0) (+ a translation),
//     F = A + b pi [[cos pi y1 sin pi y2, sin pi y1 cos pi y2], [0, 0]].
// The operators see the map only through J = det F, C = J F^-1 D F^-T in the
// cells and s = |cof(F) nu| on the edges (Sec. 3.1, Eqs. (13), (14), (16)).
#pragma once

#include "tsf_internal.cuh"

namespace tsf {

struct Deform {
    double A11, A12, A21, A22, bpi;
};

__device__ __forceinline__ Deform load_deform(const double* prm5, int i) {
    const double* pr = prm5 + (size_t)i * 5;
    return Deform{pr[0], pr[1], pr[2], pr[3], pr[4] * 3.14159265358979323846};
}

// F at reference point (y1, y2) given sin/cos of pi*y1, pi*y2.
__device__ __forceinline__ void jacobian(const Deform& d, double s1, double c1, double s2, double c2, double& F11,
                                         double& F12, double& F21, double& F22) {
    F11 = fma(d.bpi, c1 * s2, d.A11);
    F12 = fma(d.bpi, s1 * c2, d.A12);
    F21 = d.A21;
    F22 = d.A22;
}

// 2-point Gauss abscissae on [0,1]
constexpr double kGauss0 = 0.5 - 0.28867513459481288225;
constexpr double kGauss1 = 0.5 + 0.28867513459481288225;

// Bilinear shape function l (0: (0,0), 1: (1,0), 2: (0,1), 3: (1,1) corner of
// the cell) and its derivatives at local point (s, t), by selects (no arrays:
// the element loops below keep every per-thread value in registers).
__device__ __forceinline__ double q1_phi(int l, double s, double t) {
    return ((l & 1) ? s : 1.0 - s) * ((l & 2) ? t : 1.0 - t);
}
__device__ __forceinline__ double q1_ds(int l, double t) {
    const double b = (l & 2) ? t : 1.0 - t;
    return (l & 1) ? b : -b;
}
__device__ __forceinline__ double q1_dt(int l, double s) {
    const double a = (l & 1) ? s : 1.0 - s;
    return (l & 2) ? a : -a;
}

// Stored plane (0 C, 1 E, 2 N, 3 NE, 4 NW) of the coupling between local
// node la of a cell and local node lb of the same cell, seen from la; -1 for
// the couplings stored at the other node.
__host__ __device__ constexpr int q1_plane(int la, int lb) {
    return ((lb & 1) - (la & 1) == 0 && (lb >> 1) - (la >> 1) == 0)   ? 0
           : ((lb & 1) - (la & 1) == 1 && (lb >> 1) - (la >> 1) == 0) ? 1
           : ((lb & 1) - (la & 1) == 0 && (lb >> 1) - (la >> 1) == 1) ? 2
           : ((lb & 1) - (la & 1) == 1 && (lb >> 1) - (la >> 1) == 1) ? 3
           : ((lb & 1) - (la & 1) == -1 && (lb >> 1) - (la >> 1) == 1) ? 4
                                                                       : -1;
}

// The five stored couplings of node (p, q) in M = int J eta eta and in
// A = int C grad eta . grad eta, summed over the (up to four) cells around the
// node with 2x2 Gauss points; lump = row sum of M; bad = some J <= 0.  Every
// loop is unrolled, so the local node numbers and planes are compile-time
// constants and nothing is indexed at run time.
__device__ __forceinline__ void node_couplings(const Deform& d, double D11, double D12, double D22, int p, int q,
                                               int N, double (&m)[kPlanes], double (&k)[kPlanes], double& lump,
                                               bool& bad) {
    const double h = 1.0 / N;
#pragma unroll
    for (int c = 0; c < kPlanes; ++c) m[c] = k[c] = 0.0;
    lump = 0.0;
    bad = false;
#pragma unroll
    for (int cb = 0; cb < 2; ++cb) {
        const int b = q - 1 + cb;
#pragma unroll
        for (int ca = 0; ca < 2; ++ca) {
            const int ac = p - 1 + ca;
            if (b < 0 || b >= N || ac < 0 || ac >= N) continue;
            // local index of node (p, q) in this cell: (1 - ca) + 2 (1 - cb)
            const int la = (1 - ca) + 2 * (1 - cb);
#pragma unroll
            for (int qt = 0; qt < 2; ++qt) {
                const double t = qt ? kGauss1 : kGauss0;
                double s2, c2;
                sincospi((b + t) * h, &s2, &c2);
#pragma unroll
                for (int qs = 0; qs < 2; ++qs) {
                    const double s = qs ? kGauss1 : kGauss0;
                    double s1, c1;
                    sincospi((ac + s) * h, &s1, &c1);
                    double F11, F12, F21, F22;
                    jacobian(d, s1, c1, s2, c2, F11, F12, F21, F22);
                    const double J = F11 * F22 - F12 * F21;
                    if (!(J > 0.0)) bad = true;
                    // C = J F^-1 D F^-T = G D G^T / J with G = adj(F) = J F^-1
                    const double G11 = F22, G12 = -F12, G21 = -F21, G22 = F11;
                    const double GD11 = G11 * D11 + G12 * D12, GD12 = G11 * D12 + G12 * D22;
                    const double GD21 = G21 * D11 + G22 * D12, GD22 = G21 * D12 + G22 * D22;
                    const double iJ = 1.0 / J;
                    const double C11 = (GD11 * G11 + GD12 * G12) * iJ;
                    const double C12 = (GD11 * G21 + GD12 * G22) * iJ;
                    const double C22 = (GD21 * G21 + GD22 * G22) * iJ;
                    const double wm = 0.25 * h * h * J;
                    const double pa = q1_phi(la, s, t), dsa = q1_ds(la, t), dta = q1_dt(la, s);
                    const double gs = C11 * dsa + C12 * dta;
                    const double gt = C12 * dsa + C22 * dta;
#pragma unroll
                    for (int lb = 0; lb < 4; ++lb) {
                        const double me = wm * pa * q1_phi(lb, s, t);
                        lump += me;
                        const double ke = 0.25 * (gs * q1_ds(lb, t) + gt * q1_dt(lb, s));
#pragma unroll
                        for (int c = 0; c < kPlanes; ++c) {
                            // la is fixed by (ca, cb) and lb by the unrolled loop
                            if (c == q1_plane(la, lb)) {
                                m[c] += me;
                                k[c] += ke;
                            }
                        }
                    }
                }
            }
        }
    }
}

// Reference element tables of the unit square with 2x2 Gauss points (exact
// for Q1): ref[0..15] = int phi_a phi_b, ref[16..31] = int d_s phi_a d_s phi_b,
// ref[32..47] = int d_s phi_a d_t phi_b, ref[48..63] = int d_t phi_a d_t phi_b,
// entry a * 4 + b.  Filled by threads 0..15 of a block.
__device__ __forceinline__ void fill_reference_tables(double* ref) {
    const int e = threadIdx.x;
    if (e >= 16) return;
    const int la = e >> 2, lb = e & 3;
    double m = 0.0, ss = 0.0, st = 0.0, tt = 0.0;
#pragma unroll
    for (int qt = 0; qt < 2; ++qt) {
        const double t = qt ? kGauss1 : kGauss0;
#pragma unroll
        for (int qs = 0; qs < 2; ++qs) {
            const double s = qs ? kGauss1 : kGauss0;
            m += 0.25 * q1_phi(la, s, t) * q1_phi(lb, s, t);
            ss += 0.25 * q1_ds(la, t) * q1_ds(lb, t);
            st += 0.25 * q1_ds(la, t) * q1_dt(lb, s);
            tt += 0.25 * q1_dt(la, s) * q1_dt(lb, s);
        }
    }
    ref[e] = m;
    ref[16 + e] = ss;
    ref[32 + e] = st;
    ref[48 + e] = tt;
}

// node_couplings for an affine map (b = 0): F, J and C are the same at every
// quadrature point, so the element matrices are J h^2 Mref and
// C11 Kss + C12 (Kst + Kst^T) + C22 Ktt of the reference tables.
__device__ __forceinline__ void node_couplings_affine(const Deform& d, double D11, double D12, double D22, int p,
                                                      int q, int N, const double* ref, double (&m)[kPlanes],
                                                      double (&k)[kPlanes], double& lump, bool& bad) {
    const double h = 1.0 / N;
#pragma unroll
    for (int c = 0; c < kPlanes; ++c) m[c] = k[c] = 0.0;
    lump = 0.0;
    const double F11 = d.A11, F12 = d.A12, F21 = d.A21, F22 = d.A22;
    const double J = F11 * F22 - F12 * F21;
    bad = !(J > 0.0);
    const double G11 = F22, G12 = -F12, G21 = -F21, G22 = F11;
    const double GD11 = G11 * D11 + G12 * D12, GD12 = G11 * D12 + G12 * D22;
    const double GD21 = G21 * D11 + G22 * D12, GD22 = G21 * D12 + G22 * D22;
    const double iJ = 1.0 / J;
    const double C11 = (GD11 * G11 + GD12 * G12) * iJ;
    const double C12 = (GD11 * G21 + GD12 * G22) * iJ;
    const double C22 = (GD21 * G21 + GD22 * G22) * iJ;
    const double Jh2 = J * h * h;
#pragma unroll
    for (int cb = 0; cb < 2; ++cb) {
        const int b = q - 1 + cb;
#pragma unroll
        for (int ca = 0; ca < 2; ++ca) {
            const int ac = p - 1 + ca;
            if (b < 0 || b >= N || ac < 0 || ac >= N) continue;
            const int la = (1 - ca) + 2 * (1 - cb);
#pragma unroll
            for (int lb = 0; lb < 4; ++lb) {
                const int e = la * 4 + lb;
                const double me = Jh2 * ref[e];
                lump += me;
                const double ke =
                    C11 * ref[16 + e] + C12 * (ref[32 + e] + ref[32 + lb * 4 + la]) + C22 * ref[48 + e];
#pragma unroll
                for (int c = 0; c < kPlanes; ++c) {
                    if (c == q1_plane(la, lb)) {
                        m[c] += me;
                        k[c] += ke;
                    }
                }
            }
        }
    }
}

// Edges of the reference cell: 0 yhat_1 = 0, 1 yhat_1 = 1 (the nodes are
// numbered by q along them), 2 yhat_2 = 0, 3 yhat_2 = 1 (numbered by p).
enum : int { kEdgeLeft = 0, kEdgeRight = 1, kEdgeBottom = 2, kEdgeTop = 3 };

// Boundary mass R = int_edge s eta eta of one edge node (index t along the
// edge), s = |cof(F) nu|: |(F22, -F12)| on vertical edges, |(-F21, F11)| on
// horizontal ones; 2-point Gauss per segment.  Rd = diagonal, Ru = coupling to
// the next node along the edge, Rdn = coupling to the previous one.
__device__ __forceinline__ void edge_node_mass(const Deform& d, int edge, int t, int N, double& Rd, double& Ru,
                                               double& Rdn) {
    const double h = 1.0 / N;
    Rd = Ru = Rdn = 0.0;
    const bool vertical = edge == kEdgeLeft || edge == kEdgeRight;
    double sf, cf;  // sin/cos of pi times the fixed coordinate (0 or 1)
    sincospi((edge == kEdgeRight || edge == kEdgeTop) ? 1.0 : 0.0, &sf, &cf);
    const bool affine = d.bpi == 0.0;   // F = A: no trigonometry needed
    for (int seg = 0; seg < 2; ++seg) {
        const int b = t - 1 + seg;  // segment [b, b+1]
        if (b < 0 || b >= N) continue;
        for (int qt = 0; qt < 2; ++qt) {
            const double g = qt ? kGauss1 : kGauss0;
            double sa = 0.0, ca = 1.0;
            if (!affine) sincospi((b + g) * h, &sa, &ca);
            double F11, F12, F21, F22;
            if (vertical) jacobian(d, sf, cf, sa, ca, F11, F12, F21, F22);
            else jacobian(d, sa, ca, sf, cf, F11, F12, F21, F22);
            const double sg = vertical ? sqrt(F22 * F22 + F12 * F12) : sqrt(F21 * F21 + F11 * F11);
            const double w = 0.5 * h * sg;
            if (seg == 0) {  // node is the upper end (phi = g)
                Rd += w * g * g;
                Rdn += w * g * (1 - g);
            } else {         // node is the lower end (phi = 1 - g)
                Rd += w * (1 - g) * (1 - g);
                Ru += w * (1 - g) * g;
            }
        }
    }
}

}  // namespace tsf
