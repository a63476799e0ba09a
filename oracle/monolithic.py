"""Dense direct solve of one implicit Euler step of the coupled system.

TEST INFRASTRUCTURE ONLY (part of the oracle).  This is the second route to
the coupled fixed point: instead of the partitioned macro/micro iteration of
Sec. 3.3 it writes the whole step as one linear system in (u, v_1..v_nM),

    [ M_H/dt + Du K_H + kappa L Gam      -kappa L r^T    ] [u]   [ M_H(u^n/dt + fu) - L G ]
    [ -kappa r_i e_i^T            M_i/dt + A_i + kappa R_i ] [v] = [ M_i(v^n/dt + fv) + R_i g ]

(Dirichlet macro rows replaced by u_k = ud_k) and solves it with LAPACK
(numpy.linalg.solve).  The blocks are the oracle's assembled matrices; the
solver path (no CG, no coupling iteration) is independent.  Tiny meshes only.
"""
from __future__ import annotations

import numpy as np


def _boundary_mask(NM):
    n1 = NM + 1
    k = np.arange(n1 * n1)
    p, q = k % n1, k // n1
    return (p == 0) | (q == 0) | (p == NM) | (q == NM)


def monolithic_matrix(P, dt, Du=1.0, bc=0):
    """Dense monolithic matrix of one implicit Euler step (Dirichlet rows as identity)."""
    nM, nm = P.nM, P.nm
    kap = P.kappa
    gam, vol, mH = P.geometry()
    r = P.r
    N = nM + nM * nm
    A = np.zeros((N, N))
    MH = P.macro_csr("M").toarray()
    KH = P.macro_csr("K").toarray()
    A[:nM, :nM] = MH / dt + Du * KH + np.diag(kap * mH * gam)
    for i in range(nM):
        s = nM + i * nm
        A[i, s:s + nm] = -kap * mH[i] * r[i]
        Si = (P.micro_csr(i, "M") / dt + P.micro_csr(i, "A") + kap * P.micro_csr(i, "R")).toarray()
        A[s:s + nm, s:s + nm] = Si
        A[s:s + nm, i] = -kap * r[i]
    if bc == 1:
        for k in np.nonzero(_boundary_mask(P.NM))[0]:
            A[k, :] = 0.0
            A[k, k] = 1.0
    return A


def monolithic_step(P, u_n, v_n, dt, Du=1.0, bc=0, fv=None, g=None, fu=None, ud=None):
    """One implicit Euler step solved directly; returns (u, v[nM, nm])."""
    nM, nm, Nm = P.nM, P.nm, P.Nm
    gam, vol, mH = P.geometry()
    r = P.r
    A = monolithic_matrix(P, dt, Du, bc)
    rhs = np.zeros(nM + nM * nm)
    MH = P.macro_csr("M")
    fuv = np.zeros(nM) if fu is None else np.asarray(fu)
    rhs[:nM] = MH @ (np.asarray(u_n) / dt + fuv)
    v_n = np.asarray(v_n).reshape(nM, nm)
    gfull = np.zeros((nM, nm))
    if g is not None:
        gg = np.asarray(g).reshape(nM, Nm + 1)
        gfull[:, Nm + (Nm + 1) * np.arange(Nm + 1)] = gg
        rhs[:nM] -= mH * np.einsum("ij,ij->i", r, gfull)
    for i in range(nM):
        s = nM + i * nm
        w = v_n[i] / dt
        if fv is not None:
            w = w + np.asarray(fv).reshape(nM, nm)[i]
        rhs[s:s + nm] = P.micro_csr(i, "M") @ w + P.micro_csr(i, "R") @ gfull[i]
    if bc == 1:
        bnd = np.nonzero(_boundary_mask(P.NM))[0]
        rhs[bnd] = (np.asarray(u_n) if ud is None else np.asarray(ud))[bnd]
    x = np.linalg.solve(A, rhs)
    return x[:nM], x[nM:].reshape(nM, nm)
