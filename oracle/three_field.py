"""Stationary three-field two-scale system -- TEST INFRASTRUCTURE ONLY.

The paper's full model (Eq. (5)) with the pulled-back discrete form of
Eq. (17): a macro field u (Dirichlet on the edges of ``dir_mask``, Neumann
data elsewhere), one micro field v_i per macro node on the reference cell
[0,1]^2, and a macro field w (Neumann).  Robin coupling on two edges of the
reference cell: the inflow edge Gamma_I (yhat_1 = 0) with
D grad v . n = kappa_1 u - kappa_2 v + g_1 and the outflow edge Gamma_O
(yhat_1 = 1) with kappa_3 w - kappa_4 v + g_2.  The edges yhat_2 = 0, 1 carry
the flux data g_3 (Eq. (18)).  The readings match the two-field step:

* one micro system per macro node (nodal collocation in x, Sec. 3.3);
* the coupling integrals in the macro equations are lumped at the node:
  kappa_1 m_k |Gamma_I,k| u_k - kappa_2 m_k r_I,k^T v_k in the u equation
  (likewise kappa_3, kappa_4 and Gamma_O in the w equation), m = row sums
  of M_H;
* the boundary measure is |cof(F) nu| (Eq. (16)); Q1 elements with 2x2 Gauss
  in cells and 2-point Gauss on edges;
* data are nodal values, integrated as their Q1 interpolants.

Unknowns X = (u, v_1 .. v_nM, w).  The monolithic matrix, with Dirichlet rows
of u replaced by identity rows, is:

    u rows: (K_H + kappa_1 L Gam_I) u - kappa_2 L rho_I(v)
            = M_H f^u - L (r_I^T g_1) + B g^u
    v rows: (A_i + kappa_2 R_I,i + kappa_4 R_O,i) v_i - kappa_1 r_I,i u_i - kappa_3 r_O,i w_i
            = M_i f^v_i + R_I g_1 + R_O g_2 + R_B g_3 + R_T g_3
    w rows: (D^w K_H + kappa_3 L Gam_O) w - kappa_4 L rho_O(v)
            = M_H f^w - L (r_O^T g_2) + B g^w

L = diag(m), Gam_I = diag(|Gamma_I,k|), rho_I(v)_k = r_I,k^T v_k, and
B = the 1D Q1 boundary mass.  ``solve`` factorises it with a sparse LU (no
iteration).  ``dt`` adds M_H/dt, M_i/dt and M_H/dt to the three diagonal
blocks (one implicit Euler step) for the tests that reduce the system to the
two-field step.

The micro M_i and A_i come from ``assemble_q1`` (pinned with the two-field
oracle); the four edge mass matrices are assembled here.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import assemble_q1, chi_many

EDGE_LEFT, EDGE_RIGHT, EDGE_BOTTOM, EDGE_TOP = 0, 1, 2, 3   # edges of the micro reference cell
_G2 = 0.5 + np.array([-0.5, 0.5]) / np.sqrt(3.0)            # 2-point Gauss on [0, 1]


def edge_nodes(N: int, edge: int) -> np.ndarray:
    """micro node indices along a reference edge (by q for left/right, by p for bottom/top)"""
    n1 = N + 1
    t = np.arange(n1)
    return {EDGE_LEFT: n1 * t, EDGE_RIGHT: n1 * t + N, EDGE_BOTTOM: t, EDGE_TOP: n1 * N + t}[edge]


def edge_mass(N: int, family: int, prm, edge: int) -> sp.csr_matrix:
    """R_e = int_edge |cof(F) nu| eta_j eta_l dyhat (Eq. (16)) on one edge of [0,1]^2."""
    n1, h = N + 1, 1.0 / N
    seg = np.repeat(np.arange(N), 2)
    t = np.tile(_G2, N)
    along = (seg + t) * h
    fixed = np.ones_like(along) if edge in (EDGE_RIGHT, EDGE_TOP) else np.zeros_like(along)
    if edge in (EDGE_LEFT, EDGE_RIGHT):
        _, F = chi_many(family, prm, fixed, along)
        s = np.hypot(F[:, 1, 1], F[:, 0, 1])      # |cof(F) e_1| = |(F22, -F12)|
    else:
        _, F = chi_many(family, prm, along, fixed)
        s = np.hypot(F[:, 1, 0], F[:, 0, 0])      # |cof(F) e_2| = |(-F21, F11)|
    nodes = edge_nodes(N, edge)
    a, b = nodes[seg], nodes[seg + 1]
    w = 0.5 * h * s
    rows = np.concatenate([a, a, b, b])
    cols = np.concatenate([a, b, a, b])
    vals = np.concatenate([w * (1 - t) ** 2, w * (1 - t) * t, w * t * (1 - t), w * t * t])
    return sp.csr_matrix((vals, (rows, cols)), shape=(n1 * n1, n1 * n1))


def macro_edge_nodes(NM: int):
    """macro node indices per edge: bottom (by p), right (by q), top (by p), left (by q)"""
    n1 = NM + 1
    t = np.arange(n1)
    return [t, n1 * t + NM, n1 * NM + t, n1 * t]


def boundary_load(NM: int, L: float, g) -> np.ndarray:
    """int_{boundary} g xi_k for Q1 nodal data g [4][NM+1] per edge (1D consistent mass)"""
    out = np.zeros((NM + 1) ** 2)
    if g is None:
        return out
    H = L / NM
    for e, nodes in enumerate(macro_edge_nodes(NM)):
        ge = np.asarray(g[e], float)
        for s in range(NM):
            a, b = nodes[s], nodes[s + 1]
            out[a] += H / 6.0 * (2.0 * ge[s] + ge[s + 1])
            out[b] += H / 6.0 * (ge[s] + 2.0 * ge[s + 1])
    return out


def dirichlet_nodes(NM: int, dir_mask: int) -> np.ndarray:
    mask = np.zeros((NM + 1) ** 2, bool)
    for e, nodes in enumerate(macro_edge_nodes(NM)):
        if dir_mask >> e & 1:
            mask[nodes] = True
    return mask


class ThreeField:
    """Sparse monolithic solve of the stationary (or one implicit Euler step of
    the) three-field system."""

    def __init__(self, Nm, NM, family, params, D=(1.0, 0.0, 1.0), Dw=1.0, kappa=(1.0, 1.0, 1.0, 1.0), x0=0.0,
                 L=1.0, dir_mask=0):
        self.Nm, self.NM, self.family = int(Nm), int(NM), int(family)
        self.nm, self.nM = (self.Nm + 1) ** 2, (self.NM + 1) ** 2
        self.D, self.Dw, self.kappa = tuple(D), float(Dw), tuple(float(k) for k in kappa)
        self.x0, self.L, self.dir_mask = float(x0), float(L), int(dir_mask)
        self.params = np.asarray(params, float).reshape(self.nM, -1)
        MH1, KH, _ = assemble_q1(self.NM, 0, [], (1.0, 0.0, 1.0))   # unit square: scale M by L^2
        self.MH, self.KH = (self.L ** 2) * MH1, KH
        self.m = np.asarray(self.MH.sum(axis=1)).ravel()
        self.dir = dirichlet_nodes(self.NM, self.dir_mask)
        self.blocks = []
        for i in range(self.nM):
            M, A, _ = assemble_q1(self.Nm, self.family, self.params[i], self.D)
            R = [edge_mass(self.Nm, self.family, self.params[i], e) for e in range(4)]
            self.blocks.append((M, A, R))
        ones = np.ones(self.nm)
        self.rI = np.array([R[EDGE_LEFT] @ ones for (_, _, R) in self.blocks])
        self.rO = np.array([R[EDGE_RIGHT] @ ones for (_, _, R) in self.blocks])
        self.gamI, self.gamO = self.rI.sum(axis=1), self.rO.sum(axis=1)
        self.vol = np.array([M.sum() for (M, _, _) in self.blocks])

    def micro_operator(self, i, dt=None):
        M, A, R = self.blocks[i]
        k1, k2, k3, k4 = self.kappa
        S = A + k2 * R[EDGE_LEFT] + k4 * R[EDGE_RIGHT]
        return S + M / dt if dt else S

    def matrix(self, dt=None) -> sp.csc_matrix:
        nM, nm = self.nM, self.nm
        k1, k2, k3, k4 = self.kappa
        Au = self.KH + sp.diags(k1 * self.m * self.gamI)
        Aw = self.Dw * self.KH + sp.diags(k3 * self.m * self.gamO)
        if dt:
            Au = Au + self.MH / dt
            Aw = Aw + self.MH / dt
        nmv = nM * nm
        ii = np.repeat(np.arange(nM), nm)          # macro node of every micro unknown
        jj = np.arange(nmv)
        keep = ~self.dir[ii]                       # Dirichlet rows of u have no coupling
        Cuv = sp.csr_matrix(((-k2 * self.m[:, None] * self.rI).ravel()[keep], (ii[keep], jj[keep])), shape=(nM, nmv))
        Cwv = sp.csr_matrix(((-k4 * self.m[:, None] * self.rO).ravel(), (ii, jj)), shape=(nM, nmv))
        Cvu = sp.csr_matrix(((-k1 * self.rI).ravel(), (jj, ii)), shape=(nmv, nM))
        Cvw = sp.csr_matrix(((-k3 * self.rO).ravel(), (jj, ii)), shape=(nmv, nM))
        Au = Au.tolil()
        for k in np.nonzero(self.dir)[0]:
            Au[k, :] = 0.0
            Au[k, k] = 1.0
        Smic = sp.block_diag([self.micro_operator(i, dt) for i in range(nM)])
        return sp.bmat([[Au.tocsr(), Cuv, None], [Cvu, Smic, Cvw], [None, Cwv, sp.csr_matrix(Aw)]], format="csc")

    def rhs(self, fu=None, fw=None, ud=None, gu=None, gw=None, fv=None, gI=None, gO=None, gN=None, dt=None,
            prev=None) -> np.ndarray:
        nM, nm, Nm = self.nM, self.nm, self.Nm
        z = np.zeros(nM)
        bu = self.MH @ (z if fu is None else np.asarray(fu, float))
        bw = self.MH @ (z if fw is None else np.asarray(fw, float))
        GI = np.zeros(nM)
        GO = np.zeros(nM)
        bv = np.zeros((nM, nm))
        for i in range(nM):
            M, _, R = self.blocks[i]
            if fv is not None:
                bv[i] += M @ np.asarray(fv, float).reshape(nM, nm)[i]
            for e, data in ((EDGE_LEFT, gI), (EDGE_RIGHT, gO)):
                if data is not None:
                    full = np.zeros(nm)
                    full[edge_nodes(Nm, e)] = np.asarray(data, float).reshape(nM, Nm + 1)[i]
                    bv[i] += R[e] @ full
                    if e == EDGE_LEFT:
                        GI[i] = self.rI[i] @ full
                    else:
                        GO[i] = self.rO[i] @ full
            if gN is not None:
                gn = np.asarray(gN, float).reshape(nM, 2, Nm + 1)[i]
                for e, row in ((EDGE_BOTTOM, 0), (EDGE_TOP, 1)):
                    full = np.zeros(nm)
                    full[edge_nodes(Nm, e)] = gn[row]
                    bv[i] += R[e] @ full
        bu += -self.m * GI
        bw += -self.m * GO
        if gu is not None:
            gmask = np.array(gu, float)
            for e in range(4):
                if self.dir_mask >> e & 1:
                    gmask[e] = 0.0
            bu += boundary_load(self.NM, self.L, gmask)
        bw += boundary_load(self.NM, self.L, gw)
        if dt:
            u0, v0, w0 = prev
            bu += self.MH @ np.asarray(u0, float) / dt
            bw += self.MH @ np.asarray(w0, float) / dt
            v0 = np.asarray(v0, float).reshape(nM, nm)
            for i in range(nM):
                bv[i] += self.blocks[i][0] @ v0[i] / dt
        dvals = np.zeros(nM) if ud is None else np.asarray(ud, float)
        bu[self.dir] = dvals[self.dir]
        return np.concatenate([bu, bv.ravel(), bw])

    def solve(self, dt=None, prev=None, **sources):
        """(u [nM], w [nM], v [nM][nm])"""
        if not dt and not self.dir.any():
            # the constant equilibrium state spans the null space (Sec. 2.2 asks
            # for a non-empty Dirichlet boundary)
            raise ValueError("the stationary system needs at least one Dirichlet edge")
        A = self.matrix(dt)
        X = spla.spsolve(A, self.rhs(dt=dt, prev=prev, **sources))
        nM, nm = self.nM, self.nm
        return X[:nM], X[nM + nM * nm:], X[nM:nM + nM * nm].reshape(nM, nm)

    def vbar(self, v) -> np.ndarray:
        v = np.asarray(v, float).reshape(self.nM, self.nm)
        return np.array([self.blocks[i][0].sum(axis=0) @ v[i] for i in range(self.nM)]) / self.vol

    def symmetric_scaling(self) -> np.ndarray:
        """row weights that make the stationary matrix symmetric: kappa_1/kappa_2 on
        u rows, m_i on the rows of v_i, kappa_3/kappa_4 on w rows"""
        k1, k2, k3, k4 = self.kappa
        return np.concatenate([np.full(self.nM, k1 / k2), np.repeat(self.m, self.nm), np.full(self.nM, k3 / k4)])
