"""Discrete adjoint of the implicit two-scale march -- TEST INFRASTRUCTURE ONLY.

Objective: J = sum_k m_k u_k^N, the mean of the macro field over
Omega = [0,1]^2 after N implicit Euler steps (m = row sums of M_H, so this is
the exact integral of the Q1 field).  With X = (u, v_1, ..., v_nM) one step
of the coupled system (Sec. 3.3, one micro system per macro node; discrete
form Eq. (17) made parabolic) reads

    A(p) X^{n+1} = B(p) X^n,
    A = [[M_H/dt + Du K_H + kappa L Gam,   -kappa L r^T       ],
         [-kappa r_i e_i^T,               M_i/dt + A_i + kappa R_i]],
    B = diag(M_H/dt, M_i/dt),

with Dirichlet macro rows replaced by identity rows.  Here everything is
solved with sparse direct factorisations (no iteration), and the adjoint is
the literal transpose:

    A^T lam^N = dJ/dX^N,   A^T lam^n = B^T lam^{n+1},
    dJ/dp = - sum_{n=0}^{N-1} lam^{n+1}^T (dA/dp X^{n+1} - dB/dp X^n),

with dA/dp, dB/dp assembled from the analytic derivatives of J, C and
|cof(F) nu| at every quadrature point (or_assemble_q1_dparam).  Sources are
not supported (they would add their own derivative terms).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import NPARAM, Problem, assemble_q1, assemble_q1_dparam


def _boundary(NM):
    n1 = NM + 1
    k = np.arange(n1 * n1)
    p, q = k % n1, k // n1
    return (p == 0) | (q == 0) | (p == NM) | (q == NM)


class TwoScaleAdjoint:
    """Sparse monolithic forward march and its discrete adjoint."""

    def __init__(self, Nm, NM, bc, family, params, D=(1.0, 0.0, 1.0), kappa=1.0, Du=1.0):
        self.Nm, self.NM, self.bc, self.family = Nm, NM, bc, family
        self.D, self.kappa, self.Du = D, kappa, Du
        self.params = np.asarray(params, dtype=float).reshape((NM + 1) ** 2, -1)
        self.nM, self.nm = (NM + 1) ** 2, (Nm + 1) ** 2
        P = Problem(Nm, NM, bc, family, self.params, D=D, kappa=kappa, Du=Du)
        self.MH = P.macro_csr("M")
        self.KH = P.macro_csr("K")
        self.m = np.asarray(self.MH.sum(axis=1)).ravel()
        self.dir = _boundary(NM) if bc == 1 else np.zeros(self.nM, bool)
        self.blocks = [assemble_q1(Nm, family, self.params[i], D) for i in range(self.nM)]

    def matrices(self, dt):
        nM, nm, kap = self.nM, self.nm, self.kappa
        r = [Ri @ np.ones(nm) for (_, _, Ri) in self.blocks]
        gam = np.array([ri.sum() for ri in r])
        AH = (self.MH / dt + self.Du * self.KH + sp.diags(kap * self.m * gam)).tolil()
        Cuv = sp.lil_matrix((nM, nM * nm))
        Cvu = sp.lil_matrix((nM * nm, nM))
        for i in range(nM):
            Cuv[i, i * nm:(i + 1) * nm] = -kap * self.m[i] * r[i]
            Cvu[i * nm:(i + 1) * nm, i] = (-kap * r[i]).reshape(-1, 1)
        for k in np.nonzero(self.dir)[0]:
            AH[k, :] = 0.0
            AH[k, k] = 1.0
            Cuv[k, :] = 0.0
        Smic = sp.block_diag([M / dt + A + kap * R for (M, A, R) in self.blocks])
        A = sp.bmat([[AH.tocsr(), Cuv.tocsr()], [Cvu.tocsr(), Smic]], format="csc")
        BH = (self.MH / dt).tolil()
        for k in np.nonzero(self.dir)[0]:
            BH[k, :] = 0.0
            BH[k, k] = 1.0   # Dirichlet rows keep u_k
        B = sp.block_diag([BH.tocsr()] + [M / dt for (M, _, _) in self.blocks], format="csr")
        return A, B

    def forward(self, u0, v0, dt, nsteps):
        """States X^0..X^N and J."""
        A, B = self.matrices(dt)
        lu = spla.splu(A)
        X = [np.concatenate([np.asarray(u0, float), np.asarray(v0, float).ravel()])]
        for _ in range(nsteps):
            X.append(lu.solve(B @ X[-1]))
        J = float(self.m @ X[-1][:self.nM])
        return X, J

    def gradient(self, u0, v0, dt, nsteps):
        """(J, dJ/dparams [nM, nparam]) by the discrete adjoint."""
        A, B = self.matrices(dt)
        X, J = self.forward(u0, v0, dt, nsteps)
        luT = spla.splu(A.T.tocsc())
        nM, nm, kap = self.nM, self.nm, self.kappa
        g = np.zeros(nM * nm + nM)
        g[:nM] = self.m
        lam = luT.solve(g)
        npar = NPARAM[self.family]
        grad = np.zeros((nM, npar))
        dmat = [[assemble_q1_dparam(self.Nm, self.family, self.params[i], k, self.D) for k in range(npar)]
                for i in range(nM)]
        for n in range(nsteps - 1, -1, -1):
            # lam = lam^{n+1}; contribution of step n
            mu, nu = lam[:nM], lam[nM:].reshape(nM, nm)
            u1, v1 = X[n + 1][:nM], X[n + 1][nM:].reshape(nM, nm)
            v0n = X[n][nM:].reshape(nM, nm)
            for i in range(nM):
                for k in range(npar):
                    dM, dA, dR = dmat[i][k]
                    dr = dR @ np.ones(nm)
                    dgam = dr.sum()
                    t = nu[i] @ ((dM / dt + dA + kap * dR) @ v1[i] - kap * dr * u1[i] - dM @ v0n[i] / dt)
                    if not self.dir[i]:
                        t += mu[i] * kap * self.m[i] * (dgam * u1[i] - dr @ v1[i])
                    grad[i, k] -= t
            if n > 0:
                lam = luT.solve(B.T @ lam)
        return J, grad
