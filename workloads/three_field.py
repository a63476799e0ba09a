"""Inputs of the stationary three-field system (input data only).

The paper's full model (Eq. (5)): a macro nutrient u with a Dirichlet part of
the boundary, a micro field v in every cell, and a macro product w with a
Neumann boundary. v enters a cell through the inflow edge Gamma_I
(D grad v . n = kappa_1 u - kappa_2 v) and leaves through the outflow edge
Gamma_O (kappa_3 w - kappa_4 v); the other edges Gamma_N carry no flux. As in
the paper's numerical sections, Omega = Z = [-1, 1]^2 and the cell of node x is
Y_x = zeta(x, Z).

The library and the oracle take the micro reference cell as [0,1]^2 and the
macro mesh on [x0, x0 + L]^2.  A map zeta(x, z) on Z = [-1,1]^2 is handed over
as chi(yhat) = zeta(x, 2 yhat - 1); for the affine maps used here that is the
affine family (A, c) with A = 2 F and c = zeta(x, (-1, -1)).  On the reference
cell Gamma_I is the edge yhat_1 = 0 and Gamma_O is yhat_1 = 1 (the inflow
edge on the left and the outflow edge on the right, as in Fig. 1); Gamma_N is
made of yhat_2 = 0 and yhat_2 = 1.

Workloads:

* ``manufactured``: the manufactured solution of Eq. (19),
      u = x_1 sin x_0,  v = x_0 + x_1 + y_0 y_1 (1 - y_1),  w = x_0 cos x_1,
  on the affine cells of Eq. (19), with the data of Eq. (18) in closed
  form.  The printed data of Eq. (20) are partly garbled and are not used.
  The tests re-derive every function below with SymPy.  u is Dirichlet
  on all of the macro boundary.
* ``case_a`` / ``case_b``: the geometry experiment of Sec. 4.4 (Table 3 and
  Eq. (21)): zeta_0 = identity (Case A), zeta_1 (Case B), D^w = 0.1, D^v = 1,
  kappa = (0.5, 1, 0.25, 1), no sources, u = 1 on the left macro edge
  x_0 = -1, homogeneous Neumann elsewhere.  8 x 8 macro cells (81 nodes),
  64 x 64 micro cells (4225 nodes).  With these data the constant state
  u = 1, v = kappa_1/kappa_2, w = kappa_1 kappa_4 / (kappa_2 kappa_3) satisfies
  every equation and every boundary condition, so the solution is that
  constant in both cases, whatever the geometry.  ``sink=True`` adds
  u = 0 on the right macro edge x_0 = 1 (not in the paper), which gives
  non-constant profiles that do depend on the cells.

Data layout (shared by the library's three-field ABI and the oracle):

* macro node (p, q) -> index p + (NM+1) q, position x = x0 + (p, q) L / NM;
* micro node (p, q) -> index p + (Nm+1) q, reference yhat = (p, q) / Nm;
* ``fu``, ``fw``, ``ud``: [nM] nodal values; ``ud`` is read on Dirichlet nodes only;
* ``gu``, ``gw``: [4][NM+1] Neumann data of the macro edges in the order
  bottom (x_1 = x0, by p), right (by q), top (by p), left (x_0 = x0, by q);
* ``dir_mask``: bit e set = macro edge e (same order) is Dirichlet for u;
* ``fv``: [nM][nm] nodal values of f^v at the physical micro nodes;
* ``gI``, ``gO``: [nM][Nm+1] Robin data on Gamma_I (yhat_1 = 0) and Gamma_O
  (yhat_1 = 1), by q;
* ``gN``: [nM][2][Nm+1] flux data on yhat_2 = 0 and yhat_2 = 1, by p.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import FAMILY_AFFINE

EDGE_BOTTOM, EDGE_RIGHT, EDGE_TOP, EDGE_LEFT = 0, 1, 2, 3


@dataclasses.dataclass
class ThreeFieldWorkload:
    name: str
    NM: int
    Nm: int
    x0: float                     # macro domain [x0, x0 + L]^2
    L: float
    dir_mask: int                 # Dirichlet edges of u (bit e = edge e)
    family: int
    params: np.ndarray            # [nM, nparam]
    D: tuple = (1.0, 0.0, 1.0)    # D^v (D11, D12, D22)
    Dw: float = 1.0
    kappa: tuple = (1.0, 1.0, 1.0, 1.0)
    fu: np.ndarray = None
    fw: np.ndarray = None
    ud: np.ndarray = None
    gu: np.ndarray = None
    gw: np.ndarray = None
    fv: np.ndarray = None
    gI: np.ndarray = None
    gO: np.ndarray = None
    gN: np.ndarray = None
    tol: float = 1e-12

    @property
    def nM(self):
        return (self.NM + 1) ** 2

    @property
    def nm(self):
        return (self.Nm + 1) ** 2

    def sources(self):
        return dict(fu=self.fu, fw=self.fw, ud=self.ud, gu=self.gu, gw=self.gw, fv=self.fv, gI=self.gI,
                    gO=self.gO, gN=self.gN)


def macro_nodes(NM, x0, L):
    n1 = NM + 1
    k = np.arange(n1 * n1)
    return x0 + (k % n1) * (L / NM), x0 + (k // n1) * (L / NM)


def macro_edge_nodes(NM, x0, L):
    """positions [4][NM+1] x 2 of the macro boundary nodes per edge (bottom, right, top, left)"""
    t = x0 + np.arange(NM + 1) * (L / NM)
    lo, hi = np.full_like(t, x0), np.full_like(t, x0 + L)
    return [(t, lo), (hi, t), (t, hi), (lo, t)]


EDGE_NORMALS = np.array([[0.0, -1.0], [1.0, 0.0], [0.0, 1.0], [-1.0, 0.0]])


# ---------------------------------------------------------------------------
# manufactured solution (Eq. (19))
# ---------------------------------------------------------------------------
ZETA_F = np.array([[0.4 * 1.4, -0.4 * 0.54], [-0.3 * 0.4, 0.3 * 0.8]])   # d zeta / d z


def zeta_shift(x0_, x1_):
    """zeta(x, 0) for the map of Eq. (19)"""
    return 0.4 * (np.asarray(x0_) + 1.3), 0.3 * (np.asarray(x1_) + 1.2)


def u_mms(x0_, x1_):
    return x1_ * np.sin(x0_)


def grad_u_mms(x0_, x1_):
    return x1_ * np.cos(x0_), np.sin(x0_)


def w_mms(x0_, x1_):
    return x0_ * np.cos(x1_)


def grad_w_mms(x0_, x1_):
    return np.cos(x1_), -x0_ * np.sin(x1_)


def v_mms(x0_, x1_, y0, y1):
    return x0_ + x1_ + y0 * y1 * (1.0 - y1)


def grad_v_mms(x0_, x1_, y0, y1):
    """gradient with respect to the physical micro coordinate y"""
    return y1 * (1.0 - y1), y0 * (1.0 - 2.0 * y1)


def _cell_normals(F):
    """outward unit normals of zeta(x, Z) on z_0 = -1, z_0 = 1, z_1 = -1, z_1 = 1"""
    cof = np.array([[F[1, 1], -F[1, 0]], [-F[0, 1], F[0, 0]]])   # det(F) F^-T
    n0 = cof @ np.array([1.0, 0.0])
    n1 = cof @ np.array([0.0, 1.0])
    n0 /= np.linalg.norm(n0)
    n1 /= np.linalg.norm(n1)
    return -n0, n0, -n1, n1


def _flux_integral(Dv, F, x0_, x1_, z0_fixed):
    """int over the cell edge z_0 = z0_fixed of Dv grad v . n dsigma_y, for every
    macro point (exact: the integrand is a quadratic in the edge parameter,
    3-point Gauss-Legendre integrates it exactly)"""
    nI, nO, _, _ = _cell_normals(F)
    n = nO if z0_fixed > 0 else nI
    t0, t1 = zeta_shift(x0_, x1_)
    gl, gw = np.polynomial.legendre.leggauss(3)
    length = np.linalg.norm(F[:, 1])   # |d y / d z_1|
    total = 0.0
    for s, wt in zip(gl, gw):
        y0 = t0 + F[0, 0] * z0_fixed + F[0, 1] * s
        y1 = t1 + F[1, 0] * z0_fixed + F[1, 1] * s
        g0, g1 = grad_v_mms(x0_, x1_, y0, y1)
        total = total + wt * length * Dv * (g0 * n[0] + g1 * n[1])
    return total


def manufactured(NM: int, Nm: int, Dv: float = 1.0, Dw: float = 1.0, kappa=(1.0, 1.0, 1.0, 1.0),
                 tol: float = 1e-12) -> ThreeFieldWorkload:
    """The manufactured problem of Eqs. (18)-(19) on Omega = Z = [-1,1]^2."""
    k1, k2, k3, k4 = (float(k) for k in kappa)
    x0, L = -1.0, 2.0
    X0, X1 = macro_nodes(NM, x0, L)
    nM, n1m = X0.size, Nm + 1
    F = ZETA_F
    A = 2.0 * F
    t0, t1 = zeta_shift(X0, X1)
    c = np.stack([t0 - F[0, 0] - F[0, 1], t1 - F[1, 0] - F[1, 1]], axis=1)
    params = np.concatenate([np.tile(A.reshape(1, 4), (nM, 1)), c], axis=1)
    # macro data
    fu = u_mms(X0, X1) + _flux_integral(Dv, F, X0, X1, -1.0)          # -Lap u + int_GI Dv dv/dn
    fw = Dw * w_mms(X0, X1) + _flux_integral(Dv, F, X0, X1, 1.0)      # -Dw Lap w + int_GO Dv dv/dn
    ud = u_mms(X0, X1)
    gu = np.zeros((4, NM + 1))
    gw = np.zeros((4, NM + 1))
    for e, (ex0, ex1) in enumerate(macro_edge_nodes(NM, x0, L)):
        g0, g1 = grad_u_mms(ex0, ex1)
        gu[e] = g0 * EDGE_NORMALS[e, 0] + g1 * EDGE_NORMALS[e, 1]
        g0, g1 = grad_w_mms(ex0, ex1)
        gw[e] = Dw * (g0 * EDGE_NORMALS[e, 0] + g1 * EDGE_NORMALS[e, 1])
    # micro data at the physical images of the reference nodes
    yh = np.arange(n1m) / Nm
    YH1, YH2 = np.meshgrid(yh, yh, indexing="xy")
    Z0, Z1 = 2.0 * YH1.ravel() - 1.0, 2.0 * YH2.ravel() - 1.0
    y0 = t0[:, None] + F[0, 0] * Z0[None, :] + F[0, 1] * Z1[None, :]
    fv = np.broadcast_to(2.0 * Dv * y0, (nM, n1m * n1m)).copy()      # -Dv Lap_y v
    nI, nO, nB, nT = _cell_normals(F)
    zs = 2.0 * yh - 1.0

    def edge_vals(z0e, z1e):
        ye0 = t0[:, None] + F[0, 0] * z0e[None, :] + F[0, 1] * z1e[None, :]
        ye1 = t1[:, None] + F[1, 0] * z0e[None, :] + F[1, 1] * z1e[None, :]
        return ye0, ye1

    def dvdn(ye0, ye1, n):
        g0, g1 = grad_v_mms(X0[:, None], X1[:, None], ye0, ye1)
        return Dv * (g0 * n[0] + g1 * n[1])

    ye0, ye1 = edge_vals(np.full(n1m, -1.0), zs)                       # Gamma_I, by q
    vI = v_mms(X0[:, None], X1[:, None], ye0, ye1)
    gI = dvdn(ye0, ye1, nI) - k1 * u_mms(X0, X1)[:, None] + k2 * vI
    ye0, ye1 = edge_vals(np.full(n1m, 1.0), zs)                        # Gamma_O, by q
    vO = v_mms(X0[:, None], X1[:, None], ye0, ye1)
    gO = dvdn(ye0, ye1, nO) - k3 * w_mms(X0, X1)[:, None] + k4 * vO
    gN = np.zeros((nM, 2, n1m))
    ye0, ye1 = edge_vals(zs, np.full(n1m, -1.0))                       # yhat_2 = 0, by p
    gN[:, 0] = dvdn(ye0, ye1, nB)
    ye0, ye1 = edge_vals(zs, np.full(n1m, 1.0))                        # yhat_2 = 1, by p
    gN[:, 1] = dvdn(ye0, ye1, nT)
    return ThreeFieldWorkload("manufactured", NM, Nm, x0, L, 0b1111, FAMILY_AFFINE, params,
                              D=(Dv, 0.0, Dv), Dw=Dw, kappa=(k1, k2, k3, k4), fu=fu, fw=fw, ud=ud, gu=gu, gw=gw,
                              fv=fv, gI=gI, gO=gO, gN=gN, tol=tol)


def mms_exact(NM: int, Nm: int, w: ThreeFieldWorkload | None = None):
    """exact nodal u, w [nM] and v [nM][nm] of the manufactured problem"""
    X0, X1 = macro_nodes(NM, -1.0, 2.0)
    F = ZETA_F
    t0, t1 = zeta_shift(X0, X1)
    yh = np.arange(Nm + 1) / Nm
    YH1, YH2 = np.meshgrid(yh, yh, indexing="xy")
    Z0, Z1 = 2.0 * YH1.ravel() - 1.0, 2.0 * YH2.ravel() - 1.0
    y0 = t0[:, None] + F[0, 0] * Z0[None, :] + F[0, 1] * Z1[None, :]
    y1 = t1[:, None] + F[1, 0] * Z0[None, :] + F[1, 1] * Z1[None, :]
    return u_mms(X0, X1), w_mms(X0, X1), v_mms(X0[:, None], X1[:, None], y0, y1)


# ---------------------------------------------------------------------------
# geometry experiment (Sec. 4.4, Table 3, Eq. (21))
# ---------------------------------------------------------------------------
def zeta1_F(x0_, x1_):
    """d zeta_1 / d y of Eq. (21): [[(2 x_0 + 3)/4, -x_1/5], [0, (2 - x_1)/4]] per node"""
    x0_, x1_ = np.asarray(x0_, float), np.asarray(x1_, float)
    F = np.zeros(x0_.shape + (2, 2))
    F[..., 0, 0] = (2.0 * x0_ + 3.0) / 4.0
    F[..., 0, 1] = -x1_ / 5.0
    F[..., 1, 1] = (2.0 - x1_) / 4.0
    return F


def _case(name: str, heterogeneous: bool, NM: int, Nm: int, tol: float, sink: bool) -> ThreeFieldWorkload:
    x0, L = -1.0, 2.0
    X0, X1 = macro_nodes(NM, x0, L)
    nM = X0.size
    if heterogeneous:
        F = zeta1_F(X0, X1)             # zeta_1(x, 0) = 0, so c = -F (1, 1)
    else:
        F = np.broadcast_to(np.eye(2), (nM, 2, 2)).copy()
    A = 2.0 * F
    c = -(F[:, :, 0] + F[:, :, 1])
    params = np.concatenate([A.reshape(nM, 4), c], axis=1)
    mask = 1 << EDGE_LEFT
    ud = np.ones(nM)
    if sink:
        mask |= 1 << EDGE_RIGHT
        ud = np.where(X0 < x0 + 0.5 * L, 1.0, 0.0)
    return ThreeFieldWorkload(name + ("_sink" if sink else ""), NM, Nm, x0, L, mask, FAMILY_AFFINE, params,
                              D=(1.0, 0.0, 1.0), Dw=0.1, kappa=(0.5, 1.0, 0.25, 1.0), ud=ud, tol=tol)


def case_a(NM: int = 8, Nm: int = 64, tol: float = 1e-10, sink: bool = False) -> ThreeFieldWorkload:
    return _case("case_a", False, NM, Nm, tol, sink)


def case_b(NM: int = 8, Nm: int = 64, tol: float = 1e-10, sink: bool = False) -> ThreeFieldWorkload:
    return _case("case_b", True, NM, Nm, tol, sink)
