"""Manufactured solution for the parabolic u-v system (input data only).

The paper validates its method with manufactured solutions whose data are
derived symbolically (Sec. 4.1, Sec. 4.2).  Here the same idea is applied to
the time-dependent u-v system on Omega = Z = [0,1]^2 with D = I and the bump
deformation, which leaves every Y_x equal to [0,1]^2:

    u(x, t)    = (1 + t) U(x),     U = 1 + x2 sin(x1)
    v(x, y, t) = (1 + t) V(x, y),  V = x1 + x2 + y1^2 (1 + cos(pi y2) / 2)

V has zero normal derivative on y1 = 0, y2 = 0 and y2 = 1, so only the Robin
edge y1 = 1 carries data.  Being linear in t, the solution is integrated
exactly by implicit Euler, so the observed error is purely spatial.  The data
(closed forms below, checked symbolically by the tests with SymPy):

    fv = dv/dt - Lap_y v             = V - (1+t) [2 + cos(pi y2) - (pi^2/2) y1^2 cos(pi y2)]
    g  = dv/dn - kappa (u - v)  on y1 = 1
       = (1+t) [2 + cos(pi y2) - kappa (U - V(x, 1, y2))]
    fu = du/dt - Du Lap_x u + int_Gamma (kappa (u - v) + g) dsigma
       = U + (1+t) Du x2 sin(x1) + 2 (1+t)

This module evaluates problem data only (no finite element arithmetic); the
physical coordinates of a reference node under the bump map are part of the
problem definition.
"""
from __future__ import annotations

import numpy as np

from . import macro_coords, micro_coords


def U(x1, x2):
    return 1.0 + x2 * np.sin(x1)


def V(x1, x2, y1, y2):
    return x1 + x2 + y1 ** 2 * (1.0 + 0.5 * np.cos(np.pi * y2))


def u_exact(x1, x2, t):
    return (1.0 + t) * U(x1, x2)


def grad_u_exact(x1, x2, t):
    return (1.0 + t) * x2 * np.cos(x1), (1.0 + t) * np.sin(x1)


def v_exact(x1, x2, y1, y2, t):
    return (1.0 + t) * V(x1, x2, y1, y2)


def grad_v_exact(x1, x2, y1, y2, t):
    """gradient with respect to the physical micro coordinate y"""
    return ((1.0 + t) * 2.0 * y1 * (1.0 + 0.5 * np.cos(np.pi * y2)),
            (1.0 + t) * (-0.5 * np.pi) * y1 ** 2 * np.sin(np.pi * y2))


def fv(x1, x2, y1, y2, t):
    lap = 2.0 + np.cos(np.pi * y2) - 0.5 * np.pi ** 2 * y1 ** 2 * np.cos(np.pi * y2)
    return V(x1, x2, y1, y2) - (1.0 + t) * lap


def g_robin(x1, x2, y2, t, kappa=1.0):
    return (1.0 + t) * (2.0 + np.cos(np.pi * y2) - kappa * (U(x1, x2) - V(x1, x2, 1.0, y2)))


def fu(x1, x2, t, Du=1.0):
    return U(x1, x2) + (1.0 + t) * Du * x2 * np.sin(x1) + 2.0 * (1.0 + t)


def bump_map(a, yh1, yh2):
    """physical point of reference point yhat under chi = yhat + a (sin sin, 0)"""
    return yh1 + a * np.sin(np.pi * yh1) * np.sin(np.pi * yh2), yh2


def nodal_data(NM: int, Nm: int, a: np.ndarray, t: float, kappa: float = 1.0, Du: float = 1.0):
    """Nodal source arrays at time t for per-node bump amplitudes a [nM].

    Returns dict with fv [nM, nm], g [nM, Nm+1] (Robin edge nodes yhat = (1, q/Nm)),
    fu [nM], ud [nM] (= u_exact, used on Dirichlet nodes), u [nM], v [nM, nm].
    """
    x1, x2 = macro_coords(NM)
    yh1, yh2 = micro_coords(Nm)
    a = np.asarray(a).reshape(-1)
    y1, y2 = bump_map(a[:, None], yh1[None, :], yh2[None, :])
    X1, X2 = x1[:, None], x2[:, None]
    q = np.arange(Nm + 1) / Nm
    return {
        "fv": fv(X1, X2, y1, y2, t),
        "g": g_robin(X1, X2, q[None, :], t, kappa),
        "fu": fu(x1, x2, t, Du),
        "ud": u_exact(x1, x2, t),
        "u": u_exact(x1, x2, t),
        "v": v_exact(X1, X2, y1, y2, t),
    }
