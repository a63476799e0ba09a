"""Error norms on both scales (Sec. 4.2) -- TEST INFRASTRUCTURE ONLY.

e_u  = || u - u_H ||_{L2(Omega)},          e_u^grad = | u - u_H |_{H1(Omega)}
e_v  = ( sum_i m_i || v(x_i, .) - v_h,i ||^2_{L2(Y_x_i)} )^{1/2}
e_v^grad = ( sum_i m_i | v(x_i, .) - v_h,i |^2_{H1(Y_x_i)} )^{1/2}

The macro integral of the micro norms is taken with the nodal (lumped)
weights m_i, matching one micro problem per macro node (Sec. 3.3).  The micro
integrals are pulled back to Z with J and F^{-T} (Eq. (16)); all cell
integrals use 3x3 Gauss points.
"""
from __future__ import annotations

import numpy as np

from . import chi_many

_G3 = np.array([0.5 - 0.5 * np.sqrt(0.6), 0.5, 0.5 + 0.5 * np.sqrt(0.6)])
_W3 = np.array([5.0, 8.0, 5.0]) / 18.0


def _cell_points(N):
    """reference points of all cells: arrays [N*N*9] of (s, t, cell a, cell b, weight)"""
    a, b = np.meshgrid(np.arange(N), np.arange(N), indexing="xy")
    a, b = a.ravel(), b.ravel()
    S, T = np.meshgrid(_G3, _G3, indexing="xy")
    WS, WT = np.meshgrid(_W3, _W3, indexing="xy")
    s = np.tile(S.ravel(), a.size)
    t = np.tile(T.ravel(), a.size)
    w = np.tile((WS * WT).ravel(), a.size)
    A = np.repeat(a, 9)
    B = np.repeat(b, 9)
    return s, t, A, B, w


def _q1_eval(N, nodal, s, t, A, B):
    """value and reference-coordinate gradient of a Q1 field (nodal [..., (N+1)^2])"""
    n1 = N + 1
    i0 = A + n1 * B
    c0, c1, c2, c3 = nodal[..., i0], nodal[..., i0 + 1], nodal[..., i0 + n1], nodal[..., i0 + n1 + 1]
    val = c0 * (1 - s) * (1 - t) + c1 * s * (1 - t) + c2 * (1 - s) * t + c3 * s * t
    ds = (-(1 - t) * c0 + (1 - t) * c1 - t * c2 + t * c3) * N
    dt = (-(1 - s) * c0 - s * c1 + (1 - s) * c2 + s * c3) * N
    return val, ds, dt


def macro_errors(NM, uh, u_fn, grad_fn, x0=0.0, L=1.0):
    """errors of a Q1 field on the macro mesh of [x0, x0 + L]^2"""
    s, t, A, B, w = _cell_points(NM)
    H = L / NM
    x1, x2 = x0 + (A + s) * H, x0 + (B + t) * H
    val, d1, d2 = _q1_eval(NM, np.asarray(uh), s, t, A, B)
    d1, d2 = d1 / L, d2 / L
    g1, g2 = grad_fn(x1, x2)
    e2 = np.sum(w * H * H * (u_fn(x1, x2) - val) ** 2)
    h2 = np.sum(w * H * H * ((g1 - d1) ** 2 + (g2 - d2) ** 2))
    return float(np.sqrt(e2)), float(np.sqrt(h2))


def micro_errors(NM, Nm, family, params, vh, mH, v_fn, grad_fn, x0=0.0, L=1.0):
    """v_fn(x1, x2, y1, y2), grad_fn(...) -> (dv/dy1, dv/dy2) in physical coordinates;
    macro nodes on [x0, x0 + L]^2."""
    s, t, A, B, w = _cell_points(Nm)
    h = 1.0 / Nm
    yh1, yh2 = (A + s) * h, (B + t) * h
    n1 = NM + 1
    vh = np.asarray(vh).reshape((NM + 1) ** 2, -1)
    params = np.asarray(params).reshape((NM + 1) ** 2, -1)
    e2 = 0.0
    h2 = 0.0
    for i in range(vh.shape[0]):
        x1, x2 = x0 + (i % n1) * (L / NM), x0 + (i // n1) * (L / NM)
        y, F = chi_many(family, params[i], yh1, yh2)
        J = F[:, 0, 0] * F[:, 1, 1] - F[:, 0, 1] * F[:, 1, 0]
        val, ds, dt = _q1_eval(Nm, vh[i], s, t, A, B)
        # physical gradient of v_h: F^{-T} grad_hat
        g1 = (F[:, 1, 1] * ds - F[:, 1, 0] * dt) / J
        g2 = (-F[:, 0, 1] * ds + F[:, 0, 0] * dt) / J
        ex = v_fn(x1, x2, y[:, 0], y[:, 1])
        gx1, gx2 = grad_fn(x1, x2, y[:, 0], y[:, 1])
        e2 += mH[i] * np.sum(w * h * h * J * (ex - val) ** 2)
        h2 += mH[i] * np.sum(w * h * h * J * ((gx1 - g1) ** 2 + (gx2 - g2) ** 2))
    return float(np.sqrt(e2)), float(np.sqrt(h2))
