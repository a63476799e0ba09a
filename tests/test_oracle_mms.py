"""Manufactured-solution convergence of the oracle (Sec. 4.2 methodology):
observed orders ~2 in L2 and ~1 in H1 on both scales, computed with the
paper's DoF-ratio formula.  CPU only."""
import numpy as np
import pytest

import oracle
from oracle import norms
import workloads as W
from workloads import mms


def test_mms_data_satisfy_the_pde():
    """The closed-form data of workloads.mms solve the parabolic u-v system
    (checked symbolically, independent of the finite element code)."""
    sp = pytest.importorskip("sympy")
    x1, x2, y1, y2, t, kap, Du = sp.symbols("x1 x2 y1 y2 t kappa Du")
    U = 1 + x2 * sp.sin(x1)
    V = x1 + x2 + y1 ** 2 * (1 + sp.cos(sp.pi * y2) / 2)
    u = (1 + t) * U
    v = (1 + t) * V
    fv = sp.diff(v, t) - sp.diff(v, y1, 2) - sp.diff(v, y2, 2)
    # homogeneous Neumann on y1 = 0, y2 = 0, y2 = 1
    assert sp.simplify(sp.diff(v, y1).subs(y1, 0)) == 0
    assert sp.simplify(sp.diff(v, y2).subs(y2, 0)) == 0
    assert sp.simplify(sp.diff(v, y2).subs(y2, 1)) == 0
    g = sp.diff(v, y1).subs(y1, 1) - kap * (u - v.subs(y1, 1))
    flux = sp.integrate((kap * (u - v) + g).subs(y1, 1), (y2, 0, 1))
    fu = sp.diff(u, t) - Du * (sp.diff(u, x1, 2) + sp.diff(u, x2, 2)) + flux
    f_fv = sp.lambdify((x1, x2, y1, y2, t), fv, "numpy")
    f_g = sp.lambdify((x1, x2, y2, t, kap), g, "numpy")
    f_fu = sp.lambdify((x1, x2, t, Du), fu, "numpy")
    pts = W.rng(0).uniform(0, 1, (5, 50))
    assert np.allclose(mms.fv(*pts[:4], pts[4]), f_fv(*pts[:4], pts[4]), atol=1e-13)
    assert np.allclose(mms.g_robin(pts[0], pts[1], pts[3], pts[4], 1.7), f_g(pts[0], pts[1], pts[3], pts[4], 1.7),
                       atol=1e-13)
    assert np.allclose(mms.fu(pts[0], pts[1], pts[4], 0.8), f_fu(pts[0], pts[1], pts[4], 0.8), atol=1e-13)


def _solve_mms(N, nsteps=2, dt=0.01):
    NM = Nm = N
    x1, _ = W.macro_coords(NM)
    a = 0.1 * x1
    P = oracle.Problem(Nm, NM, 1, W.FAMILY_BUMP, a.reshape(-1, 1))
    d0 = mms.nodal_data(NM, Nm, a, 0.0)
    P.set_state(d0["u"], d0["v"].ravel())
    for n in range(nsteps):
        d = mms.nodal_data(NM, Nm, a, (n + 1) * dt)
        P.set_sources(d["fv"].ravel(), d["g"].ravel(), d["fu"], d["ud"])
        P.step(dt, 1, cg_tol=1e-13, coupling_tol=1e-13)
    T = nsteps * dt
    _, _, mH = P.geometry()
    eu, eug = norms.macro_errors(NM, P.u, lambda a1, a2: mms.u_exact(a1, a2, T),
                                 lambda a1, a2: mms.grad_u_exact(a1, a2, T))
    ev, evg = norms.micro_errors(NM, Nm, W.FAMILY_BUMP, a, P.v, mH,
                                 lambda a1, a2, b1, b2: mms.v_exact(a1, a2, b1, b2, T),
                                 lambda a1, a2, b1, b2: mms.grad_v_exact(a1, a2, b1, b2, T))
    return (NM + 1) ** 2, np.array([eu, eug, ev, evg])


def test_mms_convergence_rates():
    levels = [4, 8, 16]
    res = [_solve_mms(N) for N in levels]
    N = np.array([r[0] for r in res], float)
    E = np.array([r[1] for r in res])
    # orders per halving of h; the DoF-ratio formula of Tables 1-2 gives the
    # same limit but is biased upwards on coarse meshes ((N+1)^2 vs N^2)
    rates = np.log(E[:-1] / E[1:]) / np.log(2.0)
    p_macro, q_macro, p_micro, q_micro = rates[-1]
    assert abs(p_macro - 2) < 0.05 and abs(p_micro - 2) < 0.05, rates
    assert abs(q_macro - 1) < 0.05 and abs(q_micro - 1) < 0.05, rates
    dof_rates = 2 * np.log(E[:-1] / E[1:]) / np.log(N[1:, None] / N[:-1, None])
    assert np.all(np.abs(dof_rates[-1] - np.array([2, 1, 2, 1])) < 0.2), dof_rates
    assert np.all(E[1:] < E[:-1])


def test_mms_interpolant_is_not_the_solution():
    """Guard: the discrete solution differs from the interpolant of the exact
    solution by O(h^2), i.e. the error norms above measure something."""
    _, E = _solve_mms(4, nsteps=1)
    assert E[0] > 1e-5 and E[2] > 1e-5
