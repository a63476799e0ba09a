"""Pins of the three-field oracle (Eq. (5), discrete form Eq. (17)).  CPU only.

* the manufactured data of Eqs. (18)-(19) re-derived with SymPy;
* the four edge mass matrices: against the two-field assembly (right edge)
  and against the closed form for affine cells (all edges);
* the system reduces to the (pinned) two-field implicit Euler step through
  either coupling edge, when the other pair of kappas is zero;
* the stationary matrix becomes symmetric after scaling the rows by
  (kappa_1/kappa_2, m_i, kappa_3/kappa_4), and is positive definite;
* the exact constant solution of the Table 3 data;
* Sec. 4.4: with a sink, identity cells (Case A) give a solution symmetric
  about x_1 = 0 and the cells of Case B break that symmetry;
* observed orders 2 (L2) and 1 (H1) on both scales for the manufactured
  solution, the rates of Tables 1-2.
"""
import numpy as np
import pytest

import oracle
from oracle import norms
from oracle.three_field import (EDGE_BOTTOM, EDGE_LEFT, EDGE_RIGHT, EDGE_TOP, ThreeField, edge_mass, edge_nodes)
import workloads as W
from workloads import three_field as T3


def _oracle(wl, **kw):
    return ThreeField(wl.Nm, wl.NM, wl.family, wl.params, D=wl.D, Dw=wl.Dw, kappa=wl.kappa, x0=wl.x0, L=wl.L,
                      dir_mask=wl.dir_mask, **kw)


def test_manufactured_data_satisfy_the_pde():
    sp = pytest.importorskip("sympy")
    x0, x1, z0, z1, s = sp.symbols("x0 x1 z0 z1 s", real=True)
    Dv, Dw = sp.Rational(13, 10), sp.Rational(7, 10)
    k1, k2, k3, k4 = sp.Rational(1, 2), sp.Rational(3, 2), sp.Rational(1, 4), sp.Rational(6, 5)
    R = sp.Rational
    zeta = sp.Matrix([R(2, 5) * ((x0 + R(13, 10)) + (R(7, 5) * z0 - R(27, 50) * z1)),
                      R(3, 10) * ((x1 + R(6, 5)) + (-R(2, 5) * z0 + R(4, 5) * z1))])
    Y0, Y1 = sp.symbols("Y0 Y1", real=True)
    u = x1 * sp.sin(x0)
    w = x0 * sp.cos(x1)
    v = x0 + x1 + Y0 * Y1 * (1 - Y1)
    grad_v = sp.Matrix([sp.diff(v, Y0), sp.diff(v, Y1)])
    lap_v = sp.diff(v, Y0, 2) + sp.diff(v, Y1, 2)
    sub = {Y0: zeta[0], Y1: zeta[1]}
    Fe1, Fe2 = sp.diff(zeta, z0), sp.diff(zeta, z1)

    def outward(tangent, inward_dir):
        n = sp.Matrix([tangent[1], -tangent[0]]) / sp.sqrt(tangent.dot(tangent))
        return n if n.dot(inward_dir) < 0 else -n

    nI, nO = outward(Fe2, Fe1), outward(Fe2, -Fe1)          # z0 = -1 and z0 = +1
    nB, nT = outward(Fe1, Fe2), outward(Fe1, -Fe2)          # z1 = -1 and z1 = +1
    flux = lambda n: (Dv * grad_v.dot(n)).subs(sub)
    gI = (flux(nI) - k1 * u + k2 * v.subs(sub)).subs(z0, -1)
    gO = (flux(nO) - k3 * w + k4 * v.subs(sub)).subs(z0, 1)
    gB, gT = flux(nB).subs(z1, -1), flux(nT).subs(z1, 1)
    fv = (-Dv * lap_v).subs(sub)
    edge_len = sp.sqrt(Fe2.dot(Fe2))
    fu = -(sp.diff(u, x0, 2) + sp.diff(u, x1, 2)) + sp.integrate(
        (flux(nI).subs(z0, -1) * edge_len).subs(z1, s), (s, -1, 1))
    fw = -Dw * (sp.diff(w, x0, 2) + sp.diff(w, x1, 2)) + sp.integrate(
        (flux(nO).subs(z0, 1) * edge_len).subs(z1, s), (s, -1, 1))
    NM, Nm = 3, 4
    wl = T3.manufactured(NM, Nm, Dv=float(Dv), Dw=float(Dw), kappa=(0.5, 1.5, 0.25, 1.2))
    X0, X1 = T3.macro_nodes(NM, -1.0, 2.0)
    zs = 2.0 * np.arange(Nm + 1) / Nm - 1.0
    L = lambda e, *a: sp.lambdify(a, e, "numpy")
    assert np.allclose(wl.fu, L(fu, x0, x1)(X0, X1), atol=1e-13)
    assert np.allclose(wl.fw, L(fw, x0, x1)(X0, X1), atol=1e-13)
    Zq = np.broadcast_to(zs, (X0.size, Nm + 1))
    xx0, xx1 = X0[:, None] + 0 * Zq, X1[:, None] + 0 * Zq
    assert np.allclose(wl.gI, L(gI, x0, x1, z1)(xx0, xx1, Zq), atol=1e-13)
    assert np.allclose(wl.gO, L(gO, x0, x1, z1)(xx0, xx1, Zq), atol=1e-13)
    assert np.allclose(wl.gN[:, 0], L(gB, x0, x1, z0)(xx0, xx1, Zq), atol=1e-13)
    assert np.allclose(wl.gN[:, 1], L(gT, x0, x1, z0)(xx0, xx1, Zq), atol=1e-13)
    Z0g, Z1g = np.meshgrid(zs, zs, indexing="xy")
    fv_num = L(fv, x0, x1, z0, z1)(X0[:, None], X1[:, None], Z0g.ravel()[None, :], Z1g.ravel()[None, :])
    assert np.allclose(wl.fv, np.broadcast_to(fv_num, wl.fv.shape), atol=1e-13)
    # macro Neumann data: Dw grad w . n on each edge; Dirichlet values of u
    for e, (ex0, ex1) in enumerate(T3.macro_edge_nodes(NM, -1.0, 2.0)):
        n = T3.EDGE_NORMALS[e]
        gw = L(Dw * (sp.diff(w, x0) * n[0] + sp.diff(w, x1) * n[1]), x0, x1)(ex0, ex1)
        assert np.allclose(wl.gw[e], gw, atol=1e-13)
    assert np.allclose(wl.ud, X1 * np.sin(X0))


@pytest.mark.parametrize("family,prm", [(W.FAMILY_BUMP, [0.15]), (W.FAMILY_SHEAR_BUMP, [0.1, 0.12]),
                                        (W.FAMILY_AFFINE_BUMP, [1.1, 0.2, -0.1, 0.9, 0.07])])
def test_right_edge_mass_matches_the_two_field_assembly(family, prm):
    N = 6
    _, _, R = oracle.assemble_q1(N, family, prm)
    assert abs(edge_mass(N, family, prm, EDGE_RIGHT) - R).max() < 1e-15


def test_edge_mass_of_affine_cells_is_the_scaled_1d_mass_matrix():
    A = np.array([[1.3, -0.4], [0.25, 0.8]])
    prm = [A[0, 0], A[0, 1], A[1, 0], A[1, 1], 0.3, -0.2]
    N = 5
    h = 1.0 / N
    M1 = np.zeros((N + 1, N + 1))
    for s in range(N):
        M1[s:s + 2, s:s + 2] += h / 6.0 * np.array([[2.0, 1.0], [1.0, 2.0]])
    # the image of a vertical edge has length |A e2|, of a horizontal one |A e1|
    for e, length in ((EDGE_LEFT, np.linalg.norm(A[:, 1])), (EDGE_RIGHT, np.linalg.norm(A[:, 1])),
                      (EDGE_BOTTOM, np.linalg.norm(A[:, 0])), (EDGE_TOP, np.linalg.norm(A[:, 0]))):
        R = edge_mass(N, W.FAMILY_AFFINE, prm, e).toarray()
        nodes = edge_nodes(N, e)
        assert np.allclose(R[np.ix_(nodes, nodes)], length * M1, atol=1e-15)
        off = np.setdiff1d(np.arange((N + 1) ** 2), nodes)
        assert not R[off].any() and not R[:, off].any()


def _two_field_step(Nm, NM, bc, a, kap, dt, u0, v0, ud=None):
    P = oracle.Problem(Nm, NM, bc, W.FAMILY_BUMP, a, kappa=kap, Du=1.0)
    P.set_state(u0, v0)
    if ud is not None:
        P.set_sources(ud=ud)
    P.step(dt, 1, cg_tol=1e-14, coupling_tol=1e-14)
    return P.u, P.v.reshape(P.nM, P.nm)


def test_reduces_to_the_two_field_step_through_the_outflow_edge():
    """kappa_1 = kappa_2 = 0: w and v are the two-field (u, v) step on the same
    cells (the two-field Robin edge is yhat_1 = 1 = Gamma_O), u stays put."""
    g = W.rng(3)
    NM, Nm, dt, kap = 4, 5, 0.05, 1.3
    nM, nm = (NM + 1) ** 2, (Nm + 1) ** 2
    a = g.uniform(0, 0.2, (nM, 1))
    u0, v0 = g.uniform(0.5, 1.5, nM), g.uniform(0, 1, (nM, nm))
    u2, v2 = _two_field_step(Nm, NM, 0, a, kap, dt, u0, v0)
    P = ThreeField(Nm, NM, W.FAMILY_BUMP, a, Dw=1.0, kappa=(0.0, 0.0, kap, kap))
    u, w, v = P.solve(dt=dt, prev=(np.full(nM, 0.7), v0, u0))
    assert np.abs(w - u2).max() < 1e-12 and np.abs(v - v2).max() < 1e-12
    assert np.abs(u - 0.7).max() < 1e-13


@pytest.mark.parametrize("bc", [0, 1])
def test_reduces_to_the_two_field_step_through_the_inflow_edge(bc):
    """kappa_3 = kappa_4 = 0 with the cells mirrored (yhat_1 -> 1 - yhat_1 and
    y_1 -> 1 - y_1, which maps the bump a to -a): u and the mirrored v are
    the two-field step."""
    g = W.rng(4)
    NM, Nm, dt, kap = 4, 5, 0.05, 0.8
    nM, nm = (NM + 1) ** 2, (Nm + 1) ** 2
    a = g.uniform(0, 0.2, (nM, 1))
    u0, v0 = g.uniform(0.5, 1.5, nM), g.uniform(0, 1, (nM, nm))
    ud = g.uniform(0.5, 1.5, nM) if bc else None
    u2, v2 = _two_field_step(Nm, NM, bc, a, kap, dt, u0, v0, ud)
    mirror = np.arange(nm).reshape(Nm + 1, Nm + 1)[:, ::-1].ravel()
    P = ThreeField(Nm, NM, W.FAMILY_BUMP, -a, Dw=1.0, kappa=(kap, kap, 0.0, 0.0), dir_mask=15 if bc else 0)
    u, w, v = P.solve(dt=dt, prev=(u0, v0[:, mirror], np.full(nM, 0.3)), ud=ud)
    assert np.abs(u - u2).max() < 1e-12 and np.abs(v[:, mirror] - v2).max() < 1e-12
    assert np.abs(w - 0.3).max() < 1e-13


def test_stationary_matrix_is_symmetric_after_scaling_and_positive_definite():
    prm = np.tile([1.1, 0.2, -0.1, 0.9, 0.0, 0.0], (9, 1)) + W.rng(5).uniform(-0.05, 0.05, (9, 6))
    P = ThreeField(3, 2, W.FAMILY_AFFINE, prm, D=(1.0, 0.2, 0.7), Dw=0.3, kappa=(0.5, 1.0, 0.25, 2.0),
                   dir_mask=1 << 3)
    A = P.matrix().toarray()
    free = np.concatenate([~P.dir, np.ones(P.nM * P.nm + P.nM, bool)])
    B = (P.symmetric_scaling()[:, None] * A)[np.ix_(free, free)]
    assert np.abs(B - B.T).max() < 1e-15 * np.abs(B).max() * 10
    assert np.linalg.eigvalsh(0.5 * (B + B.T)).min() > 0.0
    # the unscaled matrix is not symmetric (the kappas differ)
    Af = A[np.ix_(free, free)]
    assert np.abs(Af - Af.T).max() > 1e-3


@pytest.mark.parametrize("case", [T3.case_a, T3.case_b])
def test_table3_data_give_the_constant_state(case):
    wl = case(6, 6)
    P = _oracle(wl)
    u, w, v = P.solve(**wl.sources())
    k1, k2, k3, k4 = wl.kappa
    assert np.abs(u - 1.0).max() < 1e-12
    assert np.abs(v - k1 / k2).max() < 1e-12
    assert np.abs(w - k1 * k4 / (k2 * k3)).max() < 1e-12


def test_case_a_is_symmetric_and_case_b_is_not():
    NM = 6
    sol = {}
    for case in (T3.case_a, T3.case_b):
        wl = case(NM, 6, sink=True)
        u, w, _ = _oracle(wl).solve(**wl.sources())
        sol[case] = (u.reshape(NM + 1, NM + 1), w.reshape(NM + 1, NM + 1))
    uA, wA = sol[T3.case_a]
    uB, wB = sol[T3.case_b]
    assert np.abs(uA - uA[::-1]).max() < 1e-12 and np.abs(wA - wA[::-1]).max() < 1e-12
    assert np.abs(wB - wB[::-1]).max() > 1e-2
    assert np.ptp(uA) > 0.9   # the sink makes the profile non-trivial


def _mms_errors(N):
    wl = T3.manufactured(N, N, Dv=1.0, Dw=0.5, kappa=(0.5, 1.0, 0.25, 1.0))
    P = _oracle(wl)
    u, w, v = P.solve(**wl.sources())
    eu = norms.macro_errors(N, u, T3.u_mms, T3.grad_u_mms, x0=-1.0, L=2.0)
    ew = norms.macro_errors(N, w, T3.w_mms, T3.grad_w_mms, x0=-1.0, L=2.0)
    ev = norms.micro_errors(N, N, wl.family, wl.params, v, P.m, T3.v_mms, T3.grad_v_mms, x0=-1.0, L=2.0)
    return np.array([eu[0] + ew[0], eu[1] + ew[1], ev[0], ev[1]])


def test_manufactured_convergence_rates():
    E = np.array([_mms_errors(N) for N in (4, 8, 16)])
    rates = np.log(E[:-1] / E[1:]) / np.log(2.0)
    p_macro, q_macro, p_micro, q_micro = rates[-1]
    assert abs(p_macro - 2) < 0.06 and abs(p_micro - 2) < 0.06, rates
    assert abs(q_macro - 1) < 0.06 and abs(q_micro - 1) < 0.06, rates
    assert np.all(E[1:] < E[:-1])


def test_stationary_system_without_dirichlet_edge_is_rejected():
    """Sec. 2.2 asks for a Dirichlet part: without one the constant equilibrium
    (u, kappa_1/kappa_2 u, kappa_1 kappa_4/(kappa_2 kappa_3) u) is a null vector."""
    wl = T3.case_a(3, 3)
    P = ThreeField(wl.Nm, wl.NM, wl.family, wl.params, kappa=wl.kappa, dir_mask=0)
    k1, k2, k3, k4 = wl.kappa
    null = np.concatenate([np.ones(P.nM), np.full(P.nM * P.nm, k1 / k2), np.full(P.nM, k1 * k4 / (k2 * k3))])
    assert np.abs(P.matrix() @ null).max() < 1e-13
    with pytest.raises(ValueError):
        P.solve()
