"""Pins of the oracle's implicit Euler two-scale step: the partitioned
coupling iteration against a dense monolithic direct solve, textbook special
cases, conservation, symmetry and decoupling.  CPU only."""
import numpy as np
import pytest

import oracle
from oracle.monolithic import monolithic_matrix, monolithic_step
import workloads as W


def _rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


CASES = [
    # family, Nm, NM, bc, D, kappa, Du, with_sources
    (1, 3, 2, 0, (1.0, 0.0, 1.0), 1.0, 1.0, False),
    (2, 4, 3, 0, (1.0, 0.0, 0.1), 1.7, 0.6, False),
    (4, 3, 3, 1, (0.8, 0.2, 1.1), 0.5, 1.0, True),
    (3, 2, 4, 0, (1.0, 0.0, 1.0), 2.0, 1.3, True),
    (0, 4, 2, 1, (1.0, 0.0, 1.0), 1.0, 1.0, True),
]


@pytest.mark.parametrize("case", CASES)
def test_partitioned_equals_monolithic(case):
    """Sec. 3.3 partitioned iteration converges to the solution of the whole
    coupled step solved directly (two independent routes to the fixed point)."""
    family, Nm, NM, bc, D, kappa, Du, src = case
    nM, nm = (NM + 1) ** 2, (Nm + 1) ** 2
    prm = W.random_params(family, nM, seed=10 + family)
    P = oracle.Problem(Nm, NM, bc, family, prm, D=D, kappa=kappa, Du=Du)
    u0, v0 = W.random_state(nM, nm, seed=3)
    P.set_state(u0, v0)
    g = W.rng(8)
    kw = {}
    if src:
        kw = dict(fv=g.standard_normal(nM * nm), g=g.standard_normal(nM * (Nm + 1)),
                  fu=g.standard_normal(nM), ud=g.standard_normal(nM))
        P.set_sources(**kw)
    dt = 0.02
    P.step(dt, 1, cg_tol=1e-14, coupling_tol=1e-14, macro_tol=1e-14)
    ud, vd = monolithic_step(P, u0, v0, dt, Du=Du, bc=bc, **kw)
    assert _rel(P.u, ud) < 1e-12
    assert _rel(P.v, vd) < 1e-12


def test_monolithic_symmetric_after_scaling_and_spd():
    """Scaling micro block-row i by the lumped macro mass m_i makes the step
    matrix symmetric; it is positive definite (coupling energy
    kappa sum_i m_i int_Gamma s (u_i - v_i)^2 >= 0)."""
    Nm, NM = 3, 2
    nM, nm = (NM + 1) ** 2, (Nm + 1) ** 2
    P = oracle.Problem(Nm, NM, 0, 2, W.random_params(2, nM, seed=1), D=(1.0, 0.1, 0.4), kappa=1.3)
    A = monolithic_matrix(P, 0.01)
    _, _, mH = P.geometry()
    s = np.concatenate([np.ones(nM), np.repeat(mH, nm)])
    As = s[:, None] * A
    assert np.max(np.abs(As - As.T)) < 1e-12 * np.max(np.abs(As))
    assert np.min(np.linalg.eigvalsh(0.5 * (As + As.T))) > 0


def _textbook_1d(N):
    n1 = N + 1
    h = 1.0 / N
    M1 = (h / 6) * (np.diag(np.full(n1, 4.0)) + np.diag(np.ones(n1 - 1), 1) + np.diag(np.ones(n1 - 1), -1))
    M1[0, 0] = M1[-1, -1] = 2 * h / 6
    K1 = (1 / h) * (np.diag(np.full(n1, 2.0)) - np.diag(np.ones(n1 - 1), 1) - np.diag(np.ones(n1 - 1), -1))
    K1[0, 0] = K1[-1, -1] = 1 / h
    return M1, K1


def test_identity_map_reduces_to_1d_problem():
    """Identity map, D = I, uniform u, Neumann macro, v0 depending on yhat_1
    only: every micro solution is the same, constant in yhat_2, and equal to
    the 1D Q1 solution of (M1/dt + K1 + kappa e e^T) v = M1 v^n/dt + kappa u e,
    coupled to the scalar u/dt + kappa (u - v(1)) = u^n/dt."""
    Nm, NM = 6, 3
    nM, n1 = (NM + 1) ** 2, Nm + 1
    kappa, dt, nsteps = 1.4, 0.03, 3
    P = oracle.Problem(Nm, NM, 0, 0, np.zeros((nM, 0)), kappa=kappa)
    v1 = np.cos(np.pi * np.arange(n1) / Nm) + 0.3
    P.set_state(np.full(nM, 0.8), np.tile(np.tile(v1, n1), nM))
    P.step(dt, nsteps, cg_tol=1e-14, coupling_tol=1e-14, macro_tol=1e-14)
    M1, K1 = _textbook_1d(Nm)
    e = np.zeros(n1)
    e[-1] = 1.0
    u = 0.8
    v = v1.copy()
    for _ in range(nsteps):
        # 1D monolithic system in (v, u)
        A = np.zeros((n1 + 1, n1 + 1))
        A[:n1, :n1] = M1 / dt + K1 + kappa * np.outer(e, e)
        A[:n1, n1] = -kappa * e
        A[n1, n1] = 1 / dt + kappa
        A[n1, n1 - 1] = -kappa
        rhs = np.concatenate([M1 @ v / dt, [u / dt]])
        x = np.linalg.solve(A, rhs)
        v, u = x[:n1], x[n1]
    V = P.v
    assert np.max(np.abs(P.u - u)) < 1e-12
    assert np.max(np.abs(V - V[0])) < 1e-14        # all instances identical
    assert np.max(np.abs(V.reshape(nM, n1, n1) - v[None, None, :])) < 1e-12


def test_mass_balance():
    """No sources, Neumann macro: 1^T M_H u + sum_i m_i 1^T M_i v_i is
    conserved (K_H 1 = 0, A_i 1 = 0 and the symmetric lumped coupling)."""
    Nm, NM = 5, 4
    nM, nm = (NM + 1) ** 2, (Nm + 1) ** 2
    P = oracle.Problem(Nm, NM, 0, 2, W.random_params(2, nM, seed=9), D=(1.0, 0.0, 0.1), kappa=1.5, Du=0.7)
    u0, v0 = W.random_state(nM, nm, seed=4)
    P.set_state(u0, v0)
    gam, vol, mH = P.geometry()

    def mass():
        return mH @ P.u + np.sum(mH * vol * P.vbar)

    m0 = mass()
    for _ in range(4):
        P.step(0.01, 1, cg_tol=1e-14, coupling_tol=1e-14, macro_tol=1e-14)
        assert abs(mass() - m0) < 1e-12 * abs(m0)
    # fluxes balance: what leaves the macro field enters the cells
    P.step(0.01, 1, cg_tol=1e-14, coupling_tol=1e-14, macro_tol=1e-14)


def test_decoupled_macro_mode_decay():
    """kappa = 0: u obeys the plain heat equation.  The nodal cosine mode
    cos(pi x_1) is an exact generalised eigenvector of the Q1 pencil
    (K_H, M_H) on a uniform Neumann mesh, so implicit Euler multiplies it by
    1 / (1 + dt lambda), lambda = (2/H)(1 - cos pi H) / ((H/6)(4 + 2 cos pi H))."""
    Nm, NM = 3, 8
    nM = (NM + 1) ** 2
    H = 1.0 / NM
    dt, nsteps, Du = 0.01, 5, 0.9
    P = oracle.Problem(Nm, NM, 0, 1, W.random_params(1, nM, seed=2), kappa=0.0, Du=Du)
    x1, _ = W.macro_coords(NM)
    u0 = np.cos(np.pi * x1)
    P.set_state(u0, None)
    P.step(dt, nsteps, cg_tol=1e-14, coupling_tol=1e-14, macro_tol=1e-14)
    lam = Du * (2 / H) * (1 - np.cos(np.pi * H)) / ((H / 6) * (4 + 2 * np.cos(np.pi * H)))
    assert np.max(np.abs(P.u - u0 / (1 + dt * lam) ** nsteps)) < 1e-12
    assert np.max(np.abs(P.v)) == 0.0       # cells never see u


def test_decoupled_micro_mode_decay():
    """kappa = 0, identity map, D = I: v0 = cos(pi yhat_1) decays by
    1 / (1 + dt lambda) per step with the 1D Q1 eigenvalue (textbook)."""
    Nm, NM = 8, 2
    nM = (NM + 1) ** 2
    h = 1.0 / Nm
    dt, nsteps = 0.004, 4
    P = oracle.Problem(Nm, NM, 0, 0, np.zeros((nM, 0)), kappa=0.0)
    yh1, _ = W.micro_coords(Nm)
    v0 = np.tile(np.cos(np.pi * yh1), nM)
    P.set_state(np.ones(nM), v0)
    P.step(dt, nsteps, cg_tol=1e-14, coupling_tol=1e-14, macro_tol=1e-14)
    lam = (2 / h) * (1 - np.cos(np.pi * h)) / ((h / 6) * (4 + 2 * np.cos(np.pi * h)))
    assert np.max(np.abs(P.v.ravel() - v0 / (1 + dt * lam) ** nsteps)) < 1e-12
    assert np.max(np.abs(P.u - 1.0)) < 1e-13


def test_multi_step_call_equals_repeated_steps():
    Nm, NM = 4, 3
    nM, nm = (NM + 1) ** 2, (Nm + 1) ** 2
    prm = W.random_params(1, nM, seed=5)
    u0, v0 = W.random_state(nM, nm, seed=6)
    A = oracle.Problem(Nm, NM, 0, 1, prm)
    B = oracle.Problem(Nm, NM, 0, 1, prm)
    A.set_state(u0, v0)
    B.set_state(u0, v0)
    A.step(0.01, 3, cg_tol=1e-13, coupling_tol=1e-13)
    for _ in range(3):
        B.step(0.01, 1, cg_tol=1e-13, coupling_tol=1e-13)
    assert np.array_equal(A.u, B.u) and np.array_equal(A.v, B.v)
    assert A.stats()["coupling_iters_total"] == B.stats()["coupling_iters_total"]
