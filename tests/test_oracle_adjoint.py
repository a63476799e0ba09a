"""Pins of the oracle's discrete adjoint (gradient of the mean macro
concentration with respect to the per-node deformation parameters).  CPU only."""
import numpy as np
import pytest

import oracle
from oracle.adjoint import TwoScaleAdjoint
import workloads as W


@pytest.mark.parametrize("family", [1, 2, 3, 4])
def test_parameter_derivatives_of_the_operators(family):
    """Analytic dM/dp, dA/dp, dR/dp equal central differences of the
    assembly itself (pins the differentiated pull-back formulas)."""
    N = 4
    prm = W.random_params(family, 1, seed=family)[0]
    D = (1.0, 0.3, 0.6)
    h = 1e-6
    for k in range(oracle.NPARAM[family]):
        dM, dA, dR = oracle.assemble_q1_dparam(N, family, prm, k, D)
        e = np.zeros_like(prm)
        e[k] = h
        Mp, Ap, Rp = oracle.assemble_q1(N, family, prm + e, D)
        Mm, Am, Rm = oracle.assemble_q1(N, family, prm - e, D)
        for d, p, m in ((dM, Mp, Mm), (dA, Ap, Am), (dR, Rp, Rm)):
            fd = ((p - m) / (2 * h)).toarray()
            scale = max(1.0, np.max(np.abs(fd)))
            assert np.max(np.abs(d.toarray() - fd)) < 1e-7 * scale, (family, k)


def test_bump_keeps_volume_and_robin_edge():
    """For the bump map the cell boundary is fixed pointwise: d|Y|/da = 0 and
    the Robin matrix does not depend on a at all."""
    N = 6
    for a in (0.0, 0.1, 0.25):
        dM, dA, dR = oracle.assemble_q1_dparam(N, 1, [a], 0)
        one = np.ones(dM.shape[0])
        assert abs(one @ dM @ one) < 1e-14
        assert np.max(np.abs(dR.toarray())) < 1e-30   # sin(pi) rounds to 1.2e-16
        assert np.max(np.abs(dA @ one)) < 1e-12   # constants stay in the kernel


@pytest.mark.parametrize("family,bc", [(1, 0), (2, 0), (4, 0), (2, 1)])
def test_adjoint_gradient_matches_finite_differences(family, bc):
    NM, Nm = 2, 3
    nM, nm = (NM + 1) ** 2, (Nm + 1) ** 2
    prm = W.random_params(family, nM, seed=11 + family)
    kw = dict(D=(1.0, 0.0, 0.4), kappa=1.3, Du=0.7)
    u0, v0 = W.random_state(nM, nm, seed=2)
    dt, nsteps = 0.02, 3
    J, g = TwoScaleAdjoint(Nm, NM, bc, family, prm, **kw).gradient(u0, v0, dt, nsteps)
    for seed in range(3):
        e = W.rng(100 + seed).standard_normal(g.shape)
        e /= np.linalg.norm(e)
        h = 1e-5
        Jp = TwoScaleAdjoint(Nm, NM, bc, family, prm + h * e, **kw).forward(u0, v0, dt, nsteps)[1]
        Jm = TwoScaleAdjoint(Nm, NM, bc, family, prm - h * e, **kw).forward(u0, v0, dt, nsteps)[1]
        fd = (Jp - Jm) / (2 * h)
        assert abs(np.sum(g * e) - fd) <= 1e-6 * abs(fd) + 1e-11, (seed, np.sum(g * e), fd)


def test_sparse_monolithic_forward_equals_partitioned_oracle():
    """The adjoint's forward march (sparse direct) is the oracle's step."""
    NM, Nm = 3, 4
    nM, nm = (NM + 1) ** 2, (Nm + 1) ** 2
    prm = W.random_params(2, nM, seed=4)
    u0, v0 = W.random_state(nM, nm, seed=5)
    X, J = TwoScaleAdjoint(Nm, NM, 0, 2, prm, kappa=1.1).forward(u0, v0, 0.01, 2)
    P = oracle.Problem(Nm, NM, 0, 2, prm, kappa=1.1)
    P.set_state(u0, v0)
    P.step(0.01, 2, cg_tol=1e-14, coupling_tol=1e-14, macro_tol=1e-14)
    assert np.linalg.norm(X[-1][:nM] - P.u) / np.linalg.norm(P.u) < 1e-12
    assert np.linalg.norm(X[-1][nM:] - P.v.ravel()) / np.linalg.norm(P.v) < 1e-12
    _, _, mH = P.geometry()
    assert abs(J - mH @ P.u) < 1e-12
