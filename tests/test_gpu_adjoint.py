"""Discrete adjoint on the GPU (through the C ABI) against the oracle's
literal-transpose adjoint and against central finite differences."""
import numpy as np
import pytest

import workloads as W
from oracle.adjoint import TwoScaleAdjoint

pytestmark = pytest.mark.gpu

OPTS = dict(cg_tol=1e-14, coupling_tol=1e-14, macro_tol=1e-14, cg_maxit=20000)


def _T():
    import paper_2103_17040_gb300 as T
    T.load_library()
    return T


def _gpu(T, Nm, NM, family, prm, D, kappa, Du, precision=0, coupling=0):
    P = T.TwoScale(Nm, NM, precision=precision, coupling=coupling, **OPTS)
    P.set_physics(D, kappa, Du)
    P.set_deformation(family, prm)
    return P


@pytest.mark.parametrize("family,coupling", [(1, 0), (2, 0), (4, 0), (2, 1)])
def test_gradient_matches_oracle_adjoint(family, coupling):
    NM, Nm, dt, nsteps = 3, 4, 0.02, 4
    nM, nm = (NM + 1) ** 2, (Nm + 1) ** 2
    prm = W.random_params(family, nM, seed=60 + family)
    D, kappa, Du = (1.0, 0.1, 0.5), 1.3, 0.8
    u0, v0 = W.random_state(nM, nm, seed=7)
    Jo, go = TwoScaleAdjoint(Nm, NM, 0, family, prm, D=D, kappa=kappa, Du=Du).gradient(u0, v0, dt, nsteps)
    T = _T()
    P = _gpu(T, Nm, NM, family, prm, D, kappa, Du, coupling=coupling)
    P.set_state(u0, v0)
    J, g = P.adjoint_mean_u(dt, nsteps, ckpt_every=3)
    assert abs(J - Jo) < 1e-12 * abs(Jo)
    assert np.linalg.norm(g - go) < 1e-9 * np.linalg.norm(go), np.abs(g - go).max()


@pytest.mark.parametrize("family,coupling", [(W.FAMILY_SHEAR_BUMP, 0), (W.FAMILY_SHEAR_BUMP, 1), (W.FAMILY_BUMP, 0)])
def test_gradient_over_fifty_checkpointed_steps_matches_oracle(family, coupling):
    """The differentiation workload's march length and checkpointing (50
    implicit steps, checkpoints every 10, dt = 0.005) on an 8x8 macro / 8x8
    micro mesh: the GPU gradient against the oracle's literal-transpose
    adjoint (sparse direct solves, no iteration)."""
    NM, Nm, dt, nsteps = 8, 8, 0.005, 50
    nM, nm = (NM + 1) ** 2, (Nm + 1) ** 2
    prm = W.random_params(family, nM, seed=80 + family)
    D, kappa, Du = (1.0, 0.0, 0.1), 1.0, 1.0
    u0 = np.ones(nM)
    v0 = np.zeros(nM * nm)
    Jo, go = TwoScaleAdjoint(Nm, NM, 0, family, prm, D=D, kappa=kappa, Du=Du).gradient(u0, v0, dt, nsteps)
    T = _T()
    P = _gpu(T, Nm, NM, family, prm, D, kappa, Du, coupling=coupling)
    P.set_state(u0, v0)
    J, g = P.adjoint_mean_u(dt, nsteps, ckpt_every=10)
    assert abs(J - Jo) < 1e-12 * abs(Jo)
    assert np.linalg.norm(g - go) < 1e-9 * np.linalg.norm(go), np.abs(g - go).max()


def test_gradient_at_full_size_matches_richardson_finite_differences():
    """The differentiation workload at full size (64x64 macro / 32x32 micro,
    4225 parameters, 50 steps, checkpoints every 10) on the shear+bump family
    (D = diag(1, 0.1)), whose shear changes the physical cells: along 20
    seeded unit directions e, the adjoint's dJ/dp . e against the
    Richardson-extrapolated central difference (4 D(h/2) - D(h)) / 3 of the
    GPU forward march, h = 1e-2 (truncation O(h^4)), both in FP64 at
    tolerance 1e-14 with the eliminated coupling (no coupling tolerance).  Agreement to 1e-6 relative, plus the rounding floor of
    the differences (a few ulps of J over h)."""
    w = W.c5()
    T = _T()
    family = W.FAMILY_SHEAR_BUMP
    prm = W.random_params(family, w.nM, seed=5)
    D, kappa, Du = (1.0, 0.0, 0.1), w.kappa, w.Du
    P = _gpu(T, w.Nm, w.NM, family, prm, D, kappa, Du, coupling=1)
    P.set_state(w.u0, None)
    J, g = P.adjoint_mean_u(w.dt, 50, ckpt_every=10)
    P.close()

    def J_at(p):
        Q = _gpu(T, w.Nm, w.NM, family, p, D, kappa, Du, coupling=1)
        Q.set_state(w.u0, None)
        Q.step(w.dt, 50)
        u = Q.u()
        Q.close()
        x1, x2 = W.macro_coords(w.NM)
        cx = np.where((x1 == 0) | (x1 == 1), 1.0, 2.0)
        cy = np.where((x2 == 0) | (x2 == 1), 1.0, 2.0)
        return float(np.sum(0.25 * cx * cy / w.NM ** 2 * u))

    h = 1e-2
    floor = 8 * np.finfo(float).eps * abs(J) / h
    worst = 0.0
    for seed in range(20):
        e = W.rng(300 + seed).standard_normal(prm.shape)
        e /= np.linalg.norm(e)
        d1 = (J_at(prm + h * e) - J_at(prm - h * e)) / (2 * h)
        d2 = (J_at(prm + 0.5 * h * e) - J_at(prm - 0.5 * h * e)) / h
        fd = (4.0 * d2 - d1) / 3.0
        ad = float(np.sum(g * e))
        worst = max(worst, abs(ad - fd) / abs(ad))
        assert abs(ad - fd) <= 1e-6 * abs(ad) + floor, (seed, ad, fd)


def test_gradient_matches_gpu_finite_differences():
    """Central differences of J computed by the GPU forward march (FP64,
    tolerance 1e-14) along seeded unit directions, h = 1e-6."""
    NM, Nm, dt, nsteps = 4, 6, 0.01, 5
    nM, nm = (NM + 1) ** 2, (Nm + 1) ** 2
    family = W.FAMILY_SHEAR_BUMP
    prm = W.random_params(family, nM, seed=3)
    D, kappa, Du = (1.0, 0.0, 0.1), 1.0, 1.0
    u0, v0 = W.random_state(nM, nm, seed=8)
    T = _T()
    P = _gpu(T, Nm, NM, family, prm, D, kappa, Du)
    P.set_state(u0, v0)
    J, g = P.adjoint_mean_u(dt, nsteps, ckpt_every=2)

    def J_at(p):
        Q = _gpu(T, Nm, NM, family, p, D, kappa, Du)
        Q.set_state(u0, v0)
        Q.step(dt, nsteps)
        _, vol = Q.geometry()
        u = Q.u()
        x1, x2 = W.macro_coords(NM)
        cx = np.where((x1 == 0) | (x1 == 1), 1.0, 2.0)
        cy = np.where((x2 == 0) | (x2 == 1), 1.0, 2.0)
        return float(np.sum(0.25 * cx * cy / NM ** 2 * u))

    assert abs(J_at(prm) - J) < 1e-13
    h = 1e-6
    for seed in range(3):
        e = W.rng(200 + seed).standard_normal(prm.shape)
        e /= np.linalg.norm(e)
        fd = (J_at(prm + h * e) - J_at(prm - h * e)) / (2 * h)
        ad = float(np.sum(g * e))
        assert abs(ad - fd) <= 1e-6 * abs(ad) + 1e-10, (seed, ad, fd)


def test_checkpoint_interval_does_not_change_the_result():
    NM, Nm, dt, nsteps = 3, 5, 0.02, 7
    nM, nm = (NM + 1) ** 2, (Nm + 1) ** 2
    prm = W.random_params(1, nM, seed=9)
    u0, v0 = W.random_state(nM, nm, seed=10)
    T = _T()
    res = []
    for ck in (1, 3, 7, 10):
        P = _gpu(T, Nm, NM, 1, prm, (1.0, 0.0, 1.0), 1.0, 1.0)
        P.set_state(u0, v0)
        res.append(P.adjoint_mean_u(dt, nsteps, ckpt_every=ck) + (P.u(), P.v()))
    for J, g, u, v in res[1:]:
        assert J == res[0][0] and np.array_equal(g, res[0][1])
        assert np.array_equal(u, res[0][2]) and np.array_equal(v, res[0][3])
    # the state afterwards is the state after the march
    P = _gpu(T, Nm, NM, 1, prm, (1.0, 0.0, 1.0), 1.0, 1.0)
    P.set_state(u0, v0)
    P.step(dt, nsteps)
    assert np.array_equal(P.u(), res[0][2]) and np.array_equal(P.v(), res[0][3])


def test_autograd_function():
    import torch
    from paper_2103_17040_gb300.autograd import mean_macro_concentration
    NM, Nm, dt, nsteps = 3, 4, 0.02, 3
    nM, nm = (NM + 1) ** 2, (Nm + 1) ** 2
    prm = W.random_params(1, nM, seed=12)
    u0, v0 = W.random_state(nM, nm, seed=13)
    T = _T()
    P = _gpu(T, Nm, NM, 1, prm, (1.0, 0.0, 1.0), 1.0, 1.0)
    a = torch.tensor(prm, dtype=torch.float64, device="cuda", requires_grad=True)
    J = mean_macro_concentration(a, P, 1, u0, v0, dt, nsteps, 2)
    J.backward()
    Jo, go = TwoScaleAdjoint(Nm, NM, 0, 1, prm).gradient(u0, v0, dt, nsteps)
    assert abs(J.item() - Jo) < 1e-12
    assert np.linalg.norm(a.grad.cpu().numpy() - go) < 1e-9 * np.linalg.norm(go)


def test_adjoint_rejects_unsupported_problems():
    T = _T()
    P = T.TwoScale(3, 2, bc=T.TSF_BC_DIRICHLET, precision=0)
    P.set_deformation(1, np.full(9, 0.1))
    P.set_state(np.ones(9))
    with pytest.raises(T.TsfError) as ei:
        P.adjoint_mean_u(0.01, 2)
    assert ei.value.status == T.TSF_E_ARG
    Q = T.TwoScale(3, 2, precision=0)
    Q.set_deformation(1, np.full(9, 0.1))
    Q.set_state(np.ones(9))
    Q.set_sources(fu=np.ones(9))
    with pytest.raises(T.TsfError):
        Q.adjoint_mean_u(0.01, 2)
