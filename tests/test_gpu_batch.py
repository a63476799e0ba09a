"""Batches of independent two-scale problems (one CUDA graph per batch step)
through the C ABI: against the oracle, against single contexts, recapture
after a change, errors, and sampled parity on the 32-instance uneven
workload."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

TIGHT = dict(cg_tol=1e-13, coupling_tol=1e-13, macro_tol=1e-14, cg_maxit=20000)
# (Nm, NM, family, kappa, D)
SPECS = [(3, 2, 1, 1.0, (1.0, 0.0, 1.0)), (4, 3, 2, 0.7, (1.0, 0.2, 0.5)), (6, 2, 4, 1.5, (0.8, 0.0, 1.2)),
         (5, 4, 1, 1.2, (1.0, 0.0, 1.0)), (4, 1, 3, 2.0, (1.0, -0.1, 1.0))]


def _T():
    import paper_2103_17040_gb300 as T
    T.load_library()
    return T


def _configure(p, k, spec):
    Nm, NM, fam, kappa, D = spec
    nM, nm = (NM + 1) ** 2, (Nm + 1) ** 2
    prm = W.random_params(fam, nM, seed=30 + k)
    u0, v0 = W.random_state(nM, nm, seed=40 + k)
    p.set_physics(D, kappa, 1.0)
    p.set_deformation(fam, prm)
    p.set_state(u0, v0)
    return prm, u0, v0


@pytest.mark.parametrize("coupling", [0, 1])
@pytest.mark.parametrize("precision", [0, 1])
def test_batch_matches_oracle(precision, coupling):
    T = _T()
    B = T.TwoScaleBatch([(s[0], s[1]) for s in SPECS], precision=precision, coupling=coupling, **TIGHT)
    inputs = [_configure(B[k], k, s) for k, s in enumerate(SPECS)]
    dt, n = 0.01, 3
    B.step(dt, n)
    B.synchronize()
    st = B.stats()
    assert st["steps"] == n and st["status"] == 0
    for k, (s, (prm, u0, v0)) in enumerate(zip(SPECS, inputs)):
        Nm, NM, fam, kappa, D = s
        R = oracle.Problem(Nm, NM, 0, fam, prm, D=D, kappa=kappa)
        R.set_state(u0, v0)
        R.step(dt, n, cg_tol=1e-14, coupling_tol=1e-14, macro_tol=1e-14)
        u, v = B[k].u(), B[k].v()
        assert np.linalg.norm(u - R.u) <= 1e-10 * np.linalg.norm(R.u), k
        assert np.linalg.norm(v.ravel() - R.v.ravel()) <= 1e-9 * np.linalg.norm(R.v), k
    B.close()


@pytest.mark.parametrize("use_graph", [1, 0])
def test_batch_equals_single_contexts_bitwise(use_graph):
    T = _T()
    opts = dict(TIGHT, tiling=1)
    B = T.TwoScaleBatch([(s[0], s[1]) for s in SPECS], precision=1, use_graph=use_graph, **opts)
    for k, s in enumerate(SPECS):
        _configure(B[k], k, s)
    B.step(0.01, 2)
    B.synchronize()
    for k, s in enumerate(SPECS):
        P = T.TwoScale(s[0], s[1], precision=1, **opts)
        _configure(P, k, s)
        P.step(0.01, 2)
        assert np.array_equal(P.u(), B[k].u()), k
        assert np.array_equal(P.v(), B[k].v()), k
        P.close()
    B.close()


def test_batch_recaptures_after_a_change():
    T = _T()
    opts = dict(TIGHT, tiling=1)
    specs = SPECS[:3]
    B = T.TwoScaleBatch([(s[0], s[1]) for s in specs], precision=0, **opts)
    for k, s in enumerate(specs):
        _configure(B[k], k, s)
    B.step(0.01, 1)
    # change instance 1's deformation and physics, then step again with another dt
    Nm, NM = specs[1][0], specs[1][1]
    prm2 = W.random_params(2, (NM + 1) ** 2, seed=99)
    B[1].set_deformation(2, prm2)
    B[1].set_physics((1.0, 0.0, 1.0), 0.3, 1.0)
    B.step(0.02, 2)
    B.synchronize()
    # reference: the same history on single contexts
    for k, s in enumerate(specs):
        P = T.TwoScale(s[0], s[1], precision=0, **opts)
        _configure(P, k, s)
        P.step(0.01, 1)
        if k == 1:
            P.set_deformation(2, prm2)
            P.set_physics((1.0, 0.0, 1.0), 0.3, 1.0)
        P.step(0.02, 2)
        assert np.array_equal(P.u(), B[k].u()), k
        assert np.array_equal(P.v(), B[k].v()), k
        P.close()
    B.close()


def test_batch_errors():
    T = _T()
    B = T.TwoScaleBatch([(3, 2), (4, 2)], precision=0)
    _configure(B[0], 0, SPECS[0])
    with pytest.raises(T.TsfError) as ei:
        B.step(0.01, 1)
    assert ei.value.status == T.TSF_E_STATE and "instance 1" in str(ei.value)
    with pytest.raises(T.TsfError) as ei:
        T.tsf_batch_instance(B.b, 2)
    assert ei.value.status == T.TSF_E_ARG
    with pytest.raises(T.TsfError):
        B.step(-1.0, 1)
    with pytest.raises(T.TsfError):
        T.tsf_batch_create(0)
    B.close()


@pytest.mark.parametrize("persistent", [False, True])
def test_uneven_32_instance_workload_every_instance(persistent):
    """The 32-instance uneven workload at full size (200M micro DoFs), mixed
    precision by pipelined elimination, one graph per batch step -- one
    branch per instance, or (persistent) work-queue launches, one per class
    of micro mesh, for all micro solves: every instance against the oracle after 3 steps (the extrapolated
    warm start runs), GPU at tolerance 1e-11, oracle at 1e-12; discrete mass
    balance on every instance."""
    T = _T()
    ws = W.c4()
    nsteps = 3
    B = T.TwoScaleBatch([(w.Nm, w.NM, w.bc) for w in ws], precision=1, cg_tol=1e-11, macro_tol=1e-13,
                        coupling=T.TSF_COUPLING_ELIMINATION, persistent=persistent)
    m0 = []
    for k, w in enumerate(ws):
        B[k].set_physics(w.D, w.kappa, w.Du)
        B[k].set_deformation(w.family, w.params)
        B[k].set_state(w.u0, None)
    for k, w in enumerate(ws):
        m0.append(_mass(B[k], w))
    B.step(ws[0].dt, nsteps)
    B.synchronize()
    st = B.stats()
    assert st["status"] == 0 and st["steps"] == nsteps
    for k, w in enumerate(ws):
        assert abs(_mass(B[k], w) - m0[k]) <= 1e-9 * abs(m0[k]), k
        if persistent:
            assert B[k].stats()["tiling"] == (4 if w.Nm <= 32 else 5)
        R = oracle.Problem(w.Nm, w.NM, w.bc, w.family, w.params, D=w.D, kappa=w.kappa, Du=w.Du)
        R.set_state(w.u0, None)
        R.step(w.dt, nsteps, cg_tol=1e-12, coupling_tol=1e-12, macro_tol=1e-13)
        u, v = B[k].u(), B[k].v()
        assert np.linalg.norm(u - R.u) <= 1e-8 * np.linalg.norm(R.u), k
        assert np.linalg.norm(v.ravel() - R.v.ravel()) <= 1e-8 * np.linalg.norm(R.v), k
    B.close()


def test_persistent_batch_equals_single_contexts_bitwise():
    """Persistent launches with work queues, one per class of micro mesh
    (strip height, threads a block, staging), solve the micro problems of all
    instances side by side, one block per micro problem at a time: strips of
    3 rows up to 32 micro cells per side (tiling 4), of 5 beyond (tiling 5).
    The results equal those of single contexts stepping with the same
    column-strip variant bit for bit."""
    T = _T()
    specs = SPECS + [(16, 6, 2, 0.9, (1.0, 0.0, 0.1)), (33, 2, 1, 1.1, (1.0, 0.0, 1.0)),
                     (48, 1, 1, 1.0, (1.0, 0.0, 1.0))]
    opts = dict(TIGHT, coupling=T.TSF_COUPLING_ELIMINATION)
    B = T.TwoScaleBatch([(s[0], s[1]) for s in specs], precision=1, persistent=True, **opts)
    for k, s in enumerate(specs):
        _configure(B[k], k, s)
    assert B.persistent_launches() == 0
    B.step(0.01, 4)
    B.synchronize()
    assert B.stats()["status"] == 0
    # classes (R, threads): (3, 32) for 3..6 cells, (3, 128) for 16, (5, 256)
    # for 33, (5, 512) for 48
    assert B.persistent_launches() == 4
    for k, s in enumerate(specs):
        t = B[k].stats()["tiling"]
        assert t == (4 if s[0] <= 32 else 5), k
        P = T.TwoScale(s[0], s[1], precision=1, tiling=t, **opts)
        _configure(P, k, s)
        P.step(0.01, 4)
        assert np.array_equal(P.u(), B[k].u()), k
        assert np.array_equal(P.v(), B[k].v()), k
        P.close()
    B.close()


def test_persistent_batch_many_classes():
    """Fourteen micro meshes of 2 to 47 cells per side, one macro cell each:
    a class (one persistent launch) per block size, all side by side; every
    instance bit for bit as a single context on the same variant."""
    T = _T()
    cells = [2, 5, 8, 11, 14, 17, 20, 23, 26, 29, 32, 35, 41, 47]
    specs = [(Nm, 1, 1, 1.0, (1.0, 0.0, 1.0)) for Nm in cells]
    opts = dict(TIGHT, coupling=T.TSF_COUPLING_ELIMINATION)
    B = T.TwoScaleBatch([(s[0], s[1]) for s in specs], precision=1, persistent=True, **opts)
    for k, s in enumerate(specs):
        _configure(B[k], k, s)
    B.step(0.01, 3)
    B.synchronize()
    assert B.stats()["status"] == 0
    assert B.persistent_launches() > 8
    for k, s in enumerate(specs):
        P = T.TwoScale(s[0], s[1], precision=1, tiling=B[k].stats()["tiling"], **opts)
        _configure(P, k, s)
        P.step(0.01, 3)
        assert np.array_equal(P.u(), B[k].u()), k
        assert np.array_equal(P.v(), B[k].v()), k
        P.close()
    B.close()


def test_persistent_batch_matches_oracle():
    T = _T()
    B = T.TwoScaleBatch([(s[0], s[1]) for s in SPECS], precision=1, coupling=T.TSF_COUPLING_ELIMINATION,
                        persistent=True, cg_tol=1e-11, macro_tol=1e-13)
    inputs = [_configure(B[k], k, s) for k, s in enumerate(SPECS)]
    dt, n = 0.01, 4
    B.step(dt, n)
    B.synchronize()
    for k, (s, (prm, u0, v0)) in enumerate(zip(SPECS, inputs)):
        Nm, NM, fam, kappa, D = s
        R = oracle.Problem(Nm, NM, 0, fam, prm, D=D, kappa=kappa)
        R.set_state(u0, v0)
        R.step(dt, n, cg_tol=1e-13, coupling_tol=1e-13, macro_tol=1e-13)
        assert np.linalg.norm(B[k].u() - R.u) <= 1e-8 * np.linalg.norm(R.u), k
        assert np.linalg.norm(B[k].v().ravel() - R.v.ravel()) <= 1e-8 * np.linalg.norm(R.v), k
    B.close()


def test_persistent_batch_rejects_the_partitioned_coupling():
    T = _T()
    B = T.TwoScaleBatch([(3, 2), (4, 2)], precision=1, coupling=T.TSF_COUPLING_PARTITIONED, persistent=True)
    for k in range(2):
        _configure(B[k], k, SPECS[k])
    with pytest.raises(T.TsfError) as ei:
        B.step(0.01, 1)
    assert ei.value.status == T.TSF_E_ARG
    B.close()


def _mass(P, w):
    """1^T M_H u + sum_i m_i vol_i vbar_i (total mass of both scales)."""
    x1, x2 = W.macro_coords(w.NM)
    m = 0.25 * np.where((x1 == 0) | (x1 == 1), 1.0, 2.0) * np.where((x2 == 0) | (x2 == 1), 1.0, 2.0) / w.NM ** 2
    _, vol = P.geometry()
    u = P.u()
    # consistent macro mass: 1^T M_H u = m^T u
    return float(np.dot(m, u) + np.dot(m, vol * P.vbar()))


def test_persistent_batch_limits():
    """The persistent batch takes at most 64 problems (their arguments sit in
    the kernel's parameter space) and micro meshes whose strips of 5 rows fit
    one block (at most 49 cells per side); beyond either a step reports
    TSF_E_ARG.  The branch mode steps the 65 problems."""
    T = _T()
    for specs in ([(2, 1)] * 65, [(50, 1)]):
        B = T.TwoScaleBatch(specs, precision=1, coupling=T.TSF_COUPLING_ELIMINATION, persistent=True)
        for k in range(len(specs)):
            B[k].set_deformation(W.FAMILY_BUMP, np.full((4, 1), 0.05))
            B[k].set_state(np.ones(4), None)
        with pytest.raises(T.TsfError) as ei:
            B.step(0.01, 1)
        assert ei.value.status == T.TSF_E_ARG
        if len(specs) == 65:
            T.tsf_batch_set_persistent(B.b, 0)
            B.step(0.01, 1)
            B.synchronize()
            assert all(np.all(np.isfinite(B[k].u())) for k in range(len(specs)))
        B.close()
