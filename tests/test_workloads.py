"""The seeded input generators against the recipe they implement: sizes,
parameter ranges, physics, step counts, determinism per seed, and det F > 0
of every generated deformation on a fine grid of the reference cell (the
well-posedness condition of Sec. 2, checked with the oracle's map).  CPU only."""
import numpy as np

import oracle
import workloads as W


def _det_min(family, params, n=17):
    g = np.linspace(0.0, 1.0, n)
    y1, y2 = np.meshgrid(g, g)
    worst = np.inf
    for prm in params:
        _, F = oracle.chi_many(family, prm, y1.ravel(), y2.ravel())
        worst = min(worst, float(np.min(F[:, 0, 0] * F[:, 1, 1] - F[:, 0, 1] * F[:, 1, 0])))
    return worst


def test_manufactured_two_field_workload():
    w = W.c1()
    x1, _ = W.macro_coords(8)
    assert (w.NM, w.Nm, w.bc, w.family) == (8, 8, 1, W.FAMILY_BUMP)
    assert np.array_equal(w.params[:, 0], 0.1 * x1)
    assert (w.dt, w.nsteps) == (0.01, 10)


def test_64x64_32x32_workload():
    w = W.c2()
    assert (w.NM, w.Nm, w.bc, w.family) == (64, 32, 0, W.FAMILY_BUMP)
    assert w.params.shape == (65 * 65, 1)
    a = w.params[:, 0]
    assert a.min() >= 0.0 and a.max() < 0.2 and 0.09 < a.mean() < 0.11
    assert w.D == (1.0, 0.0, 1.0) and w.kappa == 1.0
    assert np.array_equal(w.u0, np.ones(65 * 65)) and w.v0 is None
    assert (w.dt, w.nsteps, w.tol, w.coupling_tol) == (0.005, 50, 1e-8, 1e-10)
    assert np.array_equal(W.c2().params[:, 0], a) and not np.array_equal(W.c2(seed=1).params[:, 0], a)
    assert np.array_equal(W.c5().params[:, 0], a)  # the differentiation workload uses the same maps
    assert _det_min(w.family, w.params[::97]) > 0.0


def test_128x128_64x64_workload():
    w = W.c3()
    assert (w.NM, w.Nm, w.family) == (128, 64, W.FAMILY_SHEAR_BUMP)
    s, b = w.params[:, 0], w.params[:, 1]
    assert s.min() >= -0.15 and s.max() <= 0.15 and b.min() >= 0.0 and b.max() <= 0.15
    assert w.D == (1.0, 0.0, 0.1) and w.nsteps == 20
    assert _det_min(w.family, w.params[::331]) > 0.0


def test_batch_of_uneven_problems():
    ws = W.c4()
    assert len(ws) == 32
    assert {w.NM for w in ws} <= {16, 32, 64, 96} and {w.Nm for w in ws} <= {16, 32, 48}
    assert len({(w.NM, w.Nm) for w in ws}) > 4
    for w in ws:
        assert 0.5 <= w.kappa <= 2.0 and (w.dt, w.nsteps) == (0.005, 10)
        x1, x2 = W.macro_coords(w.NM)
        inner = x1 * x2 > 0
        A = w.params[inner, 0] / (x1 * x2)[inner]
        assert np.allclose(A, A[0]) and 0.0 <= A[0] <= 0.2
    dofs = sum((w.NM + 1) ** 2 * (w.Nm + 1) ** 2 for w in ws)
    assert 1.5e8 < dofs < 2.5e8


def test_random_parameters_keep_det_F_positive():
    for fam in (W.FAMILY_BUMP, W.FAMILY_SHEAR_BUMP, W.FAMILY_AFFINE, W.FAMILY_AFFINE_BUMP):
        prm = W.random_params(fam, 64, seed=3)
        assert prm.shape == (64, W.NPARAM[fam])
        assert _det_min(fam, prm) > 0.0, fam
