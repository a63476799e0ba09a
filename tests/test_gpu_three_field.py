"""GPU parity of the stationary three-field system (include/tsfem3.h) with the
oracle's monolithic sparse solve (oracle/three_field.py).

Tolerances (relative L2 over all nodes / all micro DoFs): 1e-10 in FP64 and
1e-8 in mixed precision.  Cases: the manufactured problem of Eqs. (18)-(19)
with every source and datum; random affine-bump cells with random data on
all edges, an anisotropic D^v, distinct kappas and one to four Dirichlet edges; ragged
micro meshes (7, 13, 33 cells), the 1x1 degenerate micro mesh; every
micro-solve variant; the geometry experiment of Sec. 4.4 at its full size
(8x8 macro, 64x64 micro).  Also: the exact constant state of the Table 3
data, the Case A symmetry, the observed orders of the manufactured solution
up to 64x64 on both scales, re-use of the elimination vectors for new
sources, and error statuses.
"""
import numpy as np
import pytest

import workloads as W
from workloads import three_field as T3

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2103_17040_gb300 as lib
    lib.load_library()
    return lib


def _rel(a, b):
    a, b = np.asarray(a).ravel(), np.asarray(b).ravel()
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _oracle(wl):
    from oracle.three_field import ThreeField
    P = ThreeField(wl.Nm, wl.NM, wl.family, wl.params, D=wl.D, Dw=wl.Dw, kappa=wl.kappa, x0=wl.x0, L=wl.L,
                   dir_mask=wl.dir_mask)
    u, w, v = P.solve(**wl.sources())
    return P, u, w, v


def _gpu(T, wl, precision, tol=1e-13, **opts):
    P = T.ThreeField(wl.Nm, wl.NM, x0=wl.x0, L=wl.L, dir_mask=wl.dir_mask, precision=precision, cg_tol=tol,
                     macro_tol=1e-13, **opts)
    P.set_physics(wl.D, wl.Dw, wl.kappa)
    P.set_deformation(wl.family, wl.params)
    P.set_sources(**wl.sources())
    P.solve()
    return P


def _random_case(NM, Nm, seed, dir_mask=(1 << T3.EDGE_LEFT) | (1 << T3.EDGE_BOTTOM)):
    g = W.rng(seed)
    nM, nm, n1, N1 = (NM + 1) ** 2, (Nm + 1) ** 2, Nm + 1, NM + 1
    A = np.array([1.1, 0.15, -0.1, 0.9]) + g.uniform(-0.05, 0.05, (nM, 4))
    params = np.concatenate([A, g.uniform(0.0, 0.1, (nM, 1))], axis=1)      # affine + bump
    return T3.ThreeFieldWorkload(
        "random", NM, Nm, -0.5, 1.5, dir_mask, W.FAMILY_AFFINE_BUMP, params, D=(1.0, 0.2, 0.6), Dw=0.4,
        kappa=(0.7, 1.3, 0.45, 0.9), fu=g.normal(size=nM), fw=g.normal(size=nM), ud=g.normal(size=nM),
        gu=g.normal(size=(4, N1)), gw=g.normal(size=(4, N1)), fv=g.normal(size=(nM, nm)),
        gI=g.normal(size=(nM, n1)), gO=g.normal(size=(nM, n1)), gN=g.normal(size=(nM, 2, n1)))


CASES = {
    "manufactured_4_5": lambda: T3.manufactured(4, 5, Dv=1.2, Dw=0.6, kappa=(0.5, 1.0, 0.25, 1.5)),
    "random_5_13": lambda: _random_case(5, 13, 1),
    "random_3_33_top_dirichlet": lambda: _random_case(3, 33, 2, dir_mask=1 << T3.EDGE_TOP),
    "random_4_7_all_dirichlet": lambda: _random_case(4, 7, 3, dir_mask=15),
    "random_6_1_degenerate": lambda: _random_case(6, 1, 4),
    "case_b_sink_6_7": lambda: T3.case_b(6, 7, sink=True),
}


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
@pytest.mark.parametrize("case", list(CASES))
def test_parity_with_the_monolithic_oracle(T, case, precision):
    wl = CASES[case]()
    _, u0, w0, v0 = _oracle(wl)
    P = _gpu(T, wl, precision)
    u, w, v, vbar = P.fields()
    tol = 1e-10 if precision == 0 else 1e-8
    assert _rel(u, u0) < tol and _rel(w, w0) < tol and _rel(v, v0) < tol, (_rel(u, u0), _rel(w, w0), _rel(v, v0))
    s = P.stats()
    assert s["status"] == 0 and s["micro_solves"] == 3 * wl.nM and s["macro_iters"] > 0
    P.close()


def test_every_micro_solve_variant(T):
    """The ten iterative variants and the direct banded-Cholesky solve."""
    wl = _random_case(3, 20, 5)      # every variant of each precision fits a 21 x 21 micro grid
    _, u0, w0, v0 = _oracle(wl)
    ran = 0
    for precision in (0, 1):
        for tiling in range(T.TSF3_TILING_DIRECT + 1):
            try:
                P = _gpu(T, wl, precision, tiling=tiling)
            except T.TsfError as e:
                assert e.status == T.TSF_E_ARG   # strips and the direct solve are mixed only
                continue
            u, w, v, _ = P.fields()
            tol = 1e-10 if precision == 0 else 1e-8
            assert _rel(u, u0) < tol and _rel(w, w0) < tol and _rel(v, v0) < tol, (precision, tiling)
            assert P.stats()["tiling"] == tiling
            ran += 1
            P.close()
    assert ran == 15   # 4 FP64 + 10 mixed + the direct solve


@pytest.mark.parametrize("case", [T3.case_a, T3.case_b])
def test_table3_data_give_the_constant_state_at_full_size(T, case):
    wl = case()          # 8x8 macro cells, 64x64 micro cells
    P = _gpu(T, wl, 1, tol=1e-10)
    u, w, v, vbar = P.fields()
    k1, k2, k3, k4 = wl.kappa
    assert np.abs(u - 1).max() < 1e-9 and np.abs(v - k1 / k2).max() < 1e-9
    assert np.abs(w - k1 * k4 / (k2 * k3)).max() < 1e-8 and np.abs(vbar - k1 / k2).max() < 1e-9


def test_geometry_experiment_at_full_size_against_the_oracle(T):
    """Sec. 4.4 sizes (81 macro nodes, 4225 micro DoFs each) with the sink on
    the right edge: Case B against the oracle; Case A symmetric about x_1 = 0."""
    wl = T3.case_b(sink=True)
    _, u0, w0, v0 = _oracle(wl)
    P = _gpu(T, wl, 1, tol=1e-11)
    u, w, v, _ = P.fields()
    assert _rel(u, u0) < 1e-8 and _rel(w, w0) < 1e-8 and _rel(v, v0) < 1e-8
    wa = T3.case_a(sink=True)
    ua, ww, _, _ = _gpu(T, wa, 1, tol=1e-11).fields()
    n1 = wa.NM + 1
    assert np.abs(ua.reshape(n1, n1) - ua.reshape(n1, n1)[::-1]).max() < 1e-9
    assert np.abs(ww.reshape(n1, n1) - ww.reshape(n1, n1)[::-1]).max() < 1e-9
    assert np.abs(w.reshape(n1, n1) - w.reshape(n1, n1)[::-1]).max() > 1e-2


def _mms_errors(T, N, precision=1):
    from oracle import norms
    wl = T3.manufactured(N, N, Dv=1.0, Dw=0.5, kappa=(0.5, 1.0, 0.25, 1.0), tol=1e-11)
    P = _gpu(T, wl, precision, tol=1e-11)
    u, w, v, _ = P.fields()
    H = wl.L / N
    n1 = N + 1
    k = np.arange(n1 * n1)
    cx = np.where((k % n1 == 0) | (k % n1 == N), 1.0, 2.0)
    cy = np.where((k // n1 == 0) | (k // n1 == N), 1.0, 2.0)
    m = cx * cy * H * H / 4.0
    eu = norms.macro_errors(N, u, T3.u_mms, T3.grad_u_mms, x0=-1.0, L=2.0)
    ew = norms.macro_errors(N, w, T3.w_mms, T3.grad_w_mms, x0=-1.0, L=2.0)
    ev = norms.micro_errors(N, N, wl.family, wl.params, v, m, T3.v_mms, T3.grad_v_mms, x0=-1.0, L=2.0)
    return np.array([eu[0] + ew[0], eu[1] + ew[1], ev[0], ev[1]])


def test_manufactured_convergence_on_the_gpu(T):
    """Tables 1-2: orders 2 (L2) and 1 (H1) on both scales, up to 64 x 64
    macro cells with 64 x 64 micro cells (17.8 M micro DoFs)."""
    levels = [8, 16, 32, 64]
    E = np.array([_mms_errors(T, N) for N in levels])
    rates = np.log(E[:-1] / E[1:]) / np.log(2.0)
    assert np.all(np.abs(rates[:, 0] - 2) < 0.06) and np.all(np.abs(rates[:, 2] - 2) < 0.06), rates
    assert np.all(np.abs(rates[:, 1] - 1) < 0.06) and np.all(np.abs(rates[:, 3] - 1) < 0.06), rates


@pytest.mark.parametrize("Nm", [1, 2, 30, 64])
def test_direct_solve_is_the_default_in_mixed_precision(T, Nm):
    """Band widths 4 .. 67 (one, two and three band slots per lane)."""
    wl = _random_case(2, Nm, 10 + Nm)
    _, u0, w0, v0 = _oracle(wl)
    P = _gpu(T, wl, 1)
    u, w, v, _ = P.fields()
    assert P.stats()["tiling"] == T.TSF3_TILING_DIRECT
    assert _rel(u, u0) < 1e-8 and _rel(w, w0) < 1e-8 and _rel(v, v0) < 1e-8


def test_new_sources_reuse_the_elimination_vectors(T):
    wl = _random_case(4, 9, 6)
    P = _gpu(T, wl, 1)
    g = W.rng(7)
    wl2 = _random_case(4, 9, 6)
    wl2.fu, wl2.fv, wl2.gO = g.normal(size=wl.nM), g.normal(size=(wl.nM, wl.nm)), g.normal(size=(wl.nM, wl.Nm + 1))
    P.set_sources(**wl2.sources())
    P.solve()
    s = P.stats()
    assert s["micro_solves"] == 4 * wl.nM     # 3 for the first solve, 1 for the second
    _, u0, w0, v0 = _oracle(wl2)
    u, w, v, _ = P.fields()
    assert _rel(u, u0) < 1e-8 and _rel(w, w0) < 1e-8 and _rel(v, v0) < 1e-8


def test_error_statuses(T):
    wl = _random_case(2, 3, 8)
    P = T.ThreeField(3, 2, dir_mask=8)
    with pytest.raises(T.TsfError) as e:
        P.set_physics((1.0, 0.0, 1.0), 1.0, (1.0, 0.0, 1.0, 1.0))
    assert e.value.status == T.TSF_E_ARG
    with pytest.raises(T.TsfError) as e:
        P.set_physics((1.0, 2.0, 1.0), 1.0, (1.0, 1.0, 1.0, 1.0))   # D not positive definite
    assert e.value.status == T.TSF_E_ARG
    P.set_physics()
    bad = np.tile([1.0, 0.0, 0.0, -1.0, 0.0, 0.0], (wl.nM, 1))    # det F < 0
    P.set_deformation(W.FAMILY_AFFINE, bad)
    with pytest.raises(T.TsfError) as e:
        P.solve()
    assert e.value.status == T.TSF_E_BAD_JACOBIAN
    with pytest.raises(T.TsfError) as e:
        T.ThreeField(65, 2, dir_mask=1)
    assert e.value.status == T.TSF_E_ARG
    with pytest.raises(T.TsfError) as e:
        T.ThreeField(3, 2, dir_mask=0)       # no Dirichlet edge: singular
    assert e.value.status == T.TSF_E_ARG
    P.close()


def test_pushforward_centres_every_cell_on_its_node(T):
    """Sec. 3.6 push-forward of the three-field micro fields: X = x_i + scale
    (chi(x_i, yhat) - chi(x_i, (1/2, 1/2))), against the oracle's chi (FP32)."""
    from oracle import chi_many
    wl = T3.case_b(4, 6, sink=True)
    P = _gpu(T, wl, 1)
    _, _, v, _ = P.fields()
    scale = 0.1
    xyv = P.pushforward(scale)
    assert xyv.shape == (wl.nM, wl.nm, 3) and xyv.dtype == np.float32
    X0, X1 = T3.macro_nodes(wl.NM, wl.x0, wl.L)
    yh = np.arange(wl.Nm + 1) / wl.Nm
    Y1, Y2 = np.meshgrid(yh, yh, indexing="xy")
    for i in range(wl.nM):
        y, _ = chi_many(wl.family, wl.params[i], Y1.ravel(), Y2.ravel())
        c, _ = chi_many(wl.family, wl.params[i], [0.5], [0.5])
        X = np.stack([X0[i], X1[i]]) + scale * (y - c[0])
        assert np.abs(xyv[i, :, :2] - X).max() < 1e-5
        assert np.allclose(xyv[i, :, 2], v[i], rtol=1e-6, atol=1e-6)
