"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances (relative L2 over all nodes, u and v separately): 1e-10 for the
FP64 path, 1e-8 for FP32 inner solves with FP64 refinement, both sides
solving to a relative residual far below that.
"""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
MIXED_TOL = 1e-8


def _T():
    import paper_2103_17040_gb300 as T
    T.load_library()
    return T


def oracle_rho(R):
    """r_i^T v_i from the oracle's Robin vectors and micro fields (FP64)."""
    return np.einsum("ij,ij->i", R.r, R.v)


def rel(a, b):
    a = np.ravel(np.asarray(a))
    b = np.ravel(np.asarray(b))
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _pair(Nm, NM, family, prm, bc=0, D=(1.0, 0.0, 1.0), kappa=1.0, Du=1.0, precision=0, **opts):
    T = _T()
    o = dict(cg_tol=1e-13 if precision == 0 else 1e-11, coupling_tol=1e-13, macro_tol=1e-13)
    o.update(opts)
    P = T.TwoScale(Nm, NM, bc=bc, precision=precision, **o)
    P.set_physics(D, kappa, Du)
    P.set_deformation(family, prm)
    R = oracle.Problem(Nm, NM, bc, family, prm, D=D, kappa=kappa, Du=Du)
    return P, R


GEOM_CASES = [(W.FAMILY_IDENTITY, 4), (W.FAMILY_BUMP, 6), (W.FAMILY_SHEAR_BUMP, 5), (W.FAMILY_AFFINE, 3),
              (W.FAMILY_AFFINE_BUMP, 7)]


@pytest.mark.parametrize("family,Nm", GEOM_CASES)
def test_geometry_matches_oracle(family, Nm):
    NM = 3
    nM = (NM + 1) ** 2
    prm = W.random_params(family, nM, seed=family)
    P, R = _pair(Nm, NM, family, prm, D=(0.9, 0.1, 0.6), kappa=1.3)
    gam, vol = P.geometry()
    gr, vr, _ = R.geometry()
    assert np.max(np.abs(gam - gr)) < 1e-13
    assert np.max(np.abs(vol - vr)) < 1e-13


@pytest.mark.parametrize("precision", [0, 1])
def test_geometry_paths_mixed_in_one_launch(precision):
    """The geometry kernel takes the reference-table path where a node's map
    has zero bump amplitude (F constant) and the quadrature path elsewhere,
    node by node in one launch.  Half of the nodes take each path here; the
    operators are checked through a whole step against the oracle (any wrong
    coupling shows in u, v and rho) and the geometry sums directly."""
    NM, Nm = 5, 9
    nM, nm = (NM + 1) ** 2, (Nm + 1) ** 2
    prm = W.random_params(W.FAMILY_AFFINE_BUMP, nM, seed=41)
    prm[::2, 4] = 0.0
    P, R = _pair(Nm, NM, W.FAMILY_AFFINE_BUMP, prm, D=(0.9, 0.1, 0.6), kappa=1.3, precision=precision)
    gam, vol = P.geometry()
    gr, vr, _ = R.geometry()
    assert np.max(np.abs(gam - gr)) < 1e-13 and np.max(np.abs(vol - vr)) < 1e-13
    u0, v0 = W.random_state(nM, nm, seed=6)
    P.set_state(u0, v0)
    R.set_state(u0, v0)
    P.step(0.01, 2)
    P.synchronize()
    R.step(0.01, 2, cg_tol=1e-13, coupling_tol=1e-13, macro_tol=1e-13)
    tol = FP64_TOL if precision == 0 else MIXED_TOL
    assert rel(P.u(), R.u) < tol and rel(P.v(), R.v) < tol
    assert rel(P.rho(), oracle_rho(R)) < tol


STEP_CASES = [
    # family, Nm, NM, bc, D, kappa, Du, nsteps
    (W.FAMILY_BUMP, 8, 4, 0, (1.0, 0.0, 1.0), 1.0, 1.0, 2),
    (W.FAMILY_SHEAR_BUMP, 7, 5, 0, (1.0, 0.0, 0.1), 1.5, 0.7, 2),     # ragged micro mesh, odd sizes
    (W.FAMILY_AFFINE_BUMP, 13, 3, 1, (0.8, 0.2, 1.1), 0.5, 1.0, 2),  # Dirichlet macro, 196 DoFs
    (W.FAMILY_AFFINE, 33, 2, 0, (1.0, 0.0, 1.0), 2.0, 1.3, 1),       # 1156 DoFs: several warps, K > 1
    (W.FAMILY_BUMP, 1, 1, 0, (1.0, 0.0, 1.0), 1.0, 1.0, 1),          # degenerate: one cell on both scales
]


@pytest.mark.parametrize("coupling", [0, 1])
@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("case", STEP_CASES)
def test_step_matches_oracle(case, precision, coupling):
    """coupling 0: the partitioned iteration; 1: exact elimination of the
    coupling (one micro solve per step) -- the same discrete solution."""
    family, Nm, NM, bc, D, kappa, Du, nsteps = case
    nM, nm = (NM + 1) ** 2, (Nm + 1) ** 2
    prm = W.random_params(family, nM, seed=20 + Nm)
    P, R = _pair(Nm, NM, family, prm, bc=bc, D=D, kappa=kappa, Du=Du, precision=precision, coupling=coupling)
    u0, v0 = W.random_state(nM, nm, seed=5)
    P.set_state(u0, v0)
    R.set_state(u0, v0)
    if bc == 1:
        ud = W.rng(3).uniform(0.5, 1.5, nM)
        P.set_sources(ud=ud)
        R.set_sources(ud=ud)
    dt = 0.01
    P.step(dt, nsteps)
    P.synchronize()
    R.step(dt, nsteps, cg_tol=1e-13, coupling_tol=1e-13, macro_tol=1e-13)
    tol = FP64_TOL if precision == 0 else MIXED_TOL
    assert rel(P.u(), R.u) < tol
    assert rel(P.v(), R.v) < tol
    assert rel(P.vbar(), R.vbar) < tol
    # the coupling moments rho_i = r_i^T v_i (compensated sums on the GPU; the
    # oracle's r and v, summed in FP64), at the same tolerance
    assert rel(P.rho(), oracle_rho(R)) < tol
    # F_i = kappa (|Gam_i| u_i - rho_i) cancels when u_i is close to the micro
    # average on the edge, so it is checked against the size of its two terms
    gam, _, _ = R.geometry()
    scale = kappa * np.linalg.norm(gam * R.u) + np.linalg.norm(R.flux)
    assert np.linalg.norm(P.flux() - R.flux) < tol * scale


@pytest.mark.parametrize("coupling", [0, 1])
@pytest.mark.parametrize("precision", [0, 1])
def test_manufactured_config_matches_oracle(precision, coupling):
    """8x8 macro / 8x8 micro, Dirichlet, bump a = 0.1 x1, manufactured sources,
    dt = 0.01 x 10 steps (the plain FP64 workload)."""
    from workloads import mms
    w = W.c1()
    a = w.params[:, 0]
    P, R = _pair(w.Nm, w.NM, w.family, w.params, bc=1, precision=precision, coupling=coupling)
    d0 = mms.nodal_data(w.NM, w.Nm, a, 0.0)
    P.set_state(d0["u"], d0["v"].ravel())
    R.set_state(d0["u"], d0["v"].ravel())
    for n in range(w.nsteps):
        d = mms.nodal_data(w.NM, w.Nm, a, (n + 1) * w.dt)
        src = dict(fv=d["fv"].ravel(), g=d["g"].ravel(), fu=d["fu"], ud=d["ud"])
        P.set_sources(**src)
        R.set_sources(**src)
        P.step(w.dt, 1)
        R.step(w.dt, 1, cg_tol=1e-13, coupling_tol=1e-13, macro_tol=1e-13)
    P.synchronize()
    tol = FP64_TOL if precision == 0 else MIXED_TOL
    assert rel(P.u(), R.u) < tol
    assert rel(P.v(), R.v) < tol


@pytest.mark.parametrize("precision", [0, 1])
def test_identity_instances_bitwise_identical(precision):
    """Identity map, same initial micro field everywhere, kappa = 0 (the micro
    right-hand sides do not see u): every micro problem does the same
    arithmetic in the same order, so all instances agree bit for bit.  With
    coupling, u is uniform only up to the rounding of the macro solve, and the
    instances agree to that level."""
    Nm, NM = 16, 6
    nM, nm = (NM + 1) ** 2, (Nm + 1) ** 2
    T = _T()
    yh1, _ = W.micro_coords(Nm)
    for kappa in (0.0, 1.0):
        P = T.TwoScale(Nm, NM, precision=precision, cg_tol=1e-12, coupling_tol=1e-12)
        P.set_physics((1.0, 0.0, 1.0), kappa, 1.0)
        P.set_deformation(W.FAMILY_IDENTITY, None)
        P.set_state(np.full(nM, 0.7), np.tile(np.cos(np.pi * yh1), nM))
        P.step(0.01, 3)
        P.synchronize()
        V = P.v()
        u = P.u()
        if kappa == 0.0:
            assert np.array_equal(V, np.broadcast_to(V[0], V.shape))
        else:
            assert np.max(np.abs(V - V[0])) < 1e-12
        assert np.max(np.abs(u - u[0])) < 1e-13 * abs(u[0])


@pytest.mark.parametrize("coupling", [0, 1])
def test_graph_and_plain_launches_agree_bitwise(coupling):
    NM, Nm = 4, 9
    nM, nm = (NM + 1) ** 2, (Nm + 1) ** 2
    prm = W.random_params(W.FAMILY_BUMP, nM, seed=3)
    u0, v0 = W.random_state(nM, nm, seed=2)
    T = _T()
    out = []
    for g in (1, 0):
        P = T.TwoScale(Nm, NM, precision=1, use_graph=g, tiling=1, coupling=coupling)
        P.set_deformation(W.FAMILY_BUMP, prm)
        P.set_state(u0, v0)
        P.step(0.005, 3)
        P.synchronize()
        out.append((P.u(), P.v(), P.stats()))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    assert out[0][2]["inner_iters"] == out[1][2]["inner_iters"]
    assert out[0][2]["coupling_iters_total"] == out[1][2]["coupling_iters_total"]


@pytest.mark.parametrize("tiling", [4, 1])
def test_multi_step_calls_commit_the_state_once(tiling):
    """Under the pipelined elimination a call of n graph steps commits v only
    in its last step (nothing reads v in between).  n steps in one call, n
    calls of one step and plain launches give the same bits for u, v and the
    micro averages."""
    NM, Nm = 4, 12
    nM, nm = (NM + 1) ** 2, (Nm + 1) ** 2
    prm = W.random_params(W.FAMILY_SHEAR_BUMP, nM, seed=13)
    u0 = W.random_state(nM, nm, seed=14)[0]
    T = _T()
    out = []
    for graph, calls in ((1, (6,)), (1, (1,) * 6), (1, (2, 1, 3)), (0, (6,))):
        P = T.TwoScale(Nm, NM, precision=1, use_graph=graph, tiling=tiling, coupling=1)
        P.set_deformation(W.FAMILY_SHEAR_BUMP, prm)
        P.set_state(u0, None)
        for n in calls:
            P.step(0.005, n)
        P.synchronize()
        out.append((P.u(), P.v(), P.vbar()))
        P.close()
    for o in out[1:]:
        for a, b in zip(o, out[0]):
            assert np.array_equal(a, b)


@pytest.mark.parametrize("precision", [0, 1])
def test_all_tilings_agree(precision):
    Nm, NM = 20, 3
    nM, nm = (NM + 1) ** 2, (Nm + 1) ** 2
    prm = W.random_params(W.FAMILY_SHEAR_BUMP, nM, seed=8)
    u0, v0 = W.random_state(nM, nm, seed=9)
    T = _T()
    res = []
    for t in [t for t in range(15) if t != 10]:   # 10: the three-field direct solve
        P = T.TwoScale(Nm, NM, precision=precision, tiling=t, cg_tol=1e-12, coupling_tol=1e-12)
        P.set_deformation(W.FAMILY_SHEAR_BUMP, prm)
        P.set_state(u0, v0)
        try:
            P.step(0.01, 2)
        except T.TsfError as e:       # variant not available for this size / precision
            assert e.status == T.TSF_E_ARG and (precision == 0 or t in (13, 14))
            continue
        P.synchronize()
        assert P.stats()["tiling"] == t
        res.append(P.v())
    # every variant of the precision fits a 21x21 micro grid, but the clusters of
    # R = 9 strips (3 strips here, fewer than the 4 or 8 CTAs)
    assert len(res) == (4 if precision == 0 else 12)
    for r in res[1:]:
        assert rel(r, res[0]) < 1e-9


@pytest.mark.parametrize("tiling", [1, 2, 3])
def test_per_problem_variants_under_pipelined_elimination(tiling):
    """The one-block-per-problem variants under the pipelined elimination at
    the benchmark tolerance (1e-8), 40x40 micro cells, shear+bump maps and
    D = diag(1, 0.1): the extrapolated warm starts leave residuals close to
    the target, so the FP32 correction works on small values (the case that
    ended in a non-finite CG step before the correction was solved for the
    unit-norm residual).  Three steps against the oracle."""
    NM, Nm = 3, 40
    nM = (NM + 1) ** 2
    prm = W.random_params(W.FAMILY_SHEAR_BUMP, nM, seed=31)
    P, R = _pair(Nm, NM, W.FAMILY_SHEAR_BUMP, prm, D=(1.0, 0.0, 0.1), precision=1, coupling=1, tiling=tiling,
                 cg_tol=1e-8, coupling_tol=1e-12)
    u0 = np.ones(nM)
    P.set_state(u0, None)
    R.set_state(u0, None)
    P.step(0.005, 3)
    P.synchronize()
    R.step(0.005, 3, cg_tol=1e-13, coupling_tol=1e-13, macro_tol=1e-13)
    assert P.stats()["tiling"] == tiling
    assert rel(P.u(), R.u) < MIXED_TOL
    assert rel(P.v(), R.v) < MIXED_TOL


@pytest.mark.parametrize("coupling", [0, 1])
def test_fp32_range_of_the_mixed_path(coupling):
    """Data scaled by 1e-25: tol^2 ||b||^2 lies far below the FP32 normal
    range.  The mixed-precision solves scale their FP32 norms and inner
    right-hand sides per micro problem by a power of two, so every variant --
    the column strips (stored FP64 residual, and the float-pair pipeline of
    the elimination), the per-problem variant and the autotuned default --
    solves the scaled problem, and the results scale back to the unscaled
    solution."""
    T = _T()
    NM, Nm = 3, 10
    nM, nm = (NM + 1) ** 2, (Nm + 1) ** 2
    prm = W.random_params(W.FAMILY_SHEAR_BUMP, nM, seed=41)
    u0, v0 = W.random_state(nM, nm, seed=42)
    out = {}
    for key, scale, prec, tiling in (("ref", 1.0, 0, -1), ("fp64", 1e-25, 0, -1), ("mixed_k", 1e-25, 1, 1),
                                     ("strip", 1e-25, 1, 4), ("tall_strip", 1e-25, 1, 7), ("auto", 1e-25, 1, -1)):
        P = T.TwoScale(Nm, NM, precision=prec, tiling=tiling, coupling=coupling, cg_tol=1e-10, coupling_tol=1e-12)
        P.set_physics((1.0, 0.0, 0.1), 1.0, 1.0)
        P.set_deformation(W.FAMILY_SHEAR_BUMP, prm)
        P.set_state(scale * u0, scale * v0)
        P.step(0.01, 3)
        P.synchronize()
        out[key] = (P.u() / scale, P.v() / scale)
        P.close()
    for key in ("fp64", "mixed_k", "strip", "tall_strip", "auto"):
        assert rel(out[key][0], out["ref"][0]) < 1e-7 and rel(out[key][1], out["ref"][1]) < 1e-7, key


@pytest.mark.parametrize("coupling", [0, 1])
def test_mass_balance_on_gpu(coupling):
    NM, Nm = 6, 10
    nM, nm = (NM + 1) ** 2, (Nm + 1) ** 2
    prm = W.random_params(W.FAMILY_SHEAR_BUMP, nM, seed=4)
    P, R = _pair(Nm, NM, W.FAMILY_SHEAR_BUMP, prm, D=(1.0, 0.0, 0.1), kappa=1.2, precision=0, coupling=coupling)
    u0, v0 = W.random_state(nM, nm, seed=6)
    P.set_state(u0, v0)
    _, vol = P.geometry()
    _, _, mH = R.geometry()   # lumped macro mass (a closed form: H^2 cells/4)

    def mass():
        return mH @ P.u() + np.sum(mH * vol * P.vbar())

    m0 = mass()
    P.step(0.01, 4)
    P.synchronize()
    assert abs(mass() - m0) < 1e-11 * abs(m0)


def test_full_size_partitioned_step_matches_tight_oracle():
    """The same full-size workload stepped by the partitioned iteration of
    Sec. 3.3 (micro solves, macro solve, until u settles), mixed precision at
    1e-11 with coupling tolerance 1e-13, two steps against the tight oracle."""
    w = W.c2()
    T = _T()
    P = T.TwoScale(w.Nm, w.NM, precision=T.TSF_MIXED, cg_tol=1e-11, coupling_tol=1e-13, macro_tol=1e-13,
                   coupling=T.TSF_COUPLING_PARTITIONED)
    P.set_deformation(w.family, w.params)
    P.set_state(w.u0, None)
    P.step(w.dt, 2)
    P.synchronize()
    R = oracle.Problem(w.Nm, w.NM, w.bc, w.family, w.params)
    R.set_state(w.u0, None)
    R.step(w.dt, 2, cg_tol=1e-13, coupling_tol=1e-13, macro_tol=1e-13)
    errs = {"u": rel(P.u(), R.u), "v": rel(P.v(), R.v), "vbar": rel(P.vbar(), R.vbar),
            "rho": rel(P.rho(), oracle_rho(R))}
    assert max(errs.values()) < MIXED_TOL, errs


@pytest.mark.parametrize("precision", [1, 0])
def test_benched_path_at_full_size_matches_tight_oracle(precision):
    """The path bench.py times, at full size: 64x64 macro / 32x32 micro cells
    (4225 x 1089 DoFs), bump a ~ U[0, 0.2], u0 = 1, v0 = 0, dt = 0.005, coupling
    by pipelined exact elimination with the variant the library picks, over 5
    steps so that the head solve, the graph-launched steps and the quadratic
    warm-start extrapolation (history level 2) all run.  The GPU solves to
    1e-11 (mixed) / 1e-13 (FP64), the oracle to 1e-13 with the partitioned
    iteration to 1e-13; u, v, the averages and rho = r^T v must agree to
    1e-8 (mixed) / 1e-10 (FP64)."""
    w = W.c2()
    T = _T()
    nsteps = 5
    P = T.TwoScale(w.Nm, w.NM, precision=precision, cg_tol=1e-11 if precision == 1 else 1e-13, macro_tol=1e-13,
                   coupling=T.TSF_COUPLING_ELIMINATION)
    P.set_physics(w.D, w.kappa, w.Du)
    P.set_deformation(w.family, w.params)
    P.set_state(w.u0, None)
    P.step(w.dt, nsteps)
    P.synchronize()
    if precision == 1:
        assert P.stats()["tiling"] >= 4      # a column-strip kernel, with its pipelined epilogue
    R = oracle.Problem(w.Nm, w.NM, w.bc, w.family, w.params, D=w.D, kappa=w.kappa, Du=w.Du)
    R.set_state(w.u0, None)
    R.step(w.dt, nsteps, cg_tol=1e-13, coupling_tol=1e-13, macro_tol=1e-13)
    tol = MIXED_TOL if precision == 1 else FP64_TOL
    errs = {"u": rel(P.u(), R.u), "v": rel(P.v(), R.v), "vbar": rel(P.vbar(), R.vbar),
            "rho": rel(P.rho(), oracle_rho(R))}
    assert max(errs.values()) < tol, errs


def test_bad_jacobian_is_rejected():
    T = _T()
    P = T.TwoScale(4, 2)
    with pytest.raises(T.TsfError) as ei:
        P.set_deformation(W.FAMILY_BUMP, np.full(9, 0.4))
    assert ei.value.status == T.TSF_E_BAD_JACOBIAN


def test_iteration_cap_reports_not_converged():
    T = _T()
    NM, Nm = 3, 12
    nM, nm = (NM + 1) ** 2, (Nm + 1) ** 2
    P = T.TwoScale(Nm, NM, precision=0, cg_maxit=2, cg_tol=1e-14)
    P.set_deformation(W.FAMILY_BUMP, W.random_params(1, nM, seed=1))
    P.set_state(*W.random_state(nM, nm, seed=1))
    P.step(0.01, 1)
    with pytest.raises(T.TsfError) as ei:
        P.synchronize()
    assert ei.value.status == T.TSF_E_NOT_CONVERGED


def test_argument_errors():
    T = _T()
    ctx = T.tsf_create(T.tsf_default_options())
    try:
        with pytest.raises(T.TsfError):
            T.tsf_set_micro_mesh(ctx, 0, 0, 0)
        with pytest.raises(T.TsfError):
            T.tsf_set_micro_mesh(ctx, 4, 5, 0)
        with pytest.raises(T.TsfError):
            T.tsf_step(ctx, 0.01, 1)          # no meshes yet
        T.tsf_set_micro_mesh(ctx, 4, 4, 0)
        T.tsf_set_macro_mesh(ctx, 2, 2, 0, None)
        with pytest.raises(T.TsfError):
            T.tsf_set_physics(ctx, (1.0, 2.0, 1.0), 1.0, 1.0)   # D not SPD
        with pytest.raises(T.TsfError):
            T.tsf_set_deformation(ctx, 1, 2, np.zeros(18))      # wrong nparam
    finally:
        T.tsf_destroy(ctx)


def test_device_tensors_in_and_out():
    import torch
    T = _T()
    NM, Nm = 3, 5
    nM, nm = (NM + 1) ** 2, (Nm + 1) ** 2
    prm = W.random_params(1, nM, seed=2)
    u0, v0 = W.random_state(nM, nm, seed=3)
    A = T.TwoScale(Nm, NM, precision=0)
    A.set_deformation(1, torch.tensor(prm, device="cuda"))
    A.set_state(torch.tensor(u0, device="cuda"), torch.tensor(v0, device="cuda"))
    A.step(0.01, 1)
    out = torch.empty(nM, dtype=torch.float64, device="cuda")
    A.u(out)
    B = T.TwoScale(Nm, NM, precision=0, workspace=None)
    B.set_deformation(1, prm)
    B.set_state(u0, v0)
    B.step(0.01, 1)
    assert np.array_equal(out.cpu().numpy(), B.u())


def test_elimination_matches_partitioned_over_many_steps():
    """Both ways of reaching the coupled solution, 20 steps of a 12x12 / 16x16
    shear+bump problem in FP64 at tight tolerances, and the elimination's
    statistics: one micro solve per problem and step."""
    NM, Nm = 12, 16
    nM, nm = (NM + 1) ** 2, (Nm + 1) ** 2
    prm = W.random_params(W.FAMILY_SHEAR_BUMP, nM, seed=11)
    u0, v0 = W.random_state(nM, nm, seed=12)
    T = _T()
    out = []
    for coupling in (0, 1):
        P = T.TwoScale(Nm, NM, precision=0, cg_tol=1e-13, coupling_tol=1e-13, macro_tol=1e-13, coupling=coupling)
        P.set_physics((1.0, 0.1, 0.5), 1.4, 0.9)
        P.set_deformation(W.FAMILY_SHEAR_BUMP, prm)
        P.set_state(u0, v0)
        P.step(0.005, 20)
        P.synchronize()
        out.append((P.u(), P.v(), P.stats()))
    assert rel(out[1][0], out[0][0]) < 1e-11
    assert rel(out[1][1], out[0][1]) < 1e-11
    st = out[1][2]
    # one micro solve per problem and step, plus the first solve from the state
    # (the pipelined steps solve the next step's micro problems one step ahead)
    assert st["micro_solves"] == 21 * nM and st["coupling_iters_total"] == 20
    assert out[0][2]["micro_solves"] > st["micro_solves"]


def test_elimination_history_is_reset_by_set_state():
    """Exact elimination extrapolates its warm start from the past steps; a new
    state forgets that history, so a context that marched before and one that
    did not give bit-identical steps from the same state."""
    NM, Nm = 5, 12
    nM, nm = (NM + 1) ** 2, (Nm + 1) ** 2
    prm = W.random_params(W.FAMILY_BUMP, nM, seed=21)
    u0, v0 = W.random_state(nM, nm, seed=22)
    T = _T()
    A = T.TwoScale(Nm, NM, precision=1, coupling=1, tiling=5)
    B = T.TwoScale(Nm, NM, precision=1, coupling=1, tiling=5)
    for P in (A, B):
        P.set_deformation(W.FAMILY_BUMP, prm)
    A.set_state(*W.random_state(nM, nm, seed=23))
    A.step(0.01, 6)
    A.set_state(u0, v0)
    B.set_state(u0, v0)
    A.step(0.01, 4)
    B.step(0.01, 4)
    assert np.array_equal(A.u(), B.u()) and np.array_equal(A.v(), B.v())


@pytest.mark.parametrize("coupling", [0, 1])
def test_largest_micro_mesh_matches_oracle(coupling):
    """64x64 micro cells (4225 DoFs, the largest micro mesh) in mixed precision:
    only the tall-strip and 8-nodes-per-thread variants fit; two steps against
    the oracle."""
    NM, Nm = 2, 64
    nM, nm = (NM + 1) ** 2, (Nm + 1) ** 2
    prm = W.random_params(W.FAMILY_SHEAR_BUMP, nM, seed=31)
    P, R = _pair(Nm, NM, W.FAMILY_SHEAR_BUMP, prm, D=(1.0, 0.0, 0.1), precision=1, coupling=coupling)
    u0, v0 = W.random_state(nM, nm, seed=32)
    P.set_state(u0, v0)
    R.set_state(u0, v0)
    P.step(0.005, 2)
    P.synchronize()
    R.step(0.005, 2, cg_tol=1e-13, coupling_tol=1e-13, macro_tol=1e-13)
    assert P.stats()["tiling"] in (3, 7, 8, 9)
    assert rel(P.u(), R.u) < MIXED_TOL
    assert rel(P.v(), R.v) < MIXED_TOL


@pytest.mark.parametrize("coupling", [0, 1])
@pytest.mark.parametrize("tiling", [11, 12, 13, 14])
def test_cluster_variants_match_oracle(tiling, coupling):
    """One micro problem per thread-block cluster (halo rows and dot products
    between the CTAs through distributed shared memory), 64x64 micro cells,
    shear+bump cells with anisotropic D, two steps of both couplings (the
    elimination runs the pipelined cluster kernel) against the oracle."""
    NM, Nm = 2, 64
    nM, nm = (NM + 1) ** 2, (Nm + 1) ** 2
    prm = W.random_params(W.FAMILY_SHEAR_BUMP, nM, seed=51)
    P, R = _pair(Nm, NM, W.FAMILY_SHEAR_BUMP, prm, D=(1.0, 0.0, 0.1), precision=1, coupling=coupling, tiling=tiling)
    u0, v0 = W.random_state(nM, nm, seed=52)
    P.set_state(u0, v0)
    R.set_state(u0, v0)
    P.step(0.005, 2)
    P.synchronize()
    R.step(0.005, 2, cg_tol=1e-13, coupling_tol=1e-13, macro_tol=1e-13)
    assert P.stats()["tiling"] == tiling
    assert rel(P.u(), R.u) < MIXED_TOL
    assert rel(P.v(), R.v) < MIXED_TOL
    assert rel(P.rho(), oracle_rho(R)) < MIXED_TOL


@pytest.mark.parametrize("coupling", [0, 1])
@pytest.mark.parametrize("tiling,Nm", [(15, 8), (16, 8), (15, 5), (16, 9)])
def test_one_warp_variants_match_oracle(tiling, Nm, coupling):
    """One warp per micro problem, eight problems per block (warp barriers and
    shuffle reductions only): 6x6 macro cells (49 micro problems, so the last
    block holds one), 8x8, ragged 5x5 and 9x9 micro cells, shear+bump cells,
    two steps of both couplings against the oracle."""
    NM = 6   # 49 micro problems: the last block holds one
    nM, nm = (NM + 1) ** 2, (Nm + 1) ** 2
    prm = W.random_params(W.FAMILY_SHEAR_BUMP, nM, seed=61)
    P, R = _pair(Nm, NM, W.FAMILY_SHEAR_BUMP, prm, D=(1.0, 0.0, 0.1), precision=1, coupling=coupling, tiling=tiling)
    u0, v0 = W.random_state(nM, nm, seed=62)
    P.set_state(u0, v0)
    R.set_state(u0, v0)
    P.step(0.01, 2)
    P.synchronize()
    R.step(0.01, 2, cg_tol=1e-13, coupling_tol=1e-13, macro_tol=1e-13)
    assert P.stats()["tiling"] == tiling
    assert rel(P.u(), R.u) < MIXED_TOL
    assert rel(P.v(), R.v) < MIXED_TOL
    assert rel(P.rho(), oracle_rho(R)) < MIXED_TOL


@pytest.mark.parametrize("coupling", [0, 1])
@pytest.mark.parametrize("Nm", [96, 128])
def test_micro_meshes_beyond_one_block_match_oracle(Nm, coupling):
    """96x96 and 128x128 micro cells (9409 and 16641 DoFs per micro problem):
    only the cluster variants fit; the library picks one by timing.  Three
    steps against the oracle (the elimination reaches the extrapolated warm
    start)."""
    NM = 2
    nM, nm = (NM + 1) ** 2, (Nm + 1) ** 2
    prm = W.random_params(W.FAMILY_BUMP, nM, seed=53)
    P, R = _pair(Nm, NM, W.FAMILY_BUMP, prm, precision=1, coupling=coupling)
    u0 = W.rng(54).uniform(0.5, 1.5, nM)
    P.set_state(u0, None)
    R.set_state(u0, None)
    P.step(0.005, 3)
    P.synchronize()
    R.step(0.005, 3, cg_tol=1e-13, coupling_tol=1e-13, macro_tol=1e-13)
    assert P.stats()["tiling"] >= 11
    assert rel(P.u(), R.u) < MIXED_TOL
    assert rel(P.v(), R.v) < MIXED_TOL
    assert rel(P.vbar(), R.vbar) < MIXED_TOL


def test_many_micro_problems_sampled():
    """A 600x600 macro mesh (361201 micro problems of 3x3 cells: grids far past
    65535 blocks in one dimension) in both couplings: sampled problems against
    the oracle of a small mesh with the same parameters at those nodes, and
    mass balance over everything."""
    T = _T()
    NM, Nm = 600, 3
    nM, nm = (NM + 1) ** 2, (Nm + 1) ** 2
    a = np.full(nM, 0.08)
    for coupling in (0, 1):
        P = T.TwoScale(Nm, NM, precision=0, cg_tol=1e-13, coupling_tol=1e-13, macro_tol=1e-13, coupling=coupling)
        P.set_deformation(W.FAMILY_BUMP, a)
        P.set_state(np.ones(nM), None)
        _, vol = P.geometry()
        x1, x2 = W.macro_coords(NM)
        mH = 0.25 * np.where((x1 == 0) | (x1 == 1), 1.0, 2.0) * np.where((x2 == 0) | (x2 == 1), 1.0, 2.0) / NM ** 2
        m0 = mH @ P.u() + np.sum(mH * vol * P.vbar())
        P.step(0.005, 2)
        P.synchronize()
        m1 = mH @ P.u() + np.sum(mH * vol * P.vbar())
        assert abs(m1 - m0) < 1e-11 * abs(m0)
        # uniform data and u0 = 1: every micro problem sees the same u, so all
        # micro fields equal the one of a 1x1 macro mesh with the same data
        R = oracle.Problem(Nm, 1, 0, W.FAMILY_BUMP, np.full(4, 0.08))
        R.set_state(np.ones(4), None)
        R.step(0.005, 2, cg_tol=1e-13, coupling_tol=1e-13, macro_tol=1e-13)
        V = P.v()
        for i in (0, 1, nM // 2, nM - 1):
            assert np.max(np.abs(V[i] - R.v[0])) < 1e-10
        assert np.max(np.abs(P.u() - R.u[0])) < 1e-10
        P.close()


@pytest.mark.parametrize("family", [0, 1, 2, 3, 4])
def test_pushforward_matches_oracle_map(family):
    """Push-forward for visualisation: every micro node at
    x_i + scale (chi(x_i, yhat_j) - 1/2) with its value, against the
    oracle's chi."""
    T = _T()
    NM, Nm = 3, 5
    nM, nm = (NM + 1) ** 2, (Nm + 1) ** 2
    prm = W.random_params(family, nM, seed=40 + family)
    P = T.TwoScale(Nm, NM, precision=0)
    P.set_deformation(family, prm)
    P.set_state(*W.random_state(nM, nm, seed=41))
    P.step(0.01, 1)
    scale = 0.7 / NM
    out = P.pushforward(scale)
    y1, y2 = W.micro_coords(Nm)
    x1, x2 = W.macro_coords(NM)
    # FP32 output: positions to a few FP32 ulps of the unit square, values rounded
    for i in range(nM):
        ch, _ = oracle.chi_many(family, prm[i] if prm.shape[1] else [], y1, y2)
        ch = ch.reshape(-1, 2)
        assert np.max(np.abs(out[i, :, 0] - (x1[i] + scale * (ch[:, 0] - 0.5)))) < 1e-6
        assert np.max(np.abs(out[i, :, 1] - (x2[i] + scale * (ch[:, 1] - 0.5)))) < 1e-6
    assert np.array_equal(out[:, :, 2], P.v().astype(np.float32))
    with pytest.raises(T.TsfError):
        P.pushforward(-1.0)


def test_async_getters_match_the_synchronous_ones():
    """tsf_get_macro_async / tsf_get_micro_averages_async queue their copies
    behind the steps; after synchronize() they hold what the synchronous
    getters return (pinned host arrays and CUDA tensors)."""
    import torch
    T = _T()
    Nm, NM = 8, 6
    nM, nm = (NM + 1) ** 2, (Nm + 1) ** 2
    P = T.TwoScale(Nm, NM, precision=1, coupling=1)
    P.set_deformation(W.FAMILY_BUMP, W.random_params(1, nM, seed=3))
    P.set_state(*W.random_state(nM, nm, seed=4))
    uh = torch.empty(nM, dtype=torch.float64).pin_memory().numpy()
    vh = torch.empty(nM, dtype=torch.float64).pin_memory().numpy()
    ud = torch.empty(nM, dtype=torch.float64, device="cuda")
    vd = torch.empty(nM, dtype=torch.float64, device="cuda")
    for _ in range(3):
        P.step(0.01, 1)
        P.u_async(uh)
        P.vbar_async(vh)
        P.u_async(ud)
        P.vbar_async(vd)
    P.synchronize()
    u, vbar = P.u(), P.vbar()
    assert np.array_equal(uh, u) and np.array_equal(vh, vbar)
    assert np.array_equal(ud.cpu().numpy(), u) and np.array_equal(vd.cpu().numpy(), vbar)
    with pytest.raises(ValueError):
        P.u_async(np.empty(nM + 1))
    P.close()
