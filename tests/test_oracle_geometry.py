"""Pins of the oracle's geometry and assembly (pull-back factors, element
matrices) against closed forms, the paper's printed constants and textbook
special cases.  CPU only."""
import json
import os

import numpy as np
import pytest

import oracle
import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_paper_affine_normals():
    """cof(F) nu / |cof(F) nu| reproduces the normal coefficients printed in
    the manufactured data of Sec. 4.2 (Eq. (20)) for the map of Eq. (19)."""
    d = json.load(open(os.path.join(GOLD, "paper_affine_normals.json")))
    F = np.array(d["F"])
    # the map of Eq. (19) is affine: F is its linear part
    assert np.allclose(F, [[0.4 * 1.4, -0.4 * 0.54], [-0.3 * 0.4, 0.3 * 0.8]])
    for e in d["edges"]:
        n = oracle.unit_normal(F, e["nu"])
        assert np.max(np.abs(n - np.array(e["normal"]))) < d["abs_tol"], (e, n)
    # determinant quoted for the same map
    J, _, _ = oracle.pullback(F)
    assert abs(J - 0.10848) < 1e-12


def test_rate_formula_reproduces_paper_tables():
    """The observed-order formula used by the convergence test reproduces the
    orders printed in Tables 1 and 2 (rows 2-7)."""
    d = json.load(open(os.path.join(GOLD, "paper_convergence_tables.json")))
    for t in ("table1", "table2"):
        T = d[t]
        N = np.array(T["dofs"], float)
        for key, pk in (("e", "p"), ("e_grad", "q")):
            e = np.array(T[key])
            p = 2 * np.log(e[:-1] / e[1:]) / np.log(N[1:] / N[:-1])
            assert np.max(np.abs(p - np.array(T[pk]))) < d["rate_abs_tol"]


def _problem(family, params, Nm=6, NM=2, D=(1.0, 0.0, 1.0), kappa=1.0):
    return oracle.Problem(Nm, NM, 0, family, params, D=D, kappa=kappa)


def test_bump_volume_and_robin_length():
    """Bump map fixes the boundary pointwise: |Y_x| = 1 and |Gamma| = 1 exactly
    (the Gauss sums of cos(pi y1) cancel on symmetric meshes)."""
    nM = 9
    a = W.rng(3).uniform(0.0, 0.3, (nM, 1))
    P = _problem(1, a, Nm=8)
    gam, vol, mH = P.geometry()
    assert np.allclose(vol, 1.0, atol=1e-14, rtol=0)
    assert np.allclose(gam, 1.0, atol=1e-14, rtol=0)


def test_shear_bump_robin_length():
    """Shear s moves the right edge to a segment of length sqrt(1 + s^2)."""
    nM = 9
    prm = W.random_params(2, nM, seed=4)
    P = _problem(2, prm, Nm=8)
    gam, vol, _ = P.geometry()
    assert np.allclose(gam, np.sqrt(1 + prm[:, 0] ** 2), atol=1e-13, rtol=0)
    assert np.allclose(vol, 1.0, atol=1e-13, rtol=0)


def test_affine_area_and_edge_length():
    """Affine map: |Y_x| = |det A|, |Gamma| = length of the image of the edge
    from (1,0) to (1,1) = |A e2|."""
    nM = 9
    prm = W.random_params(3, nM, seed=5)
    P = _problem(3, prm, Nm=5)
    gam, vol, _ = P.geometry()
    A = prm[:, :4].reshape(nM, 2, 2)
    assert np.allclose(vol, np.abs(np.linalg.det(A)), atol=1e-13, rtol=0)
    assert np.allclose(gam, np.linalg.norm(A[:, :, 1], axis=1), atol=1e-13, rtol=0)


@pytest.mark.parametrize("family", [1, 2, 3, 4])
def test_element_matrix_structure(family):
    """A 1 = 0 (constants are in the kernel of the stiffness), M, A, R
    symmetric, M positive definite, A positive semidefinite."""
    nM = 9
    P = _problem(family, W.random_params(family, nM, seed=family), Nm=5, D=(1.0, 0.2, 0.5))
    for i in (0, 4, 8):
        M = P.micro_csr(i, "M").toarray()
        A = P.micro_csr(i, "A").toarray()
        R = P.micro_csr(i, "R").toarray()
        assert np.max(np.abs(A @ np.ones(len(A)))) < 1e-13
        for X in (M, A, R):
            assert np.max(np.abs(X - X.T)) < 1e-14
        assert np.min(np.linalg.eigvalsh(M)) > 0
        assert np.min(np.linalg.eigvalsh(A)) > -1e-12


def _parallelogram_flux_vector(Nm, A, c, D, alpha):
    """int_{dY} (D grad l . n) psi_j dsigma for l(y) = alpha . y on the
    parallelogram Y = A Z + c, computed from the vertex coordinates only."""
    n1 = Nm + 1
    h = 1.0 / Nm
    Dm = np.array([[D[0], D[1]], [D[1], D[2]]])
    flux = Dm @ alpha
    verts = [A @ v + c for v in (np.array([0, 0.]), np.array([1, 0.]), np.array([1, 1.]), np.array([0, 1.]))]
    orient = np.sign(np.linalg.det(A))
    b = np.zeros(n1 * n1)
    # reference edges in counter-clockwise order with their node lists
    edges = [
        ([p for p in range(n1)], 0, 1),                          # bottom  q = 0
        ([Nm + n1 * q for q in range(n1)], 1, 2),                # right   p = Nm
        ([p + n1 * Nm for p in range(Nm, -1, -1)], 2, 3),        # top     q = Nm
        ([n1 * q for q in range(Nm, -1, -1)], 3, 0),             # left    p = 0
    ]
    for nodes, a0, a1 in edges:
        t = verts[a1] - verts[a0]
        L = np.linalg.norm(t)
        n = orient * np.array([t[1], -t[0]]) / L                 # outward normal
        w = np.full(n1, h)
        w[0] = w[-1] = h / 2
        for node, wj in zip(nodes, w):
            b[node] += flux @ n * L * wj
    return b


@pytest.mark.parametrize("D", [(1.0, 0.0, 1.0), (1.0, 0.0, 0.1), (0.7, 0.25, 1.3)])
def test_patch_test_affine(D):
    """Patch test: for an affine map, the stiffness applied to the nodal
    interpolant of a physical linear function equals its exact boundary flux
    vector.  Pins C = J F^{-1} D F^{-T} including the transposes and the
    position of D."""
    Nm = 6
    nM = 9
    prm = W.random_params(3, nM, seed=11)
    P = _problem(3, prm, Nm=Nm, D=D)
    yh1, yh2 = W.micro_coords(Nm)
    alpha = np.array([0.8, -1.3])
    for i in range(nM):
        A = prm[i, :4].reshape(2, 2)
        c = prm[i, 4:6]
        y = (A @ np.stack([yh1, yh2])).T + c
        lh = y @ alpha + 0.37
        lhs = P.micro_csr(i, "A") @ lh
        rhs = _parallelogram_flux_vector(Nm, A, c, D, alpha)
        assert np.max(np.abs(lhs - rhs)) < 1e-12 * max(1, np.max(np.abs(rhs)))


def test_robin_mass_is_scaled_1d_mass():
    """On an affine map the Robin matrix is the textbook 1D Q1 mass matrix of
    the edge, (h/6) tridiag(1, 4, 1) with halved end diagonals, times the
    physical edge length."""
    Nm = 7
    nM = 4
    prm = W.random_params(3, nM, seed=2)
    P = oracle.Problem(Nm, 1, 0, 3, prm)
    n1 = Nm + 1
    h = 1.0 / Nm
    M1 = (h / 6) * (np.diag(np.full(n1, 4.0)) + np.diag(np.ones(n1 - 1), 1) + np.diag(np.ones(n1 - 1), -1))
    M1[0, 0] = M1[-1, -1] = 2 * h / 6
    edge = [Nm + n1 * q for q in range(n1)]
    for i in range(nM):
        A = prm[i, :4].reshape(2, 2)
        R = P.micro_csr(i, "R").toarray()
        L = np.linalg.norm(A[:, 1])
        assert np.max(np.abs(R[np.ix_(edge, edge)] - L * M1)) < 1e-14
        mask = np.ones(n1 * n1, bool)
        mask[edge] = False
        assert np.all(R[mask] == 0) and np.all(R[:, mask] == 0)


def test_identity_matrices_are_tensor_products():
    """Identity map, D = I: M = M1 (x) M1 and A = K1 (x) M1 + M1 (x) K1 with the
    textbook 1D Q1 matrices (Sec. 3.1 spaces on a uniform mesh)."""
    Nm = 5
    P = oracle.Problem(Nm, 1, 0, 0, np.zeros((4, 0)))
    n1 = Nm + 1
    h = 1.0 / Nm
    M1 = (h / 6) * (np.diag(np.full(n1, 4.0)) + np.diag(np.ones(n1 - 1), 1) + np.diag(np.ones(n1 - 1), -1))
    M1[0, 0] = M1[-1, -1] = 2 * h / 6
    K1 = (1 / h) * (np.diag(np.full(n1, 2.0)) - np.diag(np.ones(n1 - 1), 1) - np.diag(np.ones(n1 - 1), -1))
    K1[0, 0] = K1[-1, -1] = 1 / h
    # node index p + n1 q: q is the slow index -> kron(Y-matrix, X-matrix)
    assert np.max(np.abs(P.micro_csr(0, "M").toarray() - np.kron(M1, M1))) < 1e-15
    Aref = np.kron(M1, K1) + np.kron(K1, M1)
    assert np.max(np.abs(P.micro_csr(0, "A").toarray() - Aref)) < 1e-13
    MH = P.macro_csr("M").toarray()
    assert np.allclose(MH.sum(), 1.0)


def test_bad_jacobian_rejected():
    """det F <= 0 somewhere (bump amplitude a > 1/pi) is refused (Eq. (3))."""
    prm = np.full((4, 1), 0.4)
    with pytest.raises(oracle.OracleError) as ei:
        oracle.Problem(4, 1, 0, 1, prm)
    assert ei.value.code == oracle.OR_E_BAD_JACOBIAN


def test_pcg_matches_direct_solve():
    """The oracle's Jacobi-PCG against a sparse direct solve."""
    import scipy.sparse.linalg as spla
    P = _problem(2, W.random_params(2, 9, seed=7), Nm=9)
    dt = 0.01
    S = (P.micro_csr(3, "M") / dt + P.micro_csr(3, "A") + P.micro_csr(3, "R")).tocsr()
    b = W.rng(1).standard_normal(S.shape[0])
    x, it, rr, e = oracle.pcg(S, b, tol=1e-14)
    assert e == 0 and rr <= 1e-14
    xd = spla.spsolve(S.tocsc(), b)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-12
