"""The macro solve for callers that cannot allocate device memory.

tsf_macro_solve_noalloc serves programs that cannot call cudaMalloc when they
need a solve (all device memory handed to their own pool, or a latency-bound
loop where a device-synchronising allocation is not acceptable).  It runs the
macro-solve kernel of tsf_step on caller arrays with the library's fixed
scratch array.  This test reproduces, through the C ABI, the final macro solve
of a full step taken with the existing entry point (tsf_step) and checks the
two results agree within the FP64 parity tolerance, on two calls in a row
(different problems, so the second call must not see the first one's leftover
scratch contents), then repeats the first call and expects identical bits.

This file is named so that pytest collects it last.
"""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-10  # FP64 parity tolerance used by the other GPU tests


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _reference_step(T, NM, Nm, bc, family, prm, kappa, Du, dt, seed):
    """One FP64 step with tsf_step; returns what the last macro solve saw and produced."""
    nM, nm = (NM + 1) ** 2, (Nm + 1) ** 2
    u_n, v_n = W.random_state(nM, nm, seed=seed)
    P = T.TwoScale(Nm, NM, bc=bc, precision=T.TSF_FP64, cg_tol=1e-13, coupling_tol=1e-13, macro_tol=1e-13)
    P.set_physics((1.0, 0.0, 1.0), kappa, Du)
    P.set_deformation(family, prm)
    P.set_state(u_n, v_n)
    u0 = u_n.copy()
    if bc == T.TSF_BC_DIRICHLET:
        ud = W.rng(seed + 1).uniform(0.5, 1.5, nM)
        P.set_sources(ud=ud)
        x1, x2 = W.macro_coords(NM)
        bnd = (x1 == 0) | (x2 == 0) | (x1 == 1) | (x2 == 1)
        u0[bnd] = ud[bnd]
    P.step(dt, 1)
    P.synchronize()
    u_ref = P.u()
    gam, _ = P.geometry()
    # rho_i = r_i^T v_i of the final micro iterate, from the flux F_i = kappa (|Gam_i| u_i - rho_i)
    rho = gam * u_ref - P.flux() / kappa if kappa > 0 else np.zeros(nM)
    # cH = M_H u^n / dt (no macro source)
    MH = oracle.Problem(Nm, NM, bc, family, prm).macro_csr("M")
    cH = MH @ u_n / dt
    P.close()
    return gam, cH, rho, u0, u_ref


def test_noalloc_macro_solve_matches_step():
    import torch
    import paper_2103_17040_gb300 as T
    T.load_library()
    dev = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")  # noqa: E731
    cases = [
        # NM, Nm, bc, family, kappa, Du, dt
        (8, 6, T.TSF_BC_NEUMANN, W.FAMILY_SHEAR_BUMP, 1.3, 0.8, 0.01),
        (5, 4, T.TSF_BC_DIRICHLET, W.FAMILY_BUMP, 0.0, 1.2, 0.02),
    ]
    first = None
    for n, (NM, Nm, bc, fam, kappa, Du, dt) in enumerate(cases):
        prm = W.random_params(fam, (NM + 1) ** 2, seed=30 + n)
        gam, cH, rho, u0, u_ref = _reference_step(T, NM, Nm, bc, fam, prm, kappa, Du, dt, seed=40 + n)
        args = [dev(a) for a in (gam, cH, rho, u0)]
        out = torch.empty_like(args[3])
        iters = T.tsf_macro_solve_noalloc(NM, bc, dt, Du, kappa, *args, out, tol=1e-13, maxit=500)
        u = out.cpu().numpy()
        assert iters >= 1
        assert _rel(u, u_ref) < TOL, (n, _rel(u, u_ref))
        if first is None:
            first = (NM, bc, dt, Du, kappa, args, u)
    # the first problem again, after the second one used the same scratch
    NM, bc, dt, Du, kappa, args, u1 = first
    out = torch.empty_like(args[3])
    T.tsf_macro_solve_noalloc(NM, bc, dt, Du, kappa, *args, out, tol=1e-13, maxit=500)
    assert np.array_equal(out.cpu().numpy(), u1)


def test_noalloc_at_its_size_limit():
    """NM = TSF_NOALLOC_MAX_NM (the largest mesh the fixed scratch array
    holds; the fast-diagonalisation preconditioner then takes about 207 KB of
    shared memory) with the Neumann and the Dirichlet boundary, one call after
    the other, against the macro solve inside tsf_step."""
    import torch
    import paper_2103_17040_gb300 as T
    T.load_library()
    NM = T.TSF_NOALLOC_MAX_NM
    dev = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")  # noqa: E731
    for n, (bc, fam, kappa, Du, dt) in enumerate(((T.TSF_BC_NEUMANN, W.FAMILY_BUMP, 1.0, 1.0, 0.01),
                                                  (T.TSF_BC_DIRICHLET, W.FAMILY_SHEAR_BUMP, 0.7, 1.1, 0.005))):
        prm = W.random_params(fam, (NM + 1) ** 2, seed=60 + n)
        gam, cH, rho, u0, u_ref = _reference_step(T, NM, 2, bc, fam, prm, kappa, Du, dt, seed=70 + n)
        args = [dev(a) for a in (gam, cH, rho, u0)]
        out = torch.empty_like(args[3])
        T.tsf_macro_solve_noalloc(NM, bc, dt, Du, kappa, *args, out, tol=1e-13, maxit=500)
        assert _rel(out.cpu().numpy(), u_ref) < TOL, (bc, _rel(out.cpu().numpy(), u_ref))


def test_noalloc_rejects_tensors_on_another_device():
    import torch
    import paper_2103_17040_gb300 as T
    T.load_library()
    z = torch.zeros(9, dtype=torch.float64)   # host tensor: not on the current CUDA device
    with pytest.raises(ValueError):
        T.tsf_macro_solve_noalloc(2, 0, 0.01, 1.0, 1.0, z, z, z, z, z)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    import paper_2103_17040_gb300 as T
    T.load_library()
    NM = T.TSF_NOALLOC_MAX_NM + 1
    z = torch.zeros((NM + 1) ** 2, dtype=torch.float64, device="cuda")
    with pytest.raises(T.TsfError) as ei:
        T.tsf_macro_solve_noalloc(NM, 0, 0.01, 1.0, 1.0, z, z, z, z, z)
    assert ei.value.status == T.TSF_E_ARG
