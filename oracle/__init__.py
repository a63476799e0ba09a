"""FP64 CPU oracle of the two-scale FEM time step -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never does; the
two share no code.  The arithmetic lives in ``tsf_oracle.c`` (plain C99 +
OpenMP, FP64); this module is a ctypes wrapper around it plus

* ``monolithic.py``: the same implicit Euler step solved as ONE dense linear
  system (LAPACK via NumPy), the second, independent route to the coupled
  fixed point (tiny meshes only);
* ``norms.py``: L2 / H1 error norms on both scales for the manufactured
  solution check (Sec. 4.2).

Which paper passage each C function follows is stated beside it in
``tsf_oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tsf_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libtsf_oracle.so")

OR_OK, OR_E_ARG, OR_E_BAD_JACOBIAN, OR_E_NOT_CONVERGED, OR_E_BREAKDOWN, OR_E_OOM = 0, 1, 3, 4, 5, 7

FAMILY = {"identity": 0, "bump": 1, "shear_bump": 2, "affine": 3, "affine_bump": 4}
NPARAM = {0: 0, 1: 1, 2: 2, 3: 6, 4: 5}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP, no -ffast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c99", "-fopenmp", "-fPIC", "-shared", "-Wall", "-Wno-unknown-pragmas",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Stats(ctypes.Structure):
    _fields_ = [("inner_iters", ctypes.c_int64), ("micro_solves", ctypes.c_int64),
                ("macro_iters", ctypes.c_int64), ("coupling_iters_last", ctypes.c_int),
                ("coupling_iters_total", ctypes.c_int), ("max_inner_iters", ctypes.c_int),
                ("status", ctypes.c_int), ("coupling_change", ctypes.c_double),
                ("paper_residual", ctypes.c_double)]


_lib = None
_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        vp = ctypes.c_void_p
        L.or_create.restype = vp
        L.or_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D,
                                ctypes.c_double, ctypes.c_double, _I]
        L.or_destroy.argtypes = [vp]
        L.or_set_state.argtypes = [vp, _D, _D]
        L.or_set_sources.argtypes = [vp, _D, _D, _D, _D]
        L.or_step.argtypes = [vp, ctypes.c_double, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                              ctypes.c_double, ctypes.c_int, ctypes.c_double]
        for f in ("or_get_u", "or_get_v", "or_get_vbar", "or_get_flux", "or_get_r"):
            getattr(L, f).argtypes = [vp, _D]
        L.or_get_geometry.argtypes = [vp, _D, _D, _D]
        L.or_nnz_micro.argtypes = [vp]
        L.or_nnz_macro.argtypes = [vp]
        L.or_get_micro_csr.argtypes = [vp, ctypes.c_int, ctypes.c_int, _I, _I, _D]
        L.or_get_macro_csr.argtypes = [vp, ctypes.c_int, _I, _I, _D]
        L.or_get_stats.argtypes = [vp, ctypes.POINTER(_Stats)]
        L.or_reset_stats.argtypes = [vp]
        L.or_chi.argtypes = [ctypes.c_int, _D, ctypes.c_double, ctypes.c_double, _D, _D]
        L.or_chi_many.argtypes = [ctypes.c_int, _D, ctypes.c_int, _D, _D, _D, _D]
        L.or_dchi.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, _D]
        L.or_assemble_q1_dparam.argtypes = [ctypes.c_int, ctypes.c_int, _D, ctypes.c_int, _D, _I, _I, _D, _D, _D]
        L.or_assemble_q1.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D, _I, _I, _D, _D, _D]
        L.or_pullback.argtypes = [_D, _D, _D, _D, _D, _D]
        L.or_unit_normal.argtypes = [_D, _D, _D]
        L.or_pcg.argtypes = [ctypes.c_int, _I, _I, _D, _D, _D, ctypes.c_double, ctypes.c_int, _D, _I, _D]
        L.or_q1_pattern.argtypes = [ctypes.c_int, _I, _I]
        L.or_q1_nnz.argtypes = [ctypes.c_int]
        L.or_num_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(_D) if a is not None else None


def _ip(a):
    return a.ctypes.data_as(_I)


def _f64(a, n=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if n is not None and a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a


def num_threads() -> int:
    return lib().or_num_threads()


# --------------------------------------------------------------------------
# point-wise geometry (Sec. 3.1, Eqs. (13), (14), (16))
# --------------------------------------------------------------------------
def chi(family: int, prm, y1: float, y2: float):
    """chi(yhat) and its Jacobian F (row-major 2x2) for one deformation."""
    p = _f64(prm if len(np.atleast_1d(prm)) else [0.0])
    c = np.zeros(2)
    F = np.zeros(4)
    e = lib().or_chi(int(family), _dp(p), float(y1), float(y2), _dp(c), _dp(F))
    if e:
        raise ValueError("unknown family")
    return c, F.reshape(2, 2)


def chi_many(family: int, prm, y1, y2):
    """chi [n, 2] and F [n, 2, 2] of one deformation at many reference points."""
    p = _f64(prm if len(np.atleast_1d(prm)) else [0.0])
    a1 = _f64(np.ravel(y1))
    a2 = _f64(np.ravel(y2))
    n = a1.size
    c = np.zeros(2 * n)
    F = np.zeros(4 * n)
    e = lib().or_chi_many(int(family), _dp(p), n, _dp(a1), _dp(a2), _dp(c), _dp(F))
    if e:
        raise ValueError("unknown family")
    return c.reshape(n, 2), F.reshape(n, 2, 2)


def pullback(F, D=(1.0, 0.0, 1.0), nu=(1.0, 0.0)):
    """(J, C = J F^-1 D F^-T as (C11, C12, C22), s = |cof(F) nu|)."""
    Fa = _f64(np.asarray(F).reshape(4))
    Da = _f64(D, 3)
    na = _f64(nu, 2)
    J = np.zeros(1)
    C = np.zeros(3)
    s = np.zeros(1)
    lib().or_pullback(_dp(Fa), _dp(Da), _dp(na), _dp(J), _dp(C), _dp(s))
    return float(J[0]), C, float(s[0])


def unit_normal(F, nu):
    Fa = _f64(np.asarray(F).reshape(4))
    na = _f64(nu, 2)
    out = np.zeros(2)
    lib().or_unit_normal(_dp(Fa), _dp(na), _dp(out))
    return out


def pcg(A, b, x0=None, tol=1e-12, maxit=10000):
    """Jacobi-PCG of the oracle on a scipy CSR matrix (for pinning the solver)."""
    A = A.tocsr()
    A.sort_indices()
    n = A.shape[0]
    rp = np.ascontiguousarray(A.indptr, dtype=np.int32)
    ci = np.ascontiguousarray(A.indices, dtype=np.int32)
    val = _f64(A.data)
    bb = _f64(b, n)
    x = _f64(np.zeros(n) if x0 is None else x0, n).copy()
    work = np.zeros(4 * n)
    it = np.zeros(1, dtype=np.int32)
    rr = np.zeros(1)
    e = lib().or_pcg(n, _ip(rp), _ip(ci), _dp(val), _dp(bb), _dp(x), float(tol), int(maxit), _dp(work),
                     _ip(it), _dp(rr))
    return x, int(it[0]), float(rr[0]), e


def assemble_q1(N, family, prm, D=(1.0, 0.0, 1.0)):
    """(M, A, R) of one micro problem as scipy CSR matrices (Eq. (17) micro block)."""
    import scipy.sparse as sp
    rp, ci = q1_pattern(N)
    nnz = len(ci)
    p = _f64(prm if len(np.atleast_1d(prm)) else [0.0])
    out = [np.zeros(nnz) for _ in range(3)]
    e = lib().or_assemble_q1(int(N), int(family), _dp(p), _dp(_f64(D, 3)), _ip(rp), _ip(ci), *[_dp(o) for o in out])
    if e:
        raise OracleError(e, "assembly failed")
    n = (N + 1) ** 2
    return tuple(sp.csr_matrix((o, ci, rp), shape=(n, n)) for o in out)


def assemble_q1_dparam(N, family, prm, k, D=(1.0, 0.0, 1.0)):
    """(dM, dA, dR): derivatives of (M, A, R) with respect to parameter k."""
    import scipy.sparse as sp
    rp, ci = q1_pattern(N)
    nnz = len(ci)
    p = _f64(prm if len(np.atleast_1d(prm)) else [0.0])
    out = [np.zeros(nnz) for _ in range(3)]
    e = lib().or_assemble_q1_dparam(int(N), int(family), _dp(p), int(k), _dp(_f64(D, 3)), _ip(rp), _ip(ci),
                                    *[_dp(o) for o in out])
    if e:
        raise OracleError(e, "derivative assembly failed")
    n = (N + 1) ** 2
    return tuple(sp.csr_matrix((o, ci, rp), shape=(n, n)) for o in out)


def q1_pattern(N: int):
    n = (N + 1) ** 2
    nnz = lib().or_q1_nnz(N)
    rp = np.zeros(n + 1, dtype=np.int32)
    ci = np.zeros(nnz, dtype=np.int32)
    lib().or_q1_pattern(N, _ip(rp), _ip(ci))
    return rp, ci


class OracleError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{msg} (oracle status {code})")
        self.code = code


class Problem:
    """One two-scale problem held by the C oracle.

    Nm / NM: micro / macro cells per side; bc: 0 Neumann, 1 Dirichlet on the
    whole macro boundary; family: deformation family (see ``FAMILY``);
    params: [n_M, nparam] per-node deformation parameters; D: micro diffusion
    (D11, D12, D22); kappa: Robin transfer coefficient; Du: macro diffusion.
    """

    def __init__(self, Nm, NM, bc, family, params, D=(1.0, 0.0, 1.0), kappa=1.0, Du=1.0):
        self.Nm, self.NM = int(Nm), int(NM)
        self.nm, self.nM = (self.Nm + 1) ** 2, (self.NM + 1) ** 2
        self.family = int(family)
        npar = NPARAM[self.family]
        prm = _f64(params if npar else np.zeros(1), self.nM * npar if npar else 1)
        Da = _f64(D, 3)
        err = ctypes.c_int(0)
        h = lib().or_create(self.Nm, self.NM, int(bc), self.family, _dp(prm), _dp(Da), float(kappa),
                            float(Du), ctypes.byref(err))
        if not h:
            raise OracleError(err.value, "oracle problem creation failed")
        self._h = h
        self.kappa = float(kappa)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().or_destroy(h)
            self._h = None

    def set_state(self, u, v=None):
        ua = _f64(u, self.nM)
        va = None if v is None else _f64(v, self.nM * self.nm)
        lib().or_set_state(self._h, _dp(ua), _dp(va))

    def set_sources(self, fv=None, g=None, fu=None, ud=None):
        args = [None if a is None else _f64(a, n) for a, n in
                ((fv, self.nM * self.nm), (g, self.nM * (self.Nm + 1)), (fu, self.nM), (ud, self.nM))]
        e = lib().or_set_sources(self._h, *[_dp(a) for a in args])
        if e:
            raise OracleError(e, "set_sources failed")

    def step(self, dt, nsteps=1, cg_tol=1e-12, cg_maxit=20000, coupling_tol=1e-12, coupling_maxit=50,
             macro_tol=None, check=True):
        mt = cg_tol if macro_tol is None else macro_tol
        e = lib().or_step(self._h, float(dt), int(nsteps), float(cg_tol), int(cg_maxit), float(coupling_tol),
                          int(coupling_maxit), float(mt))
        if e and check:
            raise OracleError(e, "oracle step failed")
        return e

    @property
    def u(self):
        out = np.zeros(self.nM)
        lib().or_get_u(self._h, _dp(out))
        return out

    @property
    def v(self):
        out = np.zeros(self.nM * self.nm)
        lib().or_get_v(self._h, _dp(out))
        return out.reshape(self.nM, self.nm)

    @property
    def vbar(self):
        out = np.zeros(self.nM)
        lib().or_get_vbar(self._h, _dp(out))
        return out

    @property
    def flux(self):
        out = np.zeros(self.nM)
        lib().or_get_flux(self._h, _dp(out))
        return out

    @property
    def r(self):
        out = np.zeros(self.nM * self.nm)
        lib().or_get_r(self._h, _dp(out))
        return out.reshape(self.nM, self.nm)

    def geometry(self):
        gam, vol, mH = np.zeros(self.nM), np.zeros(self.nM), np.zeros(self.nM)
        lib().or_get_geometry(self._h, _dp(gam), _dp(vol), _dp(mH))
        return gam, vol, mH

    def micro_csr(self, i, which):
        """which: 'M', 'A' or 'R' of instance i as a scipy CSR matrix."""
        import scipy.sparse as sp
        nnz = lib().or_nnz_micro(self._h)
        rp = np.zeros(self.nm + 1, dtype=np.int32)
        ci = np.zeros(nnz, dtype=np.int32)
        val = np.zeros(nnz)
        lib().or_get_micro_csr(self._h, int(i), {"M": 0, "A": 1, "R": 2}[which], _ip(rp), _ip(ci), _dp(val))
        return sp.csr_matrix((val, ci, rp), shape=(self.nm, self.nm))

    def macro_csr(self, which):
        """which: 'M' (M_H) or 'K' (K_H)."""
        import scipy.sparse as sp
        nnz = lib().or_nnz_macro(self._h)
        rp = np.zeros(self.nM + 1, dtype=np.int32)
        ci = np.zeros(nnz, dtype=np.int32)
        val = np.zeros(nnz)
        lib().or_get_macro_csr(self._h, {"M": 0, "K": 1}[which], _ip(rp), _ip(ci), _dp(val))
        return sp.csr_matrix((val, ci, rp), shape=(self.nM, self.nM))

    def stats(self):
        s = _Stats()
        lib().or_get_stats(self._h, ctypes.byref(s))
        return {k: getattr(s, k) for k, _ in _Stats._fields_}

    def reset_stats(self):
        lib().or_reset_stats(self._h)
