"""ctypes binding of ``libtsfem`` (include/tsfem.h, include/tsfem3.h), argument marshalling only.

Every C entry point has a Python function of the same name.  Array arguments
may be NumPy arrays (host memory) or CUDA ``torch.Tensor`` s (device memory,
passed by ``data_ptr()``); the ``on_device`` flag is derived from the array.
A non-OK status raises :class:`TsfError` with the library's error text.
All arithmetic runs in the CUDA library: if ``libtsfem.so`` is missing this
module raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libtsfem.so")

TSF_OK, TSF_E_ARG, TSF_E_STATE, TSF_E_BAD_JACOBIAN, TSF_E_NOT_CONVERGED = 0, 1, 2, 3, 4
TSF_E_NAN, TSF_E_CUDA, TSF_E_OOM, TSF_E_BREAKDOWN, TSF_E_TIMEOUT = 5, 6, 7, 8, 9
TSF_FP64, TSF_MIXED = 0, 1
TSF_FAMILY_IDENTITY, TSF_FAMILY_BUMP, TSF_FAMILY_SHEAR_BUMP, TSF_FAMILY_AFFINE, TSF_FAMILY_AFFINE_BUMP = 0, 1, 2, 3, 4
TSF_BC_NEUMANN, TSF_BC_DIRICHLET = 0, 1
TSF_COUPLING_PARTITIONED, TSF_COUPLING_ELIMINATION = 0, 1
STATUS_NAMES = {0: "TSF_OK", 1: "TSF_E_ARG", 2: "TSF_E_STATE", 3: "TSF_E_BAD_JACOBIAN", 4: "TSF_E_NOT_CONVERGED",
                5: "TSF_E_NAN", 6: "TSF_E_CUDA", 7: "TSF_E_OOM", 8: "TSF_E_BREAKDOWN", 9: "TSF_E_TIMEOUT"}

# every symbol include/tsfem.h declares
EXPORTS = ["tsf_default_options", "tsf_create", "tsf_set_options", "tsf_set_micro_mesh", "tsf_set_macro_mesh",
           "tsf_set_physics", "tsf_set_deformation", "tsf_set_state", "tsf_set_sources", "tsf_step",
           "tsf_synchronize", "tsf_get_macro", "tsf_get_micro_averages", "tsf_get_macro_async",
           "tsf_get_micro_averages_async", "tsf_get_micro_field", "tsf_get_flux", "tsf_get_rho", "tsf_get_geometry", "tsf_get_pushforward", "tsf_get_stats", "tsf_reset_stats", "tsf_workspace_bytes", "tsf_bind_workspace",
           "tsf_last_error", "tsf_destroy", "tsf_version", "tsf_macro_solve_noalloc", "tsf_adjoint_mean_u",
           "tsf_batch_create", "tsf_batch_instance", "tsf_batch_step", "tsf_batch_set_persistent",
           "tsf_batch_persistent_launches", "tsf_batch_synchronize",
           "tsf_batch_get_stats", "tsf_batch_reset_stats", "tsf_batch_last_error", "tsf_batch_destroy"]
# every symbol include/tsfem3.h declares (the stationary three-field system)
EXPORTS3 = ["tsf3_create", "tsf3_set_meshes", "tsf3_set_physics", "tsf3_set_deformation", "tsf3_set_sources",
            "tsf3_solve", "tsf3_get_fields", "tsf3_get_pushforward", "tsf3_get_stats", "tsf3_last_error",
            "tsf3_destroy"]
TSF3_EDGE_BOTTOM, TSF3_EDGE_RIGHT, TSF3_EDGE_TOP, TSF3_EDGE_LEFT = 1, 2, 4, 8
TSF3_TILING_DIRECT = 10
TSF_NOALLOC_MAX_NM = 128
TSF_BATCH_MAX = 4096


class tsf_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("cg_tol", ctypes.c_double), ("inner_tol", ctypes.c_double),
                ("macro_tol", ctypes.c_double), ("coupling_tol", ctypes.c_double), ("cg_maxit", ctypes.c_int),
                ("max_sweeps", ctypes.c_int), ("macro_maxit", ctypes.c_int), ("coupling_maxit", ctypes.c_int),
                ("tiling", ctypes.c_int), ("use_graph", ctypes.c_int), ("cuda_stream", ctypes.c_void_p),
                ("profile", ctypes.c_int), ("coupling", ctypes.c_int)]


class tsf_stats(ctypes.Structure):
    _fields_ = [("inner_iters", ctypes.c_int64), ("dof_cg_iters", ctypes.c_int64), ("refine_sweeps", ctypes.c_int64),
                ("micro_solves", ctypes.c_int64), ("macro_iters", ctypes.c_int64),
                ("coupling_iters_last", ctypes.c_int), ("coupling_iters_total", ctypes.c_int),
                ("max_inner_iters", ctypes.c_int), ("steps", ctypes.c_int), ("status", ctypes.c_int),
                ("tiling", ctypes.c_int), ("coupling_change", ctypes.c_double),
                ("micro_launches", ctypes.c_int64), ("macro_launches", ctypes.c_int64),
                ("micro_kernel_ms", ctypes.c_double), ("macro_kernel_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class tsf3_stats(ctypes.Structure):
    _fields_ = [("inner_iters", ctypes.c_int64), ("dof_cg_iters", ctypes.c_int64), ("refine_sweeps", ctypes.c_int64),
                ("micro_solves", ctypes.c_int64), ("macro_iters", ctypes.c_int64), ("status", ctypes.c_int),
                ("tiling", ctypes.c_int), ("micro_ms", ctypes.c_double), ("macro_ms", ctypes.c_double),
                ("total_ms", ctypes.c_double), ("factor_ms", ctypes.c_double), ("band_solve_ms", ctypes.c_double),
                ("band_launches", ctypes.c_int), ("band_rhs", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class TsfError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libtsfem.so (built by ``paper_2103_17040_gb300.build``); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} not found: build the CUDA library first "
                           "(python -m paper_2103_17040_gb300.build or __graft_entry__.build())")
    L = ctypes.CDLL(path)
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    pp = ctypes.POINTER(ctypes.c_void_p)
    L.tsf_default_options.argtypes = [ctypes.POINTER(tsf_options)]
    L.tsf_default_options.restype = None
    L.tsf_create.argtypes = [pp, ctypes.POINTER(tsf_options)]
    L.tsf_set_options.argtypes = [vp, ctypes.POINTER(tsf_options)]
    L.tsf_set_micro_mesh.argtypes = [vp, i, i, i]
    L.tsf_set_macro_mesh.argtypes = [vp, i, i, i, vp]
    L.tsf_set_physics.argtypes = [vp, vp, d, d]
    L.tsf_set_deformation.argtypes = [vp, i, i, vp, i]
    L.tsf_set_state.argtypes = [vp, vp, vp, i]
    L.tsf_set_sources.argtypes = [vp, vp, vp, vp, vp, i]
    L.tsf_step.argtypes = [vp, d, i]
    L.tsf_synchronize.argtypes = [vp]
    for f in ("tsf_get_macro", "tsf_get_micro_averages", "tsf_get_micro_field", "tsf_get_flux", "tsf_get_rho",
              "tsf_get_macro_async", "tsf_get_micro_averages_async"):
        getattr(L, f).argtypes = [vp, vp, i]
    L.tsf_get_geometry.argtypes = [vp, vp, vp, i]
    L.tsf_get_pushforward.argtypes = [vp, ctypes.c_float, vp, i]
    L.tsf_get_stats.argtypes = [vp, ctypes.POINTER(tsf_stats)]
    L.tsf_reset_stats.argtypes = [vp]
    L.tsf_workspace_bytes.argtypes = [vp, ctypes.POINTER(ctypes.c_size_t)]
    L.tsf_bind_workspace.argtypes = [vp, vp, ctypes.c_size_t]
    L.tsf_last_error.argtypes = [vp]
    L.tsf_last_error.restype = ctypes.c_char_p
    L.tsf_destroy.argtypes = [vp]
    L.tsf_destroy.restype = None
    L.tsf_version.argtypes = []
    L.tsf_macro_solve_noalloc.argtypes = [i, i, d, d, d, vp, vp, vp, vp, vp, d, i, vp, ctypes.POINTER(ctypes.c_int)]
    L.tsf_adjoint_mean_u.argtypes = [vp, d, i, i, vp, vp, i]
    L.tsf_batch_create.argtypes = [pp, i, ctypes.POINTER(tsf_options)]
    L.tsf_batch_instance.argtypes = [vp, i, pp]
    L.tsf_batch_step.argtypes = [vp, d, i]
    L.tsf_batch_set_persistent.argtypes = [vp, i]
    L.tsf_batch_persistent_launches.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
    L.tsf_batch_synchronize.argtypes = [vp]
    L.tsf_batch_get_stats.argtypes = [vp, ctypes.POINTER(tsf_stats)]
    L.tsf_batch_reset_stats.argtypes = [vp]
    L.tsf_batch_last_error.argtypes = [vp]
    L.tsf_batch_last_error.restype = ctypes.c_char_p
    L.tsf_batch_destroy.argtypes = [vp]
    L.tsf_batch_destroy.restype = None
    L.tsf3_create.argtypes = [pp, ctypes.POINTER(tsf_options)]
    L.tsf3_set_meshes.argtypes = [vp, i, i, d, d, i]
    L.tsf3_set_physics.argtypes = [vp, vp, d, vp]
    L.tsf3_set_deformation.argtypes = [vp, i, i, vp, i]
    L.tsf3_set_sources.argtypes = [vp] + [vp] * 9 + [i]
    L.tsf3_solve.argtypes = [vp]
    L.tsf3_get_fields.argtypes = [vp, vp, vp, vp, vp, i]
    L.tsf3_get_pushforward.argtypes = [vp, ctypes.c_float, vp, i]
    L.tsf3_get_stats.argtypes = [vp, ctypes.POINTER(tsf3_stats)]
    L.tsf3_last_error.argtypes = [vp]
    L.tsf3_last_error.restype = ctypes.c_char_p
    L.tsf3_destroy.argtypes = [vp]
    L.tsf3_destroy.restype = None
    for f in EXPORTS + EXPORTS3:
        fn = getattr(L, f)
        if f not in ("tsf_default_options", "tsf_last_error", "tsf_destroy", "tsf_batch_last_error",
                     "tsf_batch_destroy", "tsf3_last_error", "tsf3_destroy"):
            fn.restype = ctypes.c_int
    _lib = L
    return L


def _check(ctx, status):
    if status != TSF_OK:
        msg = _lib.tsf_last_error(ctx).decode() if ctx else ""
        raise TsfError(status, msg)


def _is_cuda_tensor(a):
    return hasattr(a, "is_cuda") and hasattr(a, "data_ptr") and a.is_cuda


def _ptr_in(a, n=None, dtype=np.float64):
    """(pointer, on_device, keepalive) for an input array; None -> NULL."""
    if a is None:
        return None, 0, None
    if _is_cuda_tensor(a):
        import torch
        t = a.contiguous()
        if t.dtype != torch.float64:
            t = t.to(torch.float64)
        if n is not None and t.numel() != n:
            raise ValueError(f"expected {n} values, got {t.numel()}")
        return t.data_ptr(), 1, t
    h = np.ascontiguousarray(np.asarray(a, dtype=dtype))
    if n is not None and h.size != n:
        raise ValueError(f"expected {n} values, got {h.size}")
    return h.ctypes.data, 0, h


def _out(out, n):
    """(pointer, on_device, array) for an output; None -> new host array."""
    if out is None:
        out = np.empty(n, dtype=np.float64)
    if _is_cuda_tensor(out):
        if out.numel() != n or not out.is_contiguous():
            raise ValueError("output tensor must be contiguous with the right size")
        return out.data_ptr(), 1, out
    if out.dtype != np.float64 or out.size != n or not out.flags.c_contiguous:
        raise ValueError("output array must be contiguous float64 with the right size")
    return out.ctypes.data, 0, out


# ---------------------------------------------------------------------------
# functions with the C names
# ---------------------------------------------------------------------------
def tsf_version() -> int:
    return load_library().tsf_version()


def tsf_default_options() -> tsf_options:
    o = tsf_options()
    load_library().tsf_default_options(ctypes.byref(o))
    return o


def tsf_create(opt: tsf_options | None = None) -> int:
    L = load_library()
    h = ctypes.c_void_p()
    st = L.tsf_create(ctypes.byref(h), ctypes.byref(opt) if opt is not None else None)
    if st != TSF_OK:
        raise TsfError(st, "tsf_create failed (no CUDA device?)")
    return h.value


def tsf_set_options(ctx, opt: tsf_options):
    _check(ctx, _lib.tsf_set_options(ctx, ctypes.byref(opt)))


def tsf_set_micro_mesh(ctx, nx, ny, robin_edge=0):
    _check(ctx, _lib.tsf_set_micro_mesh(ctx, int(nx), int(ny), int(robin_edge)))


def tsf_set_macro_mesh(ctx, nx, ny, bc=TSF_BC_NEUMANN, dirichlet_vals=None):
    h = None if dirichlet_vals is None else np.ascontiguousarray(np.asarray(dirichlet_vals, np.float64))
    _check(ctx, _lib.tsf_set_macro_mesh(ctx, int(nx), int(ny), int(bc), None if h is None else h.ctypes.data))


def tsf_set_physics(ctx, D=(1.0, 0.0, 1.0), kappa=1.0, macro_diff=1.0):
    Da = np.ascontiguousarray(np.asarray(D, np.float64))
    _check(ctx, _lib.tsf_set_physics(ctx, Da.ctypes.data, float(kappa), float(macro_diff)))


def tsf_set_deformation(ctx, family, nparam, params):
    p, dev, keep = _ptr_in(params) if nparam else (None, 0, None)
    _check(ctx, _lib.tsf_set_deformation(ctx, int(family), int(nparam), p, dev))


def tsf_set_state(ctx, u, v=None):
    pu, du, ku = _ptr_in(u)
    pv, dv, kv = _ptr_in(v)
    if v is not None and du != dv:
        raise ValueError("u and v must both be host arrays or both device tensors")
    _check(ctx, _lib.tsf_set_state(ctx, pu, pv, du))


def tsf_set_sources(ctx, fv=None, g=None, fu=None, ud=None):
    args = [_ptr_in(a) for a in (fv, g, fu, ud)]
    devs = {a[1] for a, x in zip(args, (fv, g, fu, ud)) if x is not None}
    if len(devs) > 1:
        raise ValueError("sources must all live on the host or all on the device")
    _check(ctx, _lib.tsf_set_sources(ctx, *[a[0] for a in args], devs.pop() if devs else 0))


def tsf_step(ctx, dt, nsteps=1):
    _check(ctx, _lib.tsf_step(ctx, float(dt), int(nsteps)))


def tsf_synchronize(ctx):
    _check(ctx, _lib.tsf_synchronize(ctx))


def _getter(name, ctx, n, out):
    p, dev, arr = _out(out, n)
    _check(ctx, getattr(_lib, name)(ctx, p, dev))
    return arr


def tsf_get_macro(ctx, nM, out=None):
    return _getter("tsf_get_macro", ctx, nM, out)


def tsf_get_micro_averages(ctx, nM, out=None):
    return _getter("tsf_get_micro_averages", ctx, nM, out)


def tsf_get_macro_async(ctx, nM, out):
    """Enqueue the copy of u into out (page-locked host array or CUDA tensor of nM
    doubles) without synchronising; out holds u once the stream reaches the copy."""
    ptr, dev, _ = _out(out, nM)
    _check(ctx, _lib.tsf_get_macro_async(ctx, ptr, dev))
    return out


def tsf_get_micro_averages_async(ctx, nM, out):
    """As tsf_get_macro_async, for the micro averages."""
    ptr, dev, _ = _out(out, nM)
    _check(ctx, _lib.tsf_get_micro_averages_async(ctx, ptr, dev))
    return out


def tsf_get_micro_field(ctx, n, out=None):
    return _getter("tsf_get_micro_field", ctx, n, out)


def tsf_get_flux(ctx, nM, out=None):
    return _getter("tsf_get_flux", ctx, nM, out)


def tsf_get_rho(ctx, nM, out=None):
    return _getter("tsf_get_rho", ctx, nM, out)


def tsf_get_geometry(ctx, nM):
    g = np.empty(nM)
    v = np.empty(nM)
    _check(ctx, _lib.tsf_get_geometry(ctx, g.ctypes.data, v.ctypes.data, 0))
    return g, v


def tsf_get_pushforward(ctx, nM, nm, scale, out=None):
    """(X1, X2, v) of every micro node at its macroscopic location: [nM * nm * 3]
    float32 (a NumPy array, or a float32 CUDA tensor given as out)."""
    n = nM * nm * 3
    if out is None:
        out = np.empty(n, dtype=np.float32)
    if _is_cuda_tensor(out):
        import torch
        if out.dtype != torch.float32 or out.numel() != n or not out.is_contiguous():
            raise ValueError("output tensor must be contiguous float32 with the right size")
        p, dev = out.data_ptr(), 1
    else:
        if out.dtype != np.float32 or out.size != n or not out.flags.c_contiguous:
            raise ValueError("output array must be contiguous float32 with the right size")
        p, dev = out.ctypes.data, 0
    _check(ctx, _lib.tsf_get_pushforward(ctx, float(scale), p, dev))
    return out


def tsf_get_stats(ctx) -> dict:
    s = tsf_stats()
    _check(ctx, _lib.tsf_get_stats(ctx, ctypes.byref(s)))
    return s.as_dict()


def tsf_reset_stats(ctx):
    _check(ctx, _lib.tsf_reset_stats(ctx))


def _bcheck(b, status):
    if status != TSF_OK:
        raise TsfError(status, _lib.tsf_batch_last_error(b).decode() if b else "")


def tsf_batch_create(ninst, opt: tsf_options | None = None) -> int:
    L = load_library()
    h = ctypes.c_void_p()
    st = L.tsf_batch_create(ctypes.byref(h), int(ninst), ctypes.byref(opt) if opt is not None else None)
    if st != TSF_OK:
        raise TsfError(st, "tsf_batch_create failed")
    return h.value


def tsf_batch_instance(b, inst) -> int:
    h = ctypes.c_void_p()
    _bcheck(b, _lib.tsf_batch_instance(b, int(inst), ctypes.byref(h)))
    return h.value


def tsf_batch_step(b, dt, nsteps=1):
    _bcheck(b, _lib.tsf_batch_step(b, float(dt), int(nsteps)))


def tsf_batch_set_persistent(b, on):
    _bcheck(b, _lib.tsf_batch_set_persistent(b, int(on)))


def tsf_batch_persistent_launches(b) -> int:
    n = ctypes.c_int()
    _bcheck(b, _lib.tsf_batch_persistent_launches(b, ctypes.byref(n)))
    return n.value


def tsf_batch_synchronize(b):
    _bcheck(b, _lib.tsf_batch_synchronize(b))


def tsf_batch_get_stats(b) -> dict:
    s = tsf_stats()
    _bcheck(b, _lib.tsf_batch_get_stats(b, ctypes.byref(s)))
    return s.as_dict()


def tsf_batch_reset_stats(b):
    _bcheck(b, _lib.tsf_batch_reset_stats(b))


def tsf_batch_last_error(b) -> str:
    return _lib.tsf_batch_last_error(b).decode()


def tsf_batch_destroy(b):
    if b:
        _lib.tsf_batch_destroy(b)


def tsf_adjoint_mean_u(ctx, dt, nsteps, ckpt_every, nM, nparam, grad_out=None):
    """(J, grad [nM * nparam]) of the mean macro concentration after the march."""
    p, dev, g = _out(grad_out, nM * nparam) if nparam else (None, 0, np.zeros(0))
    J = np.zeros(1)
    if dev:
        import torch
        Jt = torch.zeros(1, dtype=torch.float64, device="cuda")
        _check(ctx, _lib.tsf_adjoint_mean_u(ctx, float(dt), int(nsteps), int(ckpt_every), Jt.data_ptr(), p, 1))
        return float(Jt.item()), g
    _check(ctx, _lib.tsf_adjoint_mean_u(ctx, float(dt), int(nsteps), int(ckpt_every), J.ctypes.data, p, 0))
    return float(J[0]), g


def tsf_workspace_bytes(ctx) -> int:
    n = ctypes.c_size_t()
    _check(ctx, _lib.tsf_workspace_bytes(ctx, ctypes.byref(n)))
    return n.value


def tsf_bind_workspace(ctx, ptr, nbytes):
    _check(ctx, _lib.tsf_bind_workspace(ctx, ptr, int(nbytes)))


def tsf_last_error(ctx) -> str:
    return _lib.tsf_last_error(ctx).decode()


def tsf_destroy(ctx):
    if ctx and _lib is not None:
        _lib.tsf_destroy(ctx)


def tsf_macro_solve_noalloc(NM, bc, dt, macro_diff, kappa, gam, cH, rho, u0, u_out, tol=1e-12, maxit=500,
                            stream=None):
    """Macro solve for callers that cannot allocate device memory.

    All arrays are CUDA tensors of (NM+1)^2 float64 values; the library uses a
    fixed scratch array of its own instead of allocating.  Returns the PCG
    iteration count; a non-OK status raises TsfError (there is no context, so
    the message is the status name only).

    The call runs on the current CUDA device, so every tensor must live on
    that device (a pointer into another GPU's memory is not reachable from the
    kernel).  stream: a torch.cuda.Stream or a raw cudaStream_t handle; None
    means torch's current stream, so the solve is ordered after the work that
    produced the inputs.  The call waits for the solve to finish before it
    returns."""
    import torch
    L = load_library()
    arrs = (gam, cH, rho, u0, u_out)
    n = (int(NM) + 1) ** 2
    dev = torch.cuda.current_device()
    for a in arrs:
        if not (_is_cuda_tensor(a) and a.dtype.is_floating_point and a.element_size() == 8 and a.is_contiguous()
                and a.numel() == n):
            raise ValueError(f"expected contiguous float64 CUDA tensors of {n} values")
        if a.device.index != dev:
            raise ValueError(f"tensor on cuda:{a.device.index}, but the current device is cuda:{dev}")
    if stream is None:
        s = torch.cuda.current_stream().cuda_stream
    else:
        s = stream if isinstance(stream, int) else stream.cuda_stream
    it = ctypes.c_int(0)
    st = L.tsf_macro_solve_noalloc(int(NM), int(bc), float(dt), float(macro_diff), float(kappa),
                                   *[a.data_ptr() for a in arrs], float(tol), int(maxit), s or None,
                                   ctypes.byref(it))
    if st != TSF_OK:
        raise TsfError(st, "tsf_macro_solve_noalloc failed")
    return it.value


# ---------------------------------------------------------------------------
# stationary three-field system (include/tsfem3.h)
# ---------------------------------------------------------------------------
def _check3(ctx, status):
    if status != TSF_OK:
        msg = _lib.tsf3_last_error(ctx).decode() if ctx else ""
        raise TsfError(status, msg)


def tsf3_create(opt: tsf_options | None = None) -> int:
    L = load_library()
    out = ctypes.c_void_p()
    st = L.tsf3_create(ctypes.byref(out), ctypes.byref(opt) if opt is not None else None)
    if st != TSF_OK:
        raise TsfError(st, "tsf3_create failed")
    return out.value


def tsf3_set_meshes(ctx, Nm, NM, x0=0.0, L=1.0, dir_mask=TSF3_EDGE_LEFT):
    _check3(ctx, _lib.tsf3_set_meshes(ctx, int(Nm), int(NM), float(x0), float(L), int(dir_mask)))


def tsf3_set_physics(ctx, D=(1.0, 0.0, 1.0), Dw=1.0, kappa=(1.0, 1.0, 1.0, 1.0)):
    Da = (ctypes.c_double * 3)(*[float(x) for x in D])
    ka = (ctypes.c_double * 4)(*[float(x) for x in kappa])
    _check3(ctx, _lib.tsf3_set_physics(ctx, Da, float(Dw), ka))


def tsf3_set_deformation(ctx, family, nparam, params):
    p, dev, keep = _ptr_in(params) if nparam else (None, 0, None)
    _check3(ctx, _lib.tsf3_set_deformation(ctx, int(family), int(nparam), p, dev))


def tsf3_set_sources(ctx, fu=None, fw=None, ud=None, gu=None, gw=None, fv=None, gI=None, gO=None, gN=None):
    args = [_ptr_in(a) for a in (fu, fw, ud, gu, gw, fv, gI, gO, gN)]
    devs = {dev for (ptr, dev, _) in args if ptr is not None}
    if len(devs) > 1:
        raise ValueError("sources must all be host arrays or all CUDA tensors")
    _check3(ctx, _lib.tsf3_set_sources(ctx, *[ptr for (ptr, _, _) in args], devs.pop() if devs else 0))


def tsf3_solve(ctx):
    _check3(ctx, _lib.tsf3_solve(ctx))


def tsf3_get_fields(ctx, nM, nm, u=None, w=None, v=None, vbar=None):
    """(u [nM], w [nM], v [nM*nm], vbar [nM]); outputs None -> new host arrays."""
    outs = [_out(a, n) for a, n in ((u, nM), (w, nM), (v, nM * nm), (vbar, nM))]
    devs = {dev for (_, dev, _) in outs}
    if len(devs) > 1:
        raise ValueError("outputs must all be host arrays or all CUDA tensors")
    _check3(ctx, _lib.tsf3_get_fields(ctx, *[ptr for (ptr, _, _) in outs], devs.pop()))
    return tuple(a for (_, _, a) in outs)


def tsf3_get_pushforward(ctx, nM, nm, scale, out=None):
    """[nM * nm * 3] FP32 (X1, X2, v); out None -> new host array."""
    n = nM * nm * 3
    if out is None:
        out = np.empty(n, dtype=np.float32)
    if _is_cuda_tensor(out):
        import torch
        if out.dtype != torch.float32 or out.numel() != n or not out.is_contiguous():
            raise ValueError("output tensor must be contiguous float32 with nM*nm*3 values")
        _check3(ctx, _lib.tsf3_get_pushforward(ctx, float(scale), out.data_ptr(), 1))
        return out
    if out.dtype != np.float32 or out.size != n or not out.flags.c_contiguous:
        raise ValueError("output array must be contiguous float32 with nM*nm*3 values")
    _check3(ctx, _lib.tsf3_get_pushforward(ctx, float(scale), out.ctypes.data, 0))
    return out


def tsf3_get_stats(ctx) -> dict:
    s = tsf3_stats()
    _check3(ctx, _lib.tsf3_get_stats(ctx, ctypes.byref(s)))
    return s.as_dict()


def tsf3_last_error(ctx) -> str:
    return load_library().tsf3_last_error(ctx).decode()


def tsf3_destroy(ctx):
    if ctx:
        load_library().tsf3_destroy(ctx)


# ---------------------------------------------------------------------------
# convenience wrapper (still marshalling only)
# ---------------------------------------------------------------------------
def _make_options(precision, stream, opts):
    o = tsf_default_options()
    o.precision = int(precision)
    for k, v in opts.items():
        setattr(o, k, v)
    if stream is not None:
        o.cuda_stream = stream if isinstance(stream, int) else stream.cuda_stream
        if not o.cuda_stream:
            raise ValueError("pass a non-default stream (a NULL stream makes the library create its own)")
    return o


class TwoScale:
    """One two-scale problem on the current CUDA device.

    Meshes: Nm x Nm micro cells on the reference cell, NM x NM macro cells.
    ``workspace='torch'`` allocates the library's device workspace through
    PyTorch's caching allocator; ``None`` lets the library allocate it.
    """

    def __init__(self, Nm, NM, bc=TSF_BC_NEUMANN, precision=TSF_MIXED, stream=None, workspace="torch",
                 _instance=None, **opts):
        if _instance is None:
            self.ctx = tsf_create(_make_options(precision, stream, opts))
            self._owned = True
        else:
            self.ctx, self._owned = _instance, False
        self.Nm, self.NM = int(Nm), int(NM)
        self.nm, self.nM = (self.Nm + 1) ** 2, (self.NM + 1) ** 2
        tsf_set_micro_mesh(self.ctx, self.Nm, self.Nm, 0)
        tsf_set_macro_mesh(self.ctx, self.NM, self.NM, bc, None)
        self._ws = None
        if workspace == "torch":
            import torch
            nbytes = tsf_workspace_bytes(self.ctx)
            self._ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
            base = self._ws.data_ptr()
            tsf_bind_workspace(self.ctx, (base + 255) // 256 * 256, nbytes)

    def close(self):
        if getattr(self, "ctx", None):
            if self._owned:
                tsf_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_physics(self, D=(1.0, 0.0, 1.0), kappa=1.0, macro_diff=1.0):
        tsf_set_physics(self.ctx, D, kappa, macro_diff)

    def set_deformation(self, family, params):
        self.family = int(family)
        params = np.zeros((self.nM, 0)) if params is None else params
        nparam = {0: 0, 1: 1, 2: 2, 3: 6, 4: 5}[int(family)]
        tsf_set_deformation(self.ctx, family, nparam, params)

    def set_state(self, u, v=None):
        tsf_set_state(self.ctx, u, v)

    def set_sources(self, fv=None, g=None, fu=None, ud=None):
        tsf_set_sources(self.ctx, fv, g, fu, ud)

    def step(self, dt, nsteps=1):
        tsf_step(self.ctx, dt, nsteps)

    def synchronize(self):
        tsf_synchronize(self.ctx)

    def u(self, out=None):
        return tsf_get_macro(self.ctx, self.nM, out)

    def v(self, out=None):
        a = tsf_get_micro_field(self.ctx, self.nM * self.nm, out)
        return a.reshape(self.nM, self.nm) if isinstance(a, np.ndarray) else a

    def vbar(self, out=None):
        return tsf_get_micro_averages(self.ctx, self.nM, out)

    def u_async(self, out):
        """Queue a copy of u into ``out`` (page-locked host array or CUDA tensor of
        nM doubles); valid after ``synchronize()``."""
        return tsf_get_macro_async(self.ctx, self.nM, out)

    def vbar_async(self, out):
        """Queue the micro averages into ``out`` (as ``u_async``)."""
        return tsf_get_micro_averages_async(self.ctx, self.nM, out)

    def flux(self, out=None):
        return tsf_get_flux(self.ctx, self.nM, out)

    def rho(self, out=None):
        """coupling moments r_i^T v_i (compensated FP64 sums)"""
        return tsf_get_rho(self.ctx, self.nM, out)

    def geometry(self):
        return tsf_get_geometry(self.ctx, self.nM)

    def pushforward(self, scale=None, out=None):
        """Micro fields at their macroscopic locations, [nM, nm, 3] = (X1, X2, v);
        scale defaults to 0.8 of the macro mesh width."""
        a = tsf_get_pushforward(self.ctx, self.nM, self.nm, 0.8 / self.NM if scale is None else scale, out)
        return a.reshape(self.nM, self.nm, 3) if isinstance(a, np.ndarray) else a

    def stats(self):
        return tsf_get_stats(self.ctx)

    def reset_stats(self):
        tsf_reset_stats(self.ctx)

    def adjoint_mean_u(self, dt, nsteps, ckpt_every=10, family=None):
        """(J, dJ/dparams [nM, nparam]) after nsteps from the current state."""
        nparam = {0: 0, 1: 1, 2: 2, 3: 6, 4: 5}[self.family if family is None else family]
        J, g = tsf_adjoint_mean_u(self.ctx, dt, nsteps, ckpt_every, self.nM, nparam)
        return J, np.asarray(g).reshape(self.nM, nparam)


class TwoScaleBatch:
    """Independent two-scale problems advanced together: one CUDA graph launch
    per batch step, one branch per instance.

    ``specs``: sequence of ``(Nm, NM)`` or ``(Nm, NM, bc)``.  ``batch[i]`` is a
    :class:`TwoScale` view of instance i (configure and read it as usual; it
    is valid while the batch lives).  ``persistent=True``: the micro solves of
    all instances run in persistent launches (one per class of micro mesh) fed by work
    queues (tsf_batch_set_persistent).
    """

    def __init__(self, specs, precision=TSF_MIXED, stream=None, workspace="torch", persistent=False, **opts):
        self.b = tsf_batch_create(len(specs), _make_options(precision, stream, opts))
        self.instances = []
        for i, sp in enumerate(specs):
            Nm, NM = int(sp[0]), int(sp[1])
            bc = int(sp[2]) if len(sp) > 2 else TSF_BC_NEUMANN
            self.instances.append(TwoScale(Nm, NM, bc, workspace=workspace,
                                           _instance=tsf_batch_instance(self.b, i)))
        if persistent:
            tsf_batch_set_persistent(self.b, 1)

    def __len__(self):
        return len(self.instances)

    def __getitem__(self, i):
        return self.instances[i]

    def step(self, dt, nsteps=1):
        tsf_batch_step(self.b, dt, nsteps)

    def synchronize(self):
        tsf_batch_synchronize(self.b)

    def stats(self):
        return tsf_batch_get_stats(self.b)

    def persistent_launches(self):
        return tsf_batch_persistent_launches(self.b)

    def reset_stats(self):
        tsf_batch_reset_stats(self.b)

    def close(self):
        if getattr(self, "b", None):
            for p in self.instances:
                p.ctx = None
            tsf_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class ThreeField:
    """The stationary three-field system (u, v, w; include/tsfem3.h) on the
    current CUDA device: Nm x Nm micro cells, NM x NM macro cells on
    [x0, x0 + L]^2, u Dirichlet on the edges of ``dir_mask`` (TSF3_EDGE_*)."""

    def __init__(self, Nm, NM, x0=0.0, L=1.0, dir_mask=TSF3_EDGE_LEFT, precision=TSF_MIXED, stream=None, **opts):
        self.ctx = tsf3_create(_make_options(precision, stream, opts))
        self.Nm, self.NM = int(Nm), int(NM)
        self.nm, self.nM = (self.Nm + 1) ** 2, (self.NM + 1) ** 2
        tsf3_set_meshes(self.ctx, self.Nm, self.NM, x0, L, dir_mask)

    def close(self):
        if getattr(self, "ctx", None):
            tsf3_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_physics(self, D=(1.0, 0.0, 1.0), Dw=1.0, kappa=(1.0, 1.0, 1.0, 1.0)):
        tsf3_set_physics(self.ctx, D, Dw, kappa)

    def set_deformation(self, family, params):
        nparam = {0: 0, 1: 1, 2: 2, 3: 6, 4: 5}[int(family)]
        tsf3_set_deformation(self.ctx, family, nparam, params)

    def set_sources(self, fu=None, fw=None, ud=None, gu=None, gw=None, fv=None, gI=None, gO=None, gN=None):
        tsf3_set_sources(self.ctx, fu, fw, ud, gu, gw, fv, gI, gO, gN)

    def solve(self):
        tsf3_solve(self.ctx)

    def fields(self):
        """(u [nM], w [nM], v [nM, nm], vbar [nM]) as host arrays"""
        u, w, v, vbar = tsf3_get_fields(self.ctx, self.nM, self.nm)
        return u, w, v.reshape(self.nM, self.nm), vbar

    def pushforward(self, scale, out=None):
        """Micro fields at their macroscopic locations, [nM, nm, 3] = (X1, X2, v),
        each cell scaled by ``scale`` and centred on its macro node."""
        a = tsf3_get_pushforward(self.ctx, self.nM, self.nm, scale, out)
        return a.reshape(self.nM, self.nm, 3) if isinstance(a, np.ndarray) else a

    def stats(self):
        return tsf3_get_stats(self.ctx)
