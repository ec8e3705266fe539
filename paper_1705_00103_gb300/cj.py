"""Python binding of libcj (the C ABI declared in include/cj.h), by ctypes.

Argument marshalling only: every step of the solve runs in libcj's CUDA kernels.  Device
grids are torch CUDA tensors (float64, or float32 for the FP32 entry points), 2-D with
shape (Ny, Nx) and unit stride along x; their row stride is passed as ``ld``.  Streams
default to torch's current stream.  If libcj.so has not been built, loading raises: there
is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

CJ_OK, CJ_FLOOR, CJ_PENDING, CJ_STALLED = 0, 1, 2, 3
CJ_ERR_INVALID_ARG, CJ_ERR_NOMEM, CJ_ERR_NOT_CONVERGED = -1, -2, -3
CJ_ERR_DIVERGED, CJ_ERR_TIMEOUT, CJ_ERR_CUDA, CJ_ERR_BUDGET = -4, -5, -6, -7
CJ_ST5, CJ_ST9, CJ_ST17 = 5, 9, 17
CJ_BC_DIRICHLET0, CJ_BC_DIRICHLET = 0, 1
CJ_FP64, CJ_FP32_INNER, CJ_FP32_INNER_DD, CJ_FP64_INNER_DD = 0, 1, 2, 3
CJ_CJM, CJ_JACOBI = 0, 1
CJ_LAUNCH_AUTO, CJ_LAUNCH_STREAM, CJ_LAUNCH_GRAPH, CJ_LAUNCH_CLUSTER = 0, 1, 2, 3


class cj_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("literal_n", ctypes.c_int),
                ("inner_cycle", ctypes.c_int), ("temporal_depth", ctypes.c_int),
                ("max_sweeps", ctypes.c_longlong), ("method", ctypes.c_int), ("launch", ctypes.c_int)]


class cj_mask(ctypes.Structure):
    _fields_ = [("pattern", ctypes.c_int), ("coef", ctypes.c_void_p), ("sx", ctypes.c_longlong),
                ("sy", ctypes.c_longlong), ("sp", ctypes.c_longlong), ("scale", ctypes.c_void_p),
                ("scale_sx", ctypes.c_longlong), ("scale_sy", ctypes.c_longlong),
                ("kmin", ctypes.c_double), ("kmax", ctypes.c_double)]


class cj_result(ctypes.Structure):
    _fields_ = [("sweeps", ctypes.c_longlong), ("cycles", ctypes.c_int), ("status", ctypes.c_int),
                ("rel_res_l2", ctypes.c_double), ("rel_res_inf", ctypes.c_double),
                ("floor_est", ctypes.c_double), ("seconds", ctypes.c_double),
                ("sweep_seconds", ctypes.c_double), ("launches", ctypes.c_longlong)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class cj_problem(ctypes.Structure):
    _fields_ = [("Nx", ctypes.c_int), ("Ny", ctypes.c_int), ("st", ctypes.c_int),
                ("precision", ctypes.c_int), ("tol", ctypes.c_double),
                ("inner_cycle", ctypes.c_int), ("temporal_depth", ctypes.c_int),
                ("max_sweeps", ctypes.c_longlong), ("f", ctypes.c_void_p), ("ld_f", ctypes.c_longlong),
                ("u", ctypes.c_void_p), ("ld_u", ctypes.c_longlong)]


class cj_server_stats_t(ctypes.Structure):
    _fields_ = [("queued", ctypes.c_longlong), ("active", ctypes.c_longlong),
                ("admitted", ctypes.c_longlong), ("completed", ctypes.c_longlong),
                ("steps", ctypes.c_longlong), ("peak_active", ctypes.c_longlong),
                ("bytes_in_use", ctypes.c_size_t), ("peak_bytes", ctypes.c_size_t),
                ("budget_bytes", ctypes.c_size_t)]


class CJError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = "%s: %s (%d)" % (where, cj_status_string(status), status)
        err = _lib().cj_last_error().decode()
        if err:
            msg += " [%s]" % err
        super().__init__(msg)
        self.status = status


_L = None
_vp = ctypes.c_void_p
_ll = ctypes.c_longlong
_dp = ctypes.POINTER(ctypes.c_double)


def library_path() -> str:
    return _build.LIB


def _lib():
    global _L
    if _L is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError("libcj.so is not built (%s); run paper_1705_00103_gb300/build.py "
                               "or __graft_entry__.build() first -- there is no CPU fallback" % path)
        L = ctypes.CDLL(path)
        L.cj_status_string.argtypes = [ctypes.c_int]
        L.cj_status_string.restype = ctypes.c_char_p
        L.cj_last_error.argtypes = []
        L.cj_last_error.restype = ctypes.c_char_p
        L.cj_plan_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_double, ctypes.POINTER(cj_options), ctypes.POINTER(_vp)]
        L.cj_plan_create.restype = ctypes.c_int
        L.cj_plan_create_mask.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(cj_mask), ctypes.c_double,
                                          ctypes.POINTER(cj_options), ctypes.POINTER(_vp)]
        L.cj_plan_create_mask.restype = ctypes.c_int
        L.cj_plan_destroy.argtypes = [_vp]
        L.cj_plan_destroy.restype = None
        L.cj_plan_info.argtypes = [_vp, ctypes.POINTER(_dp), ctypes.POINTER(_ll), _dp, _dp,
                                   ctypes.POINTER(_ll)]
        L.cj_plan_info.restype = ctypes.c_int
        L.cj_solve.argtypes = [_vp, _vp, _ll, _vp, _ll, _vp, ctypes.POINTER(cj_result)]
        L.cj_solve.restype = ctypes.c_int
        L.cj_solve_history.argtypes = [_vp, _vp, _ll, _vp, _ll, _vp, ctypes.POINTER(cj_result),
                                       _dp, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
        L.cj_solve_history.restype = ctypes.c_int
        L.cj_solve_to_error.argtypes = [_vp, _vp, _ll, _vp, _ll, _vp, _ll, ctypes.c_double, _ll, _vp,
                                        ctypes.POINTER(cj_result), _dp, _dp, ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_int)]
        L.cj_solve_to_error.restype = ctypes.c_int
        L.cj_solve_host.argtypes = [_vp, _vp, _vp, _vp, ctypes.POINTER(cj_result)]
        L.cj_solve_host.restype = ctypes.c_int
        L.cj_sweeps.argtypes = [_vp, _vp, _ll, _vp, _ll, _ll, _ll, _vp]
        L.cj_sweeps.restype = ctypes.c_int
        L.cj_sweeps_ff.argtypes = [_vp, _vp, _ll, _vp, _ll, _ll, _ll, _vp]
        L.cj_sweeps_ff.restype = ctypes.c_int
        L.cj_sweeps_f32.argtypes = [_vp, _vp, _ll, _vp, _ll, _ll, _ll, _vp]
        L.cj_sweeps_f32.restype = ctypes.c_int
        L.cj_autotune_engine.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                         ctypes.POINTER(ctypes.c_int), _dp]
        L.cj_autotune_engine.restype = ctypes.c_int
        L.cj_set_boundary.argtypes = [_vp, _vp, _ll, _vp]
        L.cj_set_boundary.restype = ctypes.c_int
        L.cj_autotune_depth.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp,
                                        ctypes.POINTER(ctypes.c_int), _dp]
        L.cj_autotune_depth.restype = ctypes.c_int
        L.cj_solution_lo.argtypes = [_vp, _vp, _ll, _vp]
        L.cj_solution_lo.restype = ctypes.c_int
        L.cj_residual_noalloc.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _ll, _vp,
                                          _ll, _vp, _vp]
        L.cj_residual_noalloc.restype = ctypes.c_int
        L.cj_solve_batch.argtypes = [ctypes.POINTER(cj_problem), ctypes.c_int, _vp,
                                     ctypes.POINTER(cj_result)]
        L.cj_solve_batch.restype = ctypes.c_int
        L.cj_server_create.argtypes = [ctypes.c_size_t, ctypes.c_int, ctypes.POINTER(_vp)]
        L.cj_server_create.restype = ctypes.c_int
        L.cj_submit.argtypes = [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, _vp,
                                ctypes.POINTER(ctypes.c_uint64)]
        L.cj_submit.restype = ctypes.c_int
        L.cj_poll.argtypes = [_vp, ctypes.c_uint64, _vp, ctypes.POINTER(cj_result)]
        L.cj_poll.restype = ctypes.c_int
        L.cj_server_stats.argtypes = [_vp, ctypes.POINTER(cj_server_stats_t)]
        L.cj_server_stats.restype = ctypes.c_int
        L.cj_server_destroy.argtypes = [_vp]
        L.cj_server_destroy.restype = None
        L.cj_residual.argtypes = [_vp, _vp, _ll, _vp, _ll, _vp, _dp, _dp, _dp]
        L.cj_residual.restype = ctypes.c_int
        L.cj_issue_peaks.argtypes = [_vp, _dp, _dp]
        L.cj_issue_peaks.restype = ctypes.c_int
        L.cj_plan_weights.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int, _dp,
                                      _ll, ctypes.POINTER(_ll), _dp, _dp]
        L.cj_plan_weights.restype = ctypes.c_int
        L.cj_box_sweep.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, _vp, _ll, _vp, _ll,
                                   _vp, _ll, ctypes.c_int, _vp]
        L.cj_box_sweep.restype = ctypes.c_int
        L.cj_box_residual.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _ll, _vp, _ll, _vp, _ll, _vp,
                                      _vp]
        L.cj_box_residual.restype = ctypes.c_int
        L.cj_box_residual_slots.argtypes = [ctypes.c_int, ctypes.c_int]
        L.cj_box_residual_slots.restype = _ll
        L.cj_box_scale.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, _vp, _ll, _vp, _ll, _vp]
        L.cj_box_scale.restype = ctypes.c_int
        _L = L
    return _L


def cj_status_string(status: int) -> str:
    return _lib().cj_status_string(status).decode()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _grid(t, dtype_name: str):
    """(pointer, ld) of a 2-D CUDA tensor with unit x-stride."""
    if not (t.is_cuda and t.dim() == 2 and t.stride(1) == 1 and str(t.dtype) == "torch." + dtype_name):
        raise ValueError("expected a 2-D CUDA %s tensor with unit x-stride" % dtype_name)
    return t.data_ptr(), t.stride(0)


_plan_shape = {}   # plan handle -> (Nx, Ny), for the shape checks of the bindings


def cj_plan_create(Nx: int, Ny: int, st: int, tol: float, precision: int = CJ_FP64,
                   literal_n: int = 0, inner_cycle: int = 0, max_sweeps: int = 0,
                   bc: int = CJ_BC_DIRICHLET0, temporal_depth: int = 0, method: int = 0,
                   launch: int = 0):
    """Returns a plan handle (int); free it with cj_plan_destroy."""
    opt = cj_options(precision, literal_n, inner_cycle, temporal_depth, max_sweeps, method, launch)
    h = _vp()
    rc = _lib().cj_plan_create(Nx, Ny, st, bc, tol, ctypes.byref(opt), ctypes.byref(h))
    if rc != CJ_OK:
        raise CJError(rc, "cj_plan_create")
    _plan_shape[h.value] = (Nx, Ny)
    return h.value


def _mask_strides(t, Nx: int, Ny: int, name: str):
    """Element strides (sx, sy) of a CUDA float64 tensor whose last two axes have length Ny or
    1 and Nx or 1 (1 = the same value along that axis)."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64:
        raise ValueError("%s must be a CUDA float64 tensor" % name)
    ny, nx = t.shape[-2], t.shape[-1]
    if nx not in (1, Nx) or ny not in (1, Ny):
        raise ValueError("%s: trailing shape %s does not broadcast to (%d, %d)" % (name, tuple(t.shape), Ny, Nx))
    sx = t.stride(-1) if nx == Nx and Nx > 1 else 0
    sy = t.stride(-2) if ny == Ny and Ny > 1 else 0
    return sx, sy


def cj_plan_create_mask(Nx: int, Ny: int, pattern: int, coef, kmin: float, kmax: float, tol: float,
                        scale=None, method: int = 0, max_sweeps: int = 0):
    """Plan for a position-dependent coefficient mask (see cj_plan_create_mask in cj.h).
    coef: CUDA float64 tensor (K+1, Ny or 1, Nx or 1) -- the centre plane, then the off-centre
    offsets in row-major order; scale: None or a CUDA float64 tensor (Ny or 1, Nx or 1)."""
    if coef.dim() != 3:
        raise ValueError("coef must have shape (K+1, Ny or 1, Nx or 1)")
    sx, sy = _mask_strides(coef, Nx, Ny, "coef")
    m = cj_mask(pattern, coef.data_ptr(), sx, sy, coef.stride(0), None, 0, 0, kmin, kmax)
    if scale is not None:
        if scale.dim() != 2:
            raise ValueError("scale must have shape (Ny or 1, Nx or 1)")
        ssx, ssy = _mask_strides(scale, Nx, Ny, "scale")
        m.scale, m.scale_sx, m.scale_sy = scale.data_ptr(), ssx, ssy
    opt = cj_options(CJ_FP64, 0, 0, 0, max_sweeps, method, 0)
    h = _vp()
    rc = _lib().cj_plan_create_mask(Nx, Ny, ctypes.byref(m), tol, ctypes.byref(opt), ctypes.byref(h))
    if rc != CJ_OK:
        raise CJError(rc, "cj_plan_create_mask")
    _plan_shape[h.value] = (Nx, Ny)
    return h.value


def cj_plan_destroy(plan) -> None:
    _plan_shape.pop(plan, None)
    _lib().cj_plan_destroy(plan)


def cj_plan_info(plan) -> dict:
    w = _dp()
    M, Mi = _ll(), _ll()
    kmin, kmax = ctypes.c_double(), ctypes.c_double()
    rc = _lib().cj_plan_info(plan, ctypes.byref(w), ctypes.byref(M), ctypes.byref(kmin),
                             ctypes.byref(kmax), ctypes.byref(Mi))
    if rc != CJ_OK:
        raise CJError(rc, "cj_plan_info")
    return dict(w=np.ctypeslib.as_array(w, shape=(M.value,)).copy(), M=M.value, kmin=kmin.value,
                kmax=kmax.value, M_inner=Mi.value)


def cj_solve(plan, f, u, stream=None, check: bool = True) -> dict:
    """Solve on device tensors; u is in/out.  Returns the cj_result fields as a dict."""
    fp, ldf = _grid(f, "float64")
    up, ldu = _grid(u, "float64")
    res = cj_result()
    rc = _lib().cj_solve(plan, fp, ldf, up, ldu, _stream(stream), ctypes.byref(res))
    if check and rc < 0 and rc not in (CJ_ERR_NOT_CONVERGED, CJ_ERR_DIVERGED):
        raise CJError(rc, "cj_solve")
    d = res.as_dict()
    d["rc"] = rc
    return d


def cj_solve_to_error(plan, f, u, u_exact, err_tol: float, check_every: int = 0, stream=None,
                      cap: int = 4096, check: bool = True) -> dict:
    """Plain FP64 solve stopped by the real error max |u - u_exact| (device tensors; u in/out).
    Returns the cj_result fields plus real_error and history ((sweeps, real error) per test)."""
    fp, ldf = _grid(f, "float64")
    up, ldu = _grid(u, "float64")
    ep, lde = _grid(u_exact, "float64")
    res = cj_result()
    err = ctypes.c_double()
    hist = np.zeros(2 * cap)
    cnt = ctypes.c_int()
    rc = _lib().cj_solve_to_error(plan, fp, ldf, up, ldu, ep, lde, err_tol, check_every,
                                  _stream(stream), ctypes.byref(res), ctypes.byref(err),
                                  hist.ctypes.data_as(_dp), cap, ctypes.byref(cnt))
    if check and rc < 0 and rc not in (CJ_ERR_NOT_CONVERGED, CJ_ERR_DIVERGED):
        raise CJError(rc, "cj_solve_to_error")
    d = res.as_dict()
    d["rc"] = rc
    d["real_error"] = err.value
    d["tests"] = cnt.value
    k = min(cnt.value, cap)
    d["history"] = hist[:2 * k].reshape(k, 2).copy()
    return d


def cj_solve_history(plan, f, u, stream=None, cap: int = 4096, check: bool = True) -> dict:
    """cj_solve that also returns the relative residual at every residual test."""
    fp, ldf = _grid(f, "float64")
    up, ldu = _grid(u, "float64")
    res = cj_result()
    hist = (ctypes.c_double * cap)()
    cnt = ctypes.c_int()
    rc = _lib().cj_solve_history(plan, fp, ldf, up, ldu, _stream(stream), ctypes.byref(res),
                                 hist, cap, ctypes.byref(cnt))
    if check and rc < 0 and rc not in (CJ_ERR_NOT_CONVERGED, CJ_ERR_DIVERGED):
        raise CJError(rc, "cj_solve_history")
    d = res.as_dict()
    d["rc"] = rc
    d["history"] = list(hist[:min(cnt.value, cap)])
    return d


def cj_solve_host(plan, f_host: np.ndarray, u_host: np.ndarray, stream=None, check: bool = True) -> dict:
    """Solve on host arrays (C-contiguous float64, shape (Ny, Nx)); u_host is in/out."""
    for a in (f_host, u_host):
        if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous):
            raise ValueError("expected C-contiguous float64 numpy arrays")
    res = cj_result()
    rc = _lib().cj_solve_host(plan, f_host.ctypes.data, u_host.ctypes.data, _stream(stream),
                              ctypes.byref(res))
    if check and rc < 0 and rc not in (CJ_ERR_NOT_CONVERGED, CJ_ERR_DIVERGED):
        raise CJError(rc, "cj_solve_host")
    d = res.as_dict()
    d["rc"] = rc
    return d


def cj_sweeps(plan, f, u, first: int, count: int, stream=None) -> None:
    fp, ldf = _grid(f, "float64")
    up, ldu = _grid(u, "float64")
    rc = _lib().cj_sweeps(plan, fp, ldf, up, ldu, first, count, _stream(stream))
    if rc != CJ_OK:
        raise CJError(rc, "cj_sweeps")


def cj_sweeps_ff(plan, f, u, first: int, count: int, stream=None) -> None:
    """FP64-accuracy sweeps in float-float on the FP32 pipe (see cj.h); u in place."""
    fp, ldf = _grid(f, "float64")
    up, ldu = _grid(u, "float64")
    rc = _lib().cj_sweeps_ff(plan, fp, ldf, up, ldu, first, count, _stream(stream))
    if rc != CJ_OK:
        raise CJError(rc, "cj_sweeps_ff")


def cj_sweeps_f32(plan, r, e, first: int, count: int, stream=None) -> None:
    rp, ldr = _grid(r, "float32")
    ep, lde = _grid(e, "float32")
    rc = _lib().cj_sweeps_f32(plan, rp, ldr, ep, lde, first, count, _stream(stream))
    if rc != CJ_OK:
        raise CJError(rc, "cj_sweeps_f32")


def dirichlet_ring(Nx: int, Ny: int, g) -> np.ndarray:
    """Host array of shape (Ny+4, Nx+4) for cj_set_boundary: g(i, j) (vectorised over integer
    node indices) at every node with i or j in {-1, 0, N+1, N+2}, zero inside."""
    i = np.arange(-1, Nx + 3)[None, :]
    j = np.arange(-1, Ny + 3)[:, None]
    G = np.array(np.broadcast_to(g(i, j), (Ny + 4, Nx + 4)), dtype=np.float64)
    G[2:Ny + 2, 2:Nx + 2] = 0.0
    return G


def cj_set_boundary(plan, g, stream=None) -> None:
    """Dirichlet data of a CJ_BC_DIRICHLET plan: g is a CUDA float64 tensor of shape
    (Ny+4, >= Nx+4) holding node (i, j) at g[j+1, i+1] (the two rings around the interior)."""
    Nx, Ny = _plan_shape.get(plan, (0, 0))
    if g.dim() != 2 or g.shape[0] != Ny + 4 or g.shape[1] < Nx + 4:
        raise CJError(CJ_ERR_INVALID_ARG, "cj_set_boundary: g must have shape (Ny+4, >= Nx+4)")
    gp, ld = _grid(g, "float64")
    rc = _lib().cj_set_boundary(plan, gp, ld, _stream(stream))
    if rc != CJ_OK:
        raise CJError(rc, "cj_set_boundary")


def cj_autotune_depth(Nx: int, Ny: int, st: int, sweeps: int = 64, stream=None) -> dict:
    """Time FP32 sweeps at temporal depths 1, 2, 4, 8 and record the fastest for this
    stencil and size class; returns {"best": depth, "gupd": {depth: rate}}."""
    best = ctypes.c_int()
    rates = (ctypes.c_double * 4)()
    rc = _lib().cj_autotune_depth(Nx, Ny, st, sweeps, _stream(stream), ctypes.byref(best), rates)
    if rc != CJ_OK:
        raise CJError(rc, "cj_autotune_depth")
    return {"best": best.value, "gupd": dict(zip((1, 2, 4, 8), list(rates)))}


def cj_solution_lo(plan, u_lo, stream=None) -> None:
    """Low part of the last double-FP64 solve (CJ_FP32_INNER_DD plans)."""
    up, ld = _grid(u_lo, "float64")
    rc = _lib().cj_solution_lo(plan, up, ld, _stream(stream))
    if rc != CJ_OK:
        raise CJError(rc, "cj_solution_lo")


def cj_residual(plan, f, u, stream=None):
    """(relative L2 residual, relative max residual, FP64 floor estimate) of u."""
    fp, ldf = _grid(f, "float64")
    up, ldu = _grid(u, "float64")
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    rc = _lib().cj_residual(plan, fp, ldf, up, ldu, _stream(stream), ctypes.byref(a),
                            ctypes.byref(b), ctypes.byref(c))
    if rc != CJ_OK:
        raise CJError(rc, "cj_residual")
    return a.value, b.value, c.value


def _noalloc_args(Nx: int, Ny: int, f, u, out, current_device=None):
    """Checks of cj_residual_noalloc's tensors, all made before anything is launched: f and u are
    2-D CUDA float64 tensors with unit x-stride holding at least Ny rows of Nx columns (the
    kernel reads exactly that block), out a contiguous CUDA float64 tensor of >= 3 elements, and
    all three live on the current device (the scratch address is that device's).  Returns
    (f pointer, ld_f, u pointer, ld_u)."""
    fp, ldf = _grid(f, "float64")
    up, ldu = _grid(u, "float64")
    for name, t in (("f", f), ("u", u)):
        if t.shape[0] < Ny or t.shape[1] < Nx:
            raise ValueError("%s has shape %s, smaller than the %d x %d grid" % (name, tuple(t.shape), Ny, Nx))
    if not (out.is_cuda and str(out.dtype) == "torch.float64" and out.numel() >= 3 and out.is_contiguous()):
        raise ValueError("out must be a contiguous CUDA float64 tensor of >= 3 elements")
    if current_device is None:
        import torch
        current_device = torch.cuda.current_device()
    for name, t in (("f", f), ("u", u), ("out", out)):
        if t.device.index != current_device:
            raise ValueError("%s is on cuda:%s, not on the current device cuda:%d" % (name, t.device.index,
                                                                                    current_device))
    return fp, ldf, up, ldu


def cj_residual_noalloc(Nx: int, Ny: int, st: int, f, u, out, stream=None) -> None:
    """Allocation-free residual norms: writes (rel_l2, rel_inf, floor_est) into the device
    tensor ``out`` (3 float64) on the stream; no plan, no device allocation."""
    fp, ldf, up, ldu = _noalloc_args(Nx, Ny, f, u, out)
    rc = _lib().cj_residual_noalloc(Nx, Ny, st, fp, ldf, up, ldu, out.data_ptr(), _stream(stream))
    if rc != CJ_OK:
        raise CJError(rc, "cj_residual_noalloc")


def cj_issue_peaks(stream=None) -> dict:
    """Measured FP64 and FP32 FMA issue rates of the current device (T FMA/s), see cj.h."""
    a, b = ctypes.c_double(), ctypes.c_double()
    rc = _lib().cj_issue_peaks(_stream(stream), ctypes.byref(a), ctypes.byref(b))
    if rc != CJ_OK:
        raise CJError(rc, "cj_issue_peaks")
    return {"fp64_tfma_s": a.value, "fp32_tfma_s": b.value}


def cj_solve_batch(problems, stream=None) -> list:
    """Solve independent problems together.  Each problem is a dict with keys Nx, Ny, st,
    tol, f (CUDA float64 tensor), u (in/out CUDA float64 tensor) and optionally precision,
    inner_cycle, temporal_depth, max_sweeps.  Returns one result dict per problem."""
    n = len(problems)
    arr = (cj_problem * n)()
    for k, pr in enumerate(problems):
        fp, ldf = _grid(pr["f"], "float64")
        up, ldu = _grid(pr["u"], "float64")
        arr[k] = cj_problem(pr["Nx"], pr["Ny"], pr["st"], pr.get("precision", 0), pr["tol"],
                            pr.get("inner_cycle", 0), pr.get("temporal_depth", 0),
                            pr.get("max_sweeps", 0), fp, ldf, up, ldu)
    res = (cj_result * n)()
    rc = _lib().cj_solve_batch(arr, n, _stream(stream), res)
    if rc not in (CJ_OK, CJ_ERR_TIMEOUT):
        raise CJError(rc, "cj_solve_batch")
    out = []
    for k in range(n):
        d = res[k].as_dict()
        d["rc"] = res[k].status
        out.append(d)
    return out


class Server:
    """Request server with continuous batching (cj_server_create / cj_submit / cj_poll)."""

    def __init__(self, hbm_budget_bytes: int, max_slots: int):
        h = _vp()
        rc = _lib().cj_server_create(hbm_budget_bytes, max_slots, ctypes.byref(h))
        if rc != CJ_OK:
            raise CJError(rc, "cj_server_create")
        self.handle = h.value

    def submit(self, f_host: np.ndarray, st: int, tol: float) -> int:
        f_host = np.ascontiguousarray(f_host, dtype=np.float64)
        Ny, Nx = f_host.shape
        t = ctypes.c_uint64()
        rc = _lib().cj_submit(self.handle, Nx, Ny, st, tol, f_host.ctypes.data, ctypes.byref(t))
        if rc != CJ_OK:
            raise CJError(rc, "cj_submit")
        return t.value

    def poll(self, ticket: int, shape):
        """None while pending, else (u, result dict)."""
        u = np.empty(shape, dtype=np.float64)
        res = cj_result()
        rc = _lib().cj_poll(self.handle, ticket, u.ctypes.data, ctypes.byref(res))
        if rc == CJ_PENDING:
            return None
        d = res.as_dict()
        d["rc"] = rc
        return u, d

    def stats(self) -> dict:
        s = cj_server_stats_t()
        rc = _lib().cj_server_stats(self.handle, ctypes.byref(s))
        if rc != CJ_OK:
            raise CJError(rc, "cj_server_stats")
        return {k: getattr(s, k) for k, _ in s._fields_}

    def close(self):
        if self.handle:
            _lib().cj_server_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Plan:
    """Owning wrapper: ``with Plan(Nx, Ny, st, tol) as p: cj_solve(p.handle, f, u)``."""

    def __init__(self, Nx, Ny, st, tol, **kw):
        self.handle = cj_plan_create(Nx, Ny, st, tol, **kw)
        self.Nx, self.Ny, self.st, self.tol = Nx, Ny, st, tol

    @classmethod
    def mask(cls, Nx, Ny, pattern, coef, kmin, kmax, tol, **kw):
        """Owning wrapper of cj_plan_create_mask."""
        self = cls.__new__(cls)
        self.handle = cj_plan_create_mask(Nx, Ny, pattern, coef, kmin, kmax, tol, **kw)
        self.Nx, self.Ny, self.st, self.tol = Nx, Ny, pattern, tol
        return self

    def info(self) -> dict:
        return cj_plan_info(self.handle)

    def close(self):
        if self.handle:
            cj_plan_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cj_autotune_engine(Nx: int, Ny: int, st: int) -> dict:
    """Times the batched engine at tile rows 16/32/64 x depth 1/2/4 for this stencil and size
    class and records the fastest for cj_solve_batch and the server (see cj.h)."""
    ty, d = ctypes.c_int(), ctypes.c_int()
    g = (ctypes.c_double * 9)()
    rc = _lib().cj_autotune_engine(Nx, Ny, st, ctypes.byref(ty), ctypes.byref(d), g)
    if rc != CJ_OK:
        raise CJError(rc, "cj_autotune_engine")
    return dict(tile_rows=ty.value, depth=d.value,
                gupd={(r, k): g[i * 3 + j] for i, r in enumerate((16, 32, 64)) for j, k in enumerate((1, 2, 4))})
