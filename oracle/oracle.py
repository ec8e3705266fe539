"""ctypes front end of the plain C FP64 Chebyshev-Jacobi oracle (``cj_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test-suite, the smoke check and the CPU-baseline leg of
the benchmark may use this module; the product library never imports it.

Arrays follow the oracle's convention: interior values, shape ``(Ny, Nx)``, C order,
``float64`` (``float32`` for the FP32 inner form).  Every function cites the passage of
the paper it follows in ``cj_oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cj_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libcj_oracle.so")

_dp = ctypes.POINTER(ctypes.c_double)
_fp = ctypes.POINTER(ctypes.c_float)
_lp = ctypes.POINTER(ctypes.c_long)
_ip = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (``-ffp-contract=off``: no silent FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        os.makedirs(os.path.dirname(_LIB), exist_ok=True)
        tmp = _LIB + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        L.orc_radius.argtypes = [ctypes.c_int]
        L.orc_radius.restype = ctypes.c_int
        L.orc_centre.argtypes = [ctypes.c_int]
        L.orc_centre.restype = ctypes.c_double
        L.orc_apply_L.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp]
        L.orc_kappa_bounds.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp]
        L.orc_kappa_bounds_n.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, _dp, _dp]
        L.orc_cycle_length_min.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double]
        L.orc_cycle_length_min.restype = ctypes.c_long
        L.orc_cycle_length.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double]
        L.orc_cycle_length.restype = ctypes.c_long
        L.orc_order.argtypes = [ctypes.c_long, _lp]
        L.orc_order.restype = ctypes.c_int
        L.orc_weights_natural.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_long, _dp]
        L.orc_sweep_coeffs.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_long, _dp]
        L.orc_sweep_coeffs.restype = ctypes.c_int
        L.orc_sweep.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp, ctypes.c_double, _dp]
        L.orc_residual.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp]
        L.orc_scale_rhs.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp]
        L.orc_solve.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, ctypes.c_double,
                                ctypes.c_long, _dp, _dp, _dp, _lp, _ip]
        L.orc_solve.restype = ctypes.c_long
        L.orc_abs_coeff_sum.argtypes = [ctypes.c_int]
        L.orc_abs_coeff_sum.restype = ctypes.c_double
        L.orc_sweep_f32.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _fp, _fp, ctypes.c_float, _fp]
        L.orc_defect.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp, _fp, _dp, _dp]
        L.orc_solve_mixed.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, ctypes.c_double,
                                      ctypes.c_long, ctypes.c_long, _dp, _dp, _dp, _lp, _ip]
        L.orc_solve_mixed.restype = ctypes.c_long
        L.orc_sweep_bc.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, ctypes.c_double, _dp]
        L.orc_residual_bc.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp, _dp]
        L.orc_solve_bc.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp, ctypes.c_double,
                                   ctypes.c_long, _dp, _dp, _dp, _lp, _ip]
        L.orc_solve_bc.restype = ctypes.c_long
        L.orc_solve_jacobi.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp, ctypes.c_double,
                                       ctypes.c_long, _dp, _dp, _dp, _lp, ctypes.POINTER(ctypes.c_int)]
        L.orc_solve_jacobi.restype = ctypes.c_long
        L.orc_mask_offsets.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
        L.orc_mask_offsets.restype = ctypes.c_int
        L.orc_mask_normalize.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, ctypes.c_long,
                                         ctypes.c_long, ctypes.c_long, _dp, ctypes.c_long, ctypes.c_long,
                                         _dp, _dp]
        L.orc_mask_normalize.restype = ctypes.c_int
        L.orc_sweep_mask.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp,
                                     ctypes.c_double, _dp]
        L.orc_residual_mask.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp, _dp, _dp]
        L.orc_mask_weights.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_long, _dp]
        L.orc_mask_weights.restype = ctypes.c_int
        L.orc_solve_mask.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp, ctypes.c_long,
                                     ctypes.c_long, ctypes.c_long, _dp, ctypes.c_long, ctypes.c_long,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int, _dp,
                                     ctypes.c_long, _dp, _dp, _dp, _lp, ctypes.POINTER(ctypes.c_int)]
        L.orc_solve_mask.restype = ctypes.c_long
        L.orc_solve_mixed_to_error.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp, _dp,
                                               ctypes.c_double, ctypes.c_long, ctypes.c_int, ctypes.c_long,
                                               _dp, _dp, _dp, ctypes.c_long, _lp, _dp, _dp, _lp,
                                               ctypes.POINTER(ctypes.c_int)]
        L.orc_solve_mixed_to_error.restype = ctypes.c_long
        L.orc_real_error.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp]
        L.orc_real_error.restype = ctypes.c_double
        L.orc_solve_to_error.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp, _dp,
                                         ctypes.c_double, ctypes.c_double, ctypes.c_long,
                                         ctypes.c_long, _dp, _dp, ctypes.c_long, _lp, _dp, _dp,
                                         _lp, ctypes.POINTER(ctypes.c_int)]
        L.orc_solve_to_error.restype = ctypes.c_long
        L.orc_residual_dd.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp]
        L.orc_solve_mixed_dd.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, ctypes.c_double,
                                         ctypes.c_long, ctypes.c_long, _dp, _dp, _dp, _dp, _lp, _ip]
        L.orc_solve_mixed_dd.restype = ctypes.c_long
        L.orc_solve_mixed_bc.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp, ctypes.c_double,
                                         ctypes.c_long, ctypes.c_long, _dp, _dp, _dp, _lp, _ip]
        L.orc_solve_mixed_bc.restype = ctypes.c_long
        L.orc_solve_mixed_dd_bc.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp, ctypes.c_double,
                                            ctypes.c_long, ctypes.c_long, _dp, _dp, _dp, _dp, _lp, _ip]
        L.orc_solve_mixed_dd_bc.restype = ctypes.c_long
        L.orc_solve_fp64_dd.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp, ctypes.c_double,
                                        ctypes.c_long, ctypes.c_long, _dp, _dp, _dp, _dp, _lp, _ip]
        L.orc_solve_fp64_dd.restype = ctypes.c_long
        _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(_dp)


def _f(a):
    return a.ctypes.data_as(_fp)


def _grid(a, dtype=np.float64):
    a = np.ascontiguousarray(a, dtype=dtype)
    assert a.ndim == 2
    return a


def radius(st: int) -> int:
    return lib().orc_radius(st)


def centre(st: int) -> float:
    """c = -(centre coefficient of h^2 Delta_h)."""
    return lib().orc_centre(st)


def apply_L(st: int, u: np.ndarray) -> np.ndarray:
    """L u = h^2 Delta_h u with the homogeneous Dirichlet / odd-reflection boundary."""
    u = _grid(u)
    out = np.empty_like(u)
    lib().orc_apply_L(st, u.shape[1], u.shape[0], _d(u), _d(out))
    return out


def kappa_bounds(st: int, Nx: int, Ny: int, literal_n: bool = False):
    """(kmin, kmax) of D^-1 A (Sec. 2.1); ``literal_n`` uses N = Nx instead of Nx+1."""
    a, b = ctypes.c_double(), ctypes.c_double()
    if literal_n:
        lib().orc_kappa_bounds_n(st, float(Nx), float(Ny), ctypes.byref(a), ctypes.byref(b))
    else:
        lib().orc_kappa_bounds(st, Nx, Ny, ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def cycle_length_min(kmin: float, kmax: float, tol: float) -> int:
    return lib().orc_cycle_length_min(kmin, kmax, tol)


def cycle_length(kmin: float, kmax: float, tol: float) -> int:
    return lib().orc_cycle_length(kmin, kmax, tol)


def order(M: int) -> np.ndarray:
    idx = np.zeros(M, dtype=np.int64)
    rc = lib().orc_order(M, idx.ctypes.data_as(_lp))
    if rc != 0:
        raise ValueError("M must be a power of two")
    return idx


def weights_natural(kmin: float, kmax: float, M: int) -> np.ndarray:
    w = np.zeros(M)
    lib().orc_weights_natural(kmin, kmax, M, _d(w))
    return w


def sweep_coeffs(st: int, kmin: float, kmax: float, M: int) -> np.ndarray:
    """w_n = omega_n / c in application order."""
    w = np.zeros(M)
    if lib().orc_sweep_coeffs(st, kmin, kmax, M, _d(w)) != 0:
        raise ValueError("M must be a power of two")
    return w


def sweep(st: int, u: np.ndarray, b: np.ndarray, w: float) -> np.ndarray:
    u = _grid(u)
    b = _grid(b)
    out = np.empty_like(u)
    lib().orc_sweep(st, u.shape[1], u.shape[0], _d(u), _d(b), float(w), _d(out))
    return out


def residual(st: int, u: np.ndarray, b: np.ndarray):
    """(sum of squares, max-abs) of L u - b."""
    u = _grid(u)
    b = _grid(b)
    s, m = ctypes.c_double(), ctypes.c_double()
    lib().orc_residual(st, u.shape[1], u.shape[0], _d(u), _d(b), ctypes.byref(s), ctypes.byref(m))
    return s.value, m.value


def scale_rhs(f: np.ndarray) -> np.ndarray:
    f = _grid(f)
    b = np.empty_like(f)
    lib().orc_scale_rhs(f.shape[1], f.shape[0], _d(f), _d(b))
    return b


STATUS = {0: "converged", 1: "floor", 2: "max_sweeps", 3: "diverged", 4: "stalled"}


def abs_coeff_sum(st: int) -> float:
    return lib().orc_abs_coeff_sum(st)


def solve(st: int, f: np.ndarray, tol: float, u0: np.ndarray | None = None,
          max_sweeps: int = 1 << 40) -> dict:
    """Full FP64 CJM solve of Delta_h u = f; returns u and the run's counters."""
    f = _grid(f)
    u = np.zeros_like(f) if u0 is None else _grid(u0).copy()
    rl2, rinf = ctypes.c_double(), ctypes.c_double()
    cyc, stat = ctypes.c_long(), ctypes.c_int()
    n = lib().orc_solve(st, f.shape[1], f.shape[0], _d(f), tol, max_sweeps, _d(u),
                        ctypes.byref(rl2), ctypes.byref(rinf), ctypes.byref(cyc), ctypes.byref(stat))
    if n < 0:
        raise ValueError("bad argument")
    return dict(u=u, sweeps=n, cycles=cyc.value, rel_l2=rl2.value, rel_linf=rinf.value,
                status=STATUS[stat.value], converged=stat.value == 0)


def sweep_f32(st: int, e: np.ndarray, r: np.ndarray, w: float) -> np.ndarray:
    e = _grid(e, np.float32)
    r = _grid(r, np.float32)
    out = np.empty_like(e)
    lib().orc_sweep_f32(st, e.shape[1], e.shape[0], _f(e), _f(r), ctypes.c_float(w), _f(out))
    return out


def defect(st: int, u: np.ndarray, b: np.ndarray):
    """(rt = float32(b - L u), sum of squares, max-abs) in FP64."""
    u = _grid(u)
    b = _grid(b)
    rt = np.empty(u.shape, np.float32)
    s, m = ctypes.c_double(), ctypes.c_double()
    lib().orc_defect(st, u.shape[1], u.shape[0], _d(u), _d(b), _f(rt), ctypes.byref(s), ctypes.byref(m))
    return rt, s.value, m.value


def solve_mixed(st: int, f: np.ndarray, tol: float, M_in: int, u0: np.ndarray | None = None,
                max_outer: int = 1000, G: np.ndarray | None = None) -> dict:
    """FP32-inner / FP64-outer defect-correction CJM (with Dirichlet data G, see ghost_ring)."""
    f = _grid(f)
    u = np.zeros_like(f) if u0 is None else _grid(u0).copy()
    rl2, rinf = ctypes.c_double(), ctypes.c_double()
    outer, stat = ctypes.c_long(), ctypes.c_int()
    if G is None:
        n = lib().orc_solve_mixed(st, f.shape[1], f.shape[0], _d(f), tol, M_in, max_outer, _d(u),
                                  ctypes.byref(rl2), ctypes.byref(rinf), ctypes.byref(outer),
                                  ctypes.byref(stat))
    else:
        n = lib().orc_solve_mixed_bc(st, f.shape[1], f.shape[0], _d(f), _d(_grid(G)), tol, M_in, max_outer,
                                     _d(u), ctypes.byref(rl2), ctypes.byref(rinf), ctypes.byref(outer),
                                     ctypes.byref(stat))
    if n < 0:
        raise ValueError("bad argument")
    return dict(u=u, sweeps=n, outer=outer.value, rel_l2=rl2.value, rel_linf=rinf.value,
                status=STATUS[stat.value], converged=stat.value == 0)


def residual_dd(st: int, uh: np.ndarray, ul: np.ndarray, b: np.ndarray) -> np.ndarray:
    """R = L (uh + ul) - b evaluated to about twice FP64 precision, rounded to FP64."""
    uh, ul, b = _grid(uh), _grid(ul), _grid(b)
    R = np.empty_like(uh)
    lib().orc_residual_dd(st, uh.shape[1], uh.shape[0], _d(uh), _d(ul), _d(b), _d(R))
    return R


def solve_mixed_dd(st: int, f: np.ndarray, tol: float, M_in: int, u0: np.ndarray | None = None,
                   max_outer: int = 1000, G: np.ndarray | None = None) -> dict:
    """FP32-inner CJM cycles inside a double-FP64 defect-correction loop (with Dirichlet data
    G, see ghost_ring); returns u = fl(u_hi + u_lo) and u_lo."""
    f = _grid(f)
    u = np.zeros_like(f) if u0 is None else _grid(u0).copy()
    ulo = np.zeros_like(f)
    rl2, rinf = ctypes.c_double(), ctypes.c_double()
    outer, stat = ctypes.c_long(), ctypes.c_int()
    if G is None:
        n = lib().orc_solve_mixed_dd(st, f.shape[1], f.shape[0], _d(f), tol, M_in, max_outer, _d(u),
                                     _d(ulo), ctypes.byref(rl2), ctypes.byref(rinf),
                                     ctypes.byref(outer), ctypes.byref(stat))
    else:
        n = lib().orc_solve_mixed_dd_bc(st, f.shape[1], f.shape[0], _d(f), _d(_grid(G)), tol, M_in,
                                        max_outer, _d(u), _d(ulo), ctypes.byref(rl2), ctypes.byref(rinf),
                                        ctypes.byref(outer), ctypes.byref(stat))
    if n < 0:
        raise ValueError("bad argument")
    return dict(u=u, u_lo=ulo, sweeps=n, outer=outer.value, rel_l2=rl2.value, rel_linf=rinf.value,
                status=STATUS[stat.value], converged=stat.value == 0)


def solve_fp64_dd(st: int, f: np.ndarray, tol: float, M_in: int, u0: np.ndarray | None = None,
                  max_outer: int = 1000, G: np.ndarray | None = None) -> dict:
    """FP64-inner CJM cycles of length M_in inside the double-FP64 defect-correction loop
    (reading R20; with Dirichlet data G, see ghost_ring); returns u = fl(u_hi + u_lo), u_lo and
    the FP64 sweeps done."""
    f = _grid(f)
    u = np.zeros_like(f) if u0 is None else _grid(u0).copy()
    ulo = np.zeros_like(f)
    rl2, rinf = ctypes.c_double(), ctypes.c_double()
    outer, stat = ctypes.c_long(), ctypes.c_int()
    n = lib().orc_solve_fp64_dd(st, f.shape[1], f.shape[0], _d(f), None if G is None else _d(_grid(G)), tol,
                                M_in, max_outer, _d(u), _d(ulo), ctypes.byref(rl2), ctypes.byref(rinf),
                                ctypes.byref(outer), ctypes.byref(stat))
    if n < 0:
        raise ValueError("bad argument")
    return dict(u=u, u_lo=ulo, sweeps=n, outer=outer.value, rel_l2=rl2.value, rel_linf=rinf.value,
                status=STATUS[stat.value], converged=stat.value == 0)


def ghost_ring(Nx: int, Ny: int, g) -> np.ndarray:
    """Padded (Ny+4) x (Nx+4) array of the Dirichlet data g(i, j) at the two-node ring around
    the interior (interior entries 0): the ring the stencils reach."""
    G = np.zeros((Ny + 4, Nx + 4))
    for j in range(-1, Ny + 3):
        for i in range(-1, Nx + 3):
            if i < 1 or i > Nx or j < 1 or j > Ny:
                G[j + 1, i + 1] = g(i, j)
    return G


def sweep_bc(st: int, u: np.ndarray, G: np.ndarray, b: np.ndarray, w: float) -> np.ndarray:
    u, G, b = _grid(u), _grid(G), _grid(b)
    out = np.empty_like(u)
    lib().orc_sweep_bc(st, u.shape[1], u.shape[0], _d(u), _d(G), _d(b), float(w), _d(out))
    return out


def residual_bc(st: int, u: np.ndarray, G: np.ndarray, b: np.ndarray):
    u, G, b = _grid(u), _grid(G), _grid(b)
    s, m = ctypes.c_double(), ctypes.c_double()
    lib().orc_residual_bc(st, u.shape[1], u.shape[0], _d(u), _d(G), _d(b), ctypes.byref(s), ctypes.byref(m))
    return s.value, m.value


def solve_bc(st: int, f: np.ndarray, G: np.ndarray, tol: float, u0: np.ndarray | None = None,
             max_sweeps: int = 1 << 40) -> dict:
    """Plain FP64 CJM with non-homogeneous Dirichlet data G (see ghost_ring)."""
    f, G = _grid(f), _grid(G)
    u = np.zeros_like(f) if u0 is None else _grid(u0).copy()
    rl2, rinf = ctypes.c_double(), ctypes.c_double()
    cyc, stat = ctypes.c_long(), ctypes.c_int()
    n = lib().orc_solve_bc(st, f.shape[1], f.shape[0], _d(f), _d(G), tol, max_sweeps, _d(u),
                           ctypes.byref(rl2), ctypes.byref(rinf), ctypes.byref(cyc), ctypes.byref(stat))
    if n < 0:
        raise ValueError("bad argument")
    return dict(u=u, sweeps=n, cycles=cyc.value, rel_l2=rl2.value, rel_linf=rinf.value,
                status=STATUS[stat.value], converged=stat.value == 0)


def real_error(u: np.ndarray, u_exact: np.ndarray) -> float:
    """Infinity norm of u - u_exact (the real error of Sec. 3.4)."""
    u, ue = _grid(u), _grid(u_exact)
    return lib().orc_real_error(u.shape[1], u.shape[0], _d(u), _d(ue))


def solve_to_error(st: int, f: np.ndarray, u_exact: np.ndarray, tol: float, err_tol: float,
                   G: np.ndarray | None = None, check_every: int = 0,
                   max_sweeps: int = 1 << 40, cap: int = 4096) -> dict:
    """Plain FP64 CJM stopped by the real error (see orc_solve_to_error); G as in ghost_ring,
    None for the homogeneous boundary.  history: (sweeps, real error) at every test."""
    f, ue = _grid(f), _grid(u_exact)
    Gp = None if G is None else _d(_grid(G))
    u = np.zeros_like(f)
    hist = np.zeros(2 * cap)
    cnt, cyc, stat = ctypes.c_long(), ctypes.c_long(), ctypes.c_int()
    err, rl2 = ctypes.c_double(), ctypes.c_double()
    n = lib().orc_solve_to_error(st, f.shape[1], f.shape[0], _d(f), Gp, _d(ue), tol, err_tol,
                                 check_every, max_sweeps, _d(u), _d(hist), cap, ctypes.byref(cnt),
                                 ctypes.byref(err), ctypes.byref(rl2), ctypes.byref(cyc),
                                 ctypes.byref(stat))
    if n < 0:
        raise ValueError("bad argument")
    k = min(cnt.value, cap)
    return dict(u=u, sweeps=n, cycles=cyc.value, err=err.value, rel_l2=rl2.value,
                status=STATUS[stat.value], tests=cnt.value,
                history=hist[:2 * k].reshape(k, 2).copy())


def solve_jacobi(st: int, f: np.ndarray, tol: float, G: np.ndarray | None = None,
                 u0: np.ndarray | None = None, max_sweeps: int = 1 << 40) -> dict:
    """Classical Jacobi (omega = 1) with the residual tested every M sweeps (orc_solve_jacobi)."""
    f = _grid(f)
    Gp = None if G is None else _d(_grid(G))
    u = np.zeros_like(f) if u0 is None else _grid(u0).copy()
    rl2, rinf = ctypes.c_double(), ctypes.c_double()
    done, stat = ctypes.c_long(), ctypes.c_int()
    n = lib().orc_solve_jacobi(st, f.shape[1], f.shape[0], _d(f), Gp, tol, max_sweeps, _d(u),
                               ctypes.byref(rl2), ctypes.byref(rinf), ctypes.byref(done),
                               ctypes.byref(stat))
    if n < 0:
        raise ValueError("bad argument")
    return dict(u=u, sweeps=n, cycles=done.value, rel_l2=rl2.value, rel_linf=rinf.value,
                status=STATUS[stat.value], converged=stat.value == 0)


# ----------------------------------------------------------------- coefficient masks (R19)

def mask_offsets(pat: int):
    """Off-centre offsets (dx, dy) of a mask pattern, in application order."""
    dx, dy = (ctypes.c_int * 24)(), (ctypes.c_int * 24)()
    K = lib().orc_mask_offsets(pat, dx, dy)
    return [(dx[k], dy[k]) for k in range(K)]


def _bcast(a: np.ndarray, Nx: int, Ny: int, planes: bool):
    """A C-contiguous copy of a (possibly broadcast) coefficient array and its element strides
    (sx, sy, sp): the last two axes have length Nx / Ny or 1 (1 = repeated along that axis)."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    ny, nx = a.shape[-2], a.shape[-1]
    if nx not in (1, Nx) or ny not in (1, Ny):
        raise ValueError("coefficient shape %s does not broadcast to (%d, %d)" % (a.shape, Ny, Nx))
    sx = 1 if nx == Nx and Nx > 1 else 0
    sy = nx if ny == Ny and Ny > 1 else 0
    return a, sx, sy, nx * ny


def mask_normalize(pat: int, coef: np.ndarray, scale: np.ndarray | None, Nx: int, Ny: int):
    """(chat, dC): the normalised off-centre coefficients (K, Ny, Nx) and s * c_C (Ny, Nx)."""
    c, sx, sy, sp = _bcast(coef, Nx, Ny, True)
    K = len(mask_offsets(pat))
    if c.shape[0] != K + 1:
        raise ValueError("expected %d planes" % (K + 1))
    if scale is not None:
        sc, ssx, ssy, _ = _bcast(scale, Nx, Ny, False)
    chat = np.zeros((max(K, 1), Ny, Nx))
    dC = np.zeros((Ny, Nx))
    rc = lib().orc_mask_normalize(pat, Nx, Ny, _d(c), sx, sy, sp, None if scale is None else _d(sc),
                                  0 if scale is None else ssx, 0 if scale is None else ssy, _d(chat), _d(dC))
    if rc < 0:
        raise ValueError("bad mask")
    return chat[:K], dC


def sweep_mask(pat: int, u: np.ndarray, G, bhat: np.ndarray, chat: np.ndarray, w: float) -> np.ndarray:
    u, bhat, chat = _grid(u), _grid(bhat), np.ascontiguousarray(chat, dtype=np.float64)
    out = np.empty_like(u)
    lib().orc_sweep_mask(pat, u.shape[1], u.shape[0], _d(u), None if G is None else _d(_grid(G)),
                         _d(bhat), _d(chat), float(w), _d(out))
    return out


def residual_mask(pat: int, u: np.ndarray, G, bhat: np.ndarray, chat: np.ndarray):
    u, bhat, chat = _grid(u), _grid(bhat), np.ascontiguousarray(chat, dtype=np.float64)
    sq, mx = ctypes.c_double(), ctypes.c_double()
    lib().orc_residual_mask(pat, u.shape[1], u.shape[0], _d(u), None if G is None else _d(_grid(G)),
                            _d(bhat), _d(chat), ctypes.byref(sq), ctypes.byref(mx))
    return sq.value, mx.value


def mask_weights(kmin: float, kmax: float, M: int) -> np.ndarray:
    w = np.zeros(M)
    if lib().orc_mask_weights(kmin, kmax, M, _d(w)) != 0:
        raise ValueError("M must be a power of two")
    return w


def solve_mask(pat: int, f: np.ndarray, coef: np.ndarray, kmin: float, kmax: float, tol: float,
               scale: np.ndarray | None = None, G: np.ndarray | None = None, method: int = 0,
               max_sweeps: int = 1 << 40, u0: np.ndarray | None = None) -> dict:
    """CJM (method 0) or classical Jacobi (1) on the masked operator A u = f (orc_solve_mask)."""
    f = _grid(f)
    Ny, Nx = f.shape
    c, sx, sy, sp = _bcast(coef, Nx, Ny, True)
    if scale is not None:
        sc, ssx, ssy, _ = _bcast(scale, Nx, Ny, False)
    u = np.zeros_like(f) if u0 is None else _grid(u0).copy()
    rl2, rinf = ctypes.c_double(), ctypes.c_double()
    cyc, stat = ctypes.c_long(), ctypes.c_int()
    n = lib().orc_solve_mask(pat, Nx, Ny, _d(f), _d(c), sx, sy, sp, None if scale is None else _d(sc),
                             0 if scale is None else ssx, 0 if scale is None else ssy, kmin, kmax, tol,
                             method, None if G is None else _d(_grid(G)), max_sweeps, _d(u),
                             ctypes.byref(rl2), ctypes.byref(rinf), ctypes.byref(cyc), ctypes.byref(stat))
    if n < 0:
        raise ValueError("bad argument")
    return dict(u=u, sweeps=n, cycles=cyc.value, rel_l2=rl2.value, rel_linf=rinf.value,
                status=STATUS[stat.value], converged=stat.value == 0)


def solve_mixed_to_error(st: int, f: np.ndarray, u_exact: np.ndarray, err_goal: float, M_in: int,
                         dd: int = 0, G: np.ndarray | None = None, max_outer: int = 1000,
                         cap: int = 4096) -> dict:
    """Defect correction stopped by the real error at the outer steps (orc_solve_mixed_to_error):
    dd = 0 FP32 inner cycles in FP64 outer steps, 1 (or True) FP32 inner cycles in double-FP64
    outer steps, 2 FP64 inner cycles in double-FP64 outer steps."""
    f, ue = _grid(f), _grid(u_exact)
    u, ulo = np.zeros_like(f), np.zeros_like(f)
    hist = np.zeros(2 * cap)
    cnt, outer, stat = ctypes.c_long(), ctypes.c_long(), ctypes.c_int()
    err, rl2 = ctypes.c_double(), ctypes.c_double()
    n = lib().orc_solve_mixed_to_error(st, f.shape[1], f.shape[0], _d(f), None if G is None else _d(_grid(G)),
                                       _d(ue), err_goal, M_in, int(dd), max_outer, _d(u), _d(ulo), _d(hist),
                                       cap, ctypes.byref(cnt), ctypes.byref(err), ctypes.byref(rl2),
                                       ctypes.byref(outer), ctypes.byref(stat))
    if n < 0:
        raise ValueError("bad argument")
    k = min(cnt.value, cap)
    return dict(u=u, u_lo=ulo, sweeps=n, outer=outer.value, err=err.value, rel_l2=rl2.value,
                status=STATUS[stat.value], tests=cnt.value, history=hist[:2 * k].reshape(k, 2).copy())
