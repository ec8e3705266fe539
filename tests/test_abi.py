"""CPU checks of the C-ABI library: it builds, loads, exports every declared entry point,
and rejects invalid arguments before touching the GPU."""
import ctypes
import os
import re
import numpy as np

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "cj.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(cj_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1705_00103_gb300 import build
    return ctypes.CDLL(build.build())


def test_header_declares_the_boundary():
    names = _declared_functions()
    for n in ("cj_plan_create", "cj_plan_destroy", "cj_plan_info", "cj_solve", "cj_solve_host",
              "cj_solve_history", "cj_solution_lo", "cj_set_boundary", "cj_solve_to_error", "cj_plan_create_mask", "cj_autotune_depth",
              "cj_solve_batch", "cj_server_create", "cj_submit", "cj_poll",
              "cj_sweeps", "cj_sweeps_f32", "cj_residual", "cj_status_string", "cj_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_library_is_built_for_sm_103a():
    from paper_1705_00103_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)


def test_invalid_arguments_rejected_without_gpu():
    import paper_1705_00103_gb300 as cj
    bad = [dict(Nx=0, Ny=4, st=5, tol=1e-6), dict(Nx=4, Ny=-1, st=5, tol=1e-6),
           dict(Nx=4, Ny=4, st=7, tol=1e-6), dict(Nx=4, Ny=4, st=9, tol=0.0),
           dict(Nx=4, Ny=4, st=9, tol=1.0), dict(Nx=4, Ny=4, st=17, tol=1e-6, inner_cycle=12),
           dict(Nx=4, Ny=4, st=17, tol=1e-6, precision=4), dict(Nx=4, Ny=4, st=5, tol=1e-6, bc=2),
           dict(Nx=4, Ny=4, st=9, tol=1e-6, method=3),
           dict(Nx=4, Ny=4, st=9, tol=1e-6, method=1, precision=2), dict(Nx=4, Ny=4, st=9, tol=1e-6, launch=4),
           dict(Nx=(1 << 20) + 1, Ny=1, st=5, tol=1e-6), dict(Nx=1, Ny=(1 << 20) + 1, st=9, tol=1e-6)]
    for kw in bad:
        with pytest.raises(cj.CJError) as ei:
            cj.cj_plan_create(**kw)
        assert ei.value.status == cj.CJ_ERR_INVALID_ARG, kw


def test_null_plan_rejected(lib):
    lib.cj_solve.restype = ctypes.c_int
    assert lib.cj_solve(None, None, 0, None, 0, None, None) == -1
    lib.cj_plan_destroy(None)


def test_status_strings(lib):
    lib.cj_status_string.restype = ctypes.c_char_p
    assert lib.cj_status_string(0) == b"converged"
    assert lib.cj_status_string(1).startswith(b"stopped at")
    assert lib.cj_status_string(-6) == b"CUDA error"


def test_dirichlet_ring_layout_matches_the_oracle():
    """The binding's ring builder puts g(i, j) where the oracle's data array has it."""
    import paper_1705_00103_gb300 as cj
    from oracle import oracle as orc
    import workloads
    for Nx, Ny in [(1, 1), (5, 3), (17, 9)]:
        _, _, g = workloads.paper_problem(Nx, Ny)
        np.testing.assert_array_equal(cj.dirichlet_ring(Nx, Ny, g), orc.ghost_ring(Nx, Ny, g))


def test_batch_server_and_mask_arguments_rejected_without_gpu(lib):
    """Entry points check their arguments before any CUDA call: no GPU is needed to see the
    rejections."""
    I = ctypes.c_int
    lib.cj_solve_batch.restype = I
    assert lib.cj_solve_batch(None, 0, None, None) == -1
    lib.cj_server_create.restype = I
    out = ctypes.c_void_p()
    assert lib.cj_server_create(ctypes.c_size_t(0), 4, ctypes.byref(out)) == -1
    assert lib.cj_server_create(ctypes.c_size_t(1 << 30), 0, ctypes.byref(out)) == -1
    lib.cj_submit.restype = I
    t = ctypes.c_uint64()
    assert lib.cj_submit(None, 8, 8, 5, ctypes.c_double(1e-6), None, ctypes.byref(t)) == -1
    lib.cj_poll.restype = I
    assert lib.cj_poll(None, ctypes.c_uint64(1), None, None) == -1
    lib.cj_plan_create_mask.restype = I
    h = ctypes.c_void_p()
    assert lib.cj_plan_create_mask(8, 8, None, ctypes.c_double(1e-6), None, ctypes.byref(h)) == -1
    lib.cj_autotune_engine.restype = I
    assert lib.cj_autotune_engine(0, 8, 5, None, None, None) == -1
    assert lib.cj_autotune_engine(8, 8, 7, None, None, None) == -1
    lib.cj_set_boundary.restype = I
    assert lib.cj_set_boundary(None, None, ctypes.c_longlong(0), None) == -1
    lib.cj_solve_to_error.restype = I
    assert lib.cj_solve_to_error(None, None, ctypes.c_longlong(0), None, ctypes.c_longlong(0), None,
                                 ctypes.c_longlong(0), ctypes.c_double(0.0), ctypes.c_longlong(0), None,
                                 None, None, None, 0, None) == -1


class _FakeCuda:
    """Stands in for a CUDA float64 tensor in the binding's argument checks (no GPU here)."""
    is_cuda = True
    dtype = "torch.float64"

    def __init__(self, shape, device=0):
        self.shape = shape
        self.device = type("dev", (), {"index": device})()

    def dim(self):
        return len(self.shape)

    def stride(self, k):
        return (self.shape[1], 1)[k] if len(self.shape) == 2 else 1

    def data_ptr(self):
        return 64

    def numel(self):
        n = 1
        for s in self.shape:
            n *= s
        return n

    def is_contiguous(self):
        return True

    def __str__(self):
        return "fake"


def test_noalloc_binding_rejects_mismatched_tensors_before_any_launch(monkeypatch):
    """The Python binding of cj_residual_noalloc refuses, with ValueError and before the library
    is called, tensors smaller than the Nx x Ny grid it is told about and tensors on another
    device than the current one."""
    import paper_1705_00103_gb300.cj as cjm

    def no_call():
        raise AssertionError("the library was called")
    monkeypatch.setattr(cjm, "_lib", no_call)
    monkeypatch.setattr(cjm, "_grid", lambda t, name: (t.data_ptr(), t.shape[1]))
    out = _FakeCuda((3,))
    ok = _FakeCuda((20, 30))
    assert cjm._noalloc_args(30, 20, ok, ok, out, current_device=0) == (64, 30, 64, 30)
    for f, u in ((_FakeCuda((19, 30)), ok), (ok, _FakeCuda((20, 29))), (_FakeCuda((20, 8)), ok)):
        with pytest.raises(ValueError):
            cjm.cj_residual_noalloc(30, 20, 9, f, u, out, stream=0)
    with pytest.raises(ValueError):
        cjm._noalloc_args(30, 20, ok, _FakeCuda((20, 30), device=1), out, current_device=0)
    with pytest.raises(ValueError):
        cjm._noalloc_args(30, 20, ok, ok, _FakeCuda((3,), device=1), current_device=0)


def test_noalloc_rejects_sizes_without_gpu(lib):
    """Sides beyond 2^20 and grids needing more than the 16384 scratch slots (here 2^20 x 129:
    8192 x 3 blocks) are refused before the scratch or the arrays are touched."""
    fn = lib.cj_residual_noalloc
    fn.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_longlong,
                   ctypes.c_void_p, ctypes.c_longlong, ctypes.c_void_p, ctypes.c_void_p]
    lib.cj_last_error.restype = ctypes.c_char_p
    p = ctypes.c_void_p(64)
    for Nx, Ny in (((1 << 20) + 1, 1), (1, (1 << 20) + 1), ((1 << 31) - 1, 1), (0, 4), (4, 0)):
        assert fn(Nx, Ny, 5, p, max(Nx, 1), p, max(Nx, 1), p, None) == -1, (Nx, Ny)
    assert fn(1 << 20, 129, 9, p, 1 << 20, p, 1 << 20, p, None) == -1
    assert b"limit" in lib.cj_last_error()
