"""The allocation-free residual entry point, against the plan-based one.

cj_residual_noalloc exists for callers that cannot allocate device memory (a framework's
caching allocator owns the device, or a latency-critical loop must not synchronise on
cudaMalloc).  It keeps its block partial sums in a fixed static device array shared by all
calls; this file checks, through the C ABI, that two calls in a row give the norms the
plan-based cj_residual gives, within the tolerance of the other residual tests, and that
oversized grids are refused.  It is named to be collected last.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cj():
    import paper_1705_00103_gb300 as cj
    cj.build.build()
    return cj


@pytest.mark.parametrize("st", (5, 9, 17))
def test_noalloc_matches_plan_residual_twice(cj, st):
    import torch
    Nx, Ny = 300, 131
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    with cj.Plan(Nx, Ny, st, 1e-8) as p:
        for call in range(2):
            rng = np.random.default_rng(100 * st + call)
            f = torch.from_numpy(rng.standard_normal((Ny, Nx))).cuda()
            u = torch.from_numpy(rng.standard_normal((Ny, Nx)) * (1 + call)).cuda()
            ref = cj.cj_residual(p.handle, f, u)
            cj.cj_residual_noalloc(Nx, Ny, st, f, u, out)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            np.testing.assert_allclose(got, ref, rtol=1e-12, atol=0)


def test_noalloc_strided_and_tiny(cj):
    import torch
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    for Nx, Ny, ld in ((1, 1, 1), (45, 20, 64)):
        rng = np.random.default_rng(Nx)
        fb = torch.from_numpy(rng.standard_normal((Ny, ld))).cuda()
        ub = torch.from_numpy(rng.standard_normal((Ny, ld))).cuda()
        with cj.Plan(Nx, Ny, 17, 1e-8) as p:
            ref = cj.cj_residual(p.handle, fb[:, :Nx], ub[:, :Nx])
        cj.cj_residual_noalloc(Nx, Ny, 17, fb[:, :Nx], ub[:, :Nx], out)
        np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=1e-12, atol=0)


def test_noalloc_rejects_grids_beyond_its_scratch(cj):
    """16385 column blocks of one row strip need one slot more than the 16384 the scratch
    holds.  The size check comes before any access to f or u, so a small buffer with a
    large row stride stands in for the grid."""
    import torch
    from paper_1705_00103_gb300.cj import _lib
    f = torch.zeros((2, 2), dtype=torch.float64, device="cuda")
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    nx = 16385 * 128
    rc = _lib().cj_residual_noalloc(nx, 1, 5, f.data_ptr(), nx, f.data_ptr(), nx,
                                    out.data_ptr(), None)
    assert rc == cj.CJ_ERR_INVALID_ARG
    assert "limit" in _lib().cj_last_error().decode()
    assert float(out.abs().sum()) == 0.0
