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

from oracle import oracle as orc

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
            # and directly against the oracle's residual of the same arrays
            fh, uh = f.cpu().numpy(), u.cpu().numpy()
            b = orc.scale_rhs(fh)
            s, m = orc.residual(st, uh, b)
            assert got[0] == pytest.approx(np.sqrt(s) / np.linalg.norm(b), rel=1e-12)
            assert got[1] == pytest.approx(m / np.abs(b).max(), rel=1e-14)


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
    """A 2^20 x 129 grid needs 8192 x 3 = 24576 scratch slots, more than the 16384 the scratch
    holds.  The size check comes before any access to f or u, so a small buffer with a
    large row stride stands in for the grid."""
    import torch
    from paper_1705_00103_gb300.cj import _lib
    f = torch.zeros((2, 2), dtype=torch.float64, device="cuda")
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    nx = 1 << 20
    rc = _lib().cj_residual_noalloc(nx, 129, 5, f.data_ptr(), nx, f.data_ptr(), nx,
                                    out.data_ptr(), None)
    assert rc == cj.CJ_ERR_INVALID_ARG
    assert "limit" in _lib().cj_last_error().decode()
    assert float(out.abs().sum()) == 0.0


def test_noalloc_at_full_scratch_capacity(cj):
    """A 16384 x 8192 grid needs exactly the 16384 slots the scratch holds (128 x 128 blocks of
    128 x 64 nodes): it is accepted and its norms equal the plan-based ones, twice in a row."""
    import torch
    Nx, Ny, st = 16384, 8192, 5
    g = torch.Generator(device="cuda").manual_seed(7)
    f = torch.randn((Ny, Nx), dtype=torch.float64, device="cuda", generator=g)
    u = torch.randn((Ny, Nx), dtype=torch.float64, device="cuda", generator=g)
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    with cj.Plan(Nx, Ny, st, 1e-6) as p:
        ref = cj.cj_residual(p.handle, f, u)
    for _ in range(2):
        out.zero_()
        cj.cj_residual_noalloc(Nx, Ny, st, f, u, out)
        torch.cuda.synchronize()
        np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=1e-12, atol=0)


def test_noalloc_keeps_a_nan_in_both_norms(cj):
    import torch
    Nx, Ny = 200, 90
    rng = np.random.default_rng(3)
    f = torch.from_numpy(rng.standard_normal((Ny, Nx))).cuda()
    u = torch.from_numpy(rng.standard_normal((Ny, Nx))).cuda()
    u[40, 150] = float("nan")
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    cj.cj_residual_noalloc(Nx, Ny, 9, f, u, out)
    got = out.cpu().numpy()
    assert np.isnan(got[0]) and np.isnan(got[1])
