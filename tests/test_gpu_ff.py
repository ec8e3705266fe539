"""GPU accuracy of the float-float sweeps (cj_sweeps_ff) against the FP64 oracle, through the C ABI.

The float-float sweep evaluates the sweep of Sec. 2.1 with 48-bit pairs of floats (17 points in the
FP64 sweep's order, 5 and 9 points in an algebraically equal scaled form), so it is not bit-equal
to the FP64 sweep; each sweep is held to

    |got - ref| <= 1e-12 x (max|u| + |w| (S max|u| + max|b|))

node by node, S = 9 bounding the sum of the stencil's absolute coefficients (8, 6.67 and 8.89):
the terms the sweep adds, each carried to about 2^-47 of its size (1e-12 is 140 x 2^-47).  Each
sweep starts from the oracle's own iterate, so the bound is per sweep, not an accumulation.
"""
import numpy as np
import pytest

from oracle import oracle as orc
import workloads

pytestmark = pytest.mark.gpu

STENCILS = (5, 9, 17)
SHAPES = [(1, 1), (1, 7), (6, 1), (3, 5), (17, 9), (130, 70), (257, 131), (300, 64)]
S = 9.0
REL = 1e-12


@pytest.fixture(scope="module")
def cj():
    import paper_1705_00103_gb300 as cj
    cj.build.build()
    return cj


@pytest.fixture(scope="module")
def torch():
    import torch
    return torch


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def bound(u, b, w):
    umax = float(np.max(np.abs(u)))
    bmax = float(np.max(np.abs(b)))
    return REL * (umax + abs(w) * (S * umax + bmax))


def positions(w):
    """Weight positions that include the largest and smallest weights and both ends."""
    M = len(w)
    return sorted({0, 1 % M, M // 2, M - 1, int(np.argmax(w)), int(np.argmin(w))})


def check_one(cj, torch, p, st, u, f, b, k, w):
    fd, ud = dev(torch, f), dev(torch, u)
    cj.cj_sweeps_ff(p.handle, fd, ud, k, 1)
    got = ud.cpu().numpy()
    ref = orc.sweep(st, u, b, w[k])
    err = float(np.max(np.abs(got - ref)))
    tol = bound(u, b, w[k])
    assert np.all(np.isfinite(got))
    assert err <= tol, "sweep at weight %d: %.3g > %.3g" % (k, err, tol)
    return err, tol


@pytest.mark.parametrize("st", STENCILS)
@pytest.mark.parametrize("Nx,Ny", SHAPES)
def test_ff_sweep_within_the_fp64_bound(cj, torch, st, Nx, Ny):
    """One float-float sweep at each of several weight positions against the FP64 sweep."""
    rng = np.random.default_rng(100 * Nx + Ny + st)
    f, u = rng.standard_normal((Ny, Nx)), rng.standard_normal((Ny, Nx))
    b = orc.scale_rhs(f)
    with cj.Plan(Nx, Ny, st, 1e-10) as p:
        w = p.info()["w"]
        for k in positions(w):
            check_one(cj, torch, p, st, u, f, b, k, w)


@pytest.mark.parametrize("st", STENCILS)
def test_ff_sweeps_sweep_by_sweep(cj, torch, st):
    """Twelve consecutive sweeps, each started from the oracle's iterate of the sweep before."""
    Nx, Ny = 203, 77
    rng = np.random.default_rng(st)
    f, u = rng.standard_normal((Ny, Nx)), np.zeros((Ny, Nx))
    b = orc.scale_rhs(f)
    with cj.Plan(Nx, Ny, st, 1e-10) as p:
        w = p.info()["w"]
        for k in range(min(12, len(w))):
            check_one(cj, torch, p, st, u, f, b, k, w)
            u = orc.sweep(st, u, b, w[k])


S_ABS = {5: 8.0, 9: 40.0 / 6.0, 17: 640.0 / 72.0}


def growth(M):
    """Growth of the partial products of a cycle of M mirror-paired weights, as measured for the
    inner-cycle planner: 10^(2.6 + 0.62 log2(M / 512))."""
    return 10.0 ** (2.6 + 0.62 * np.log2(M / 512.0))


def ff_and_fp64_cycle(cj, torch, st, tol):
    Nx, Ny = 96, 80
    f = workloads.smooth_random_rhs(Nx, Ny, 7)
    u0 = np.zeros((Ny, Nx))
    b = orc.scale_rhs(f)
    with cj.Plan(Nx, Ny, st, tol) as p:
        w = p.info()["w"]
        fd, ud = dev(torch, f), dev(torch, u0)
        cj.cj_sweeps_ff(p.handle, fd, ud, 0, len(w))
        got = ud.cpu().numpy()
    ref = u0
    for k in range(len(w)):
        ref = orc.sweep(st, ref, b, w[k])
    bn = np.sqrt(orc.residual(st, np.zeros_like(b), b)[0])
    r_ff = np.sqrt(orc.residual(st, got, b)[0]) / bn
    r_64 = np.sqrt(orc.residual(st, ref, b)[0]) / bn
    fl = 2.0 ** -53 * S_ABS[st] * np.linalg.norm(ref) / bn
    return got, ref, r_ff, r_64, fl, len(w)


@pytest.mark.parametrize("st", STENCILS)
@pytest.mark.parametrize("tol", (1e-4, 1e-10))
def test_ff_cycle_matches_fp64_to_its_rounding_floor(cj, torch, st, tol):
    """A whole cycle in one call: the float-float residual differs from the FP64 cycle's by no more
    than 1 % plus the cycle's rounding floor at 48 bits -- 2^6 times the FP64 array floor
    2^-53 S ||u|| / ||b||, amplified by the growth of the cycle's partial products -- far below
    the FP32 level, and the iterates agree to 1e-9 of max |u|."""
    got, ref, r_ff, r_64, fl, M = ff_and_fp64_cycle(cj, torch, st, tol)
    dev_max = float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
    assert abs(r_ff - r_64) <= 0.01 * r_64 + 64 * growth(M) * fl, (r_ff, r_64, fl, M, dev_max)
    assert r_ff < max(tol, 1e-8)
    assert dev_max <= 1e-9, (r_ff, r_64, dev_max)


def test_ff_full_size_sweeps(cj, torch):
    """Two float-float sweeps of the 4096^2 9-point problem in the solver's launch configuration,
    against the oracle on the whole grid (the first from the oracle's input, the second from
    the oracle's first iterate)."""
    N, st = 4096, 9
    f = workloads.smooth_random_rhs(N, N, 1)
    b = orc.scale_rhs(f)
    u = np.zeros((N, N))
    with cj.Plan(N, N, st, 1e-10) as p:
        w = p.info()["w"]
        for k in (0, int(np.argmax(w))):
            check_one(cj, torch, p, st, u, f, b, k, w)
            u = orc.sweep(st, u, b, w[k])


def test_ff_host_arrays_and_strided_rows(cj, torch):
    """Host (NumPy) arrays and caller rows with ld > Nx: only the Nx x Ny nodes are written."""
    Nx, Ny, ld, st = 45, 20, 64, 9
    rng = np.random.default_rng(3)
    f, u = rng.standard_normal((Ny, Nx)), rng.standard_normal((Ny, Nx))
    fbig = np.full((Ny, ld), 7.0)
    ubig = np.full((Ny, ld), -3.0)
    fbig[:, :Nx] = f
    ubig[:, :Nx] = u
    fd = dev(torch, fbig)[:, :Nx]
    ud = dev(torch, ubig)
    with cj.Plan(Nx, Ny, st, 1e-8) as p:
        w = p.info()["w"]
        cj.cj_sweeps_ff(p.handle, fd, ud[:, :Nx], 2, 1)
    got = ud.cpu().numpy()
    np.testing.assert_array_equal(got[:, Nx:], -3.0)
    b = orc.scale_rhs(f)
    ref = orc.sweep(st, u, b, w[2])
    assert np.max(np.abs(got[:, :Nx] - ref)) <= bound(u, b, w[2])


def test_ff_argument_checks(cj, torch):
    """FP32-inner, Dirichlet-data and mask plans and a negative first weight are refused."""
    Nx, Ny = 32, 24
    f = dev(torch, np.ones((Ny, Nx)))
    u = dev(torch, np.zeros((Ny, Nx)))
    with cj.Plan(Nx, Ny, 9, 1e-8, precision=cj.CJ_FP32_INNER) as p:
        with pytest.raises(cj.CJError):
            cj.cj_sweeps_ff(p.handle, f, u, 0, 1)
    with cj.Plan(Nx, Ny, 9, 1e-8, bc=cj.CJ_BC_DIRICHLET) as p:
        with pytest.raises(cj.CJError):
            cj.cj_sweeps_ff(p.handle, f, u, 0, 1)
    with cj.Plan(Nx, Ny, 9, 1e-8) as p:
        with pytest.raises(cj.CJError):
            cj.cj_sweeps_ff(p.handle, f, u, -1, 1)
        cj.cj_sweeps_ff(p.handle, f, u, 0, 0)
        assert float(u.abs().max()) == 0.0
