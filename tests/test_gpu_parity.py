"""GPU parity of libcj against the FP64 CPU oracle, through the C ABI.

The sweep, the FP32 inner sweep and the whole FP64 / mixed solves evaluate the same
arithmetic in the same order on both sides, so they are compared bit for bit (integer
counters too).  Residual norms are sums reduced in a different order on each side and are
compared to 1e-12 relative.
"""
import numpy as np
import pytest

from oracle import oracle as orc
import workloads

pytestmark = pytest.mark.gpu

STENCILS = (5, 9, 17)
# sizes that span several 128-column blocks and row strips, with ragged tails
SHAPES = [(1, 1), (1, 7), (6, 1), (3, 5), (17, 9), (130, 70), (257, 131), (300, 64)]


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


def rand_problem(Nx, Ny, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((Ny, Nx)), rng.standard_normal((Ny, Nx))


# ----------------------------------------------------------------- plan

@pytest.mark.parametrize("st", STENCILS)
@pytest.mark.parametrize("Nx,Ny,tol", [(64, 64, 1e-10), (1, 1, 1e-6), (100, 37, 1e-8),
                                       (4096, 4096, 1e-10), (8192, 8192, 1e-10)])
def test_plan_matches_oracle(cj, st, Nx, Ny, tol):
    with cj.Plan(Nx, Ny, st, tol) as p:
        info = p.info()
    kmin, kmax = orc.kappa_bounds(st, Nx, Ny)
    assert info["kmin"] == kmin and info["kmax"] == kmax
    M = orc.cycle_length(kmin, kmax, tol)
    assert info["M"] == M
    np.testing.assert_array_equal(info["w"], orc.sweep_coeffs(st, kmin, kmax, M))


def test_plan_literal_n_option(cj):
    with cj.Plan(63, 63, 9, 1e-8, literal_n=1) as p:
        info = p.info()
    assert info["kmin"] == orc.kappa_bounds(9, 63, 63, literal_n=True)[0]


# ----------------------------------------------------------------- sweeps

@pytest.mark.parametrize("st", STENCILS)
@pytest.mark.parametrize("Nx,Ny", SHAPES)
def test_fp64_sweeps_bit_exact(cj, torch, st, Nx, Ny):
    """Each of the first sweeps of a cycle equals the oracle's bit for bit."""
    f, u0 = rand_problem(Nx, Ny, 10 * Nx + Ny + st)
    with cj.Plan(Nx, Ny, st, 1e-8) as p:
        w = p.info()["w"]
        fd = dev(torch, f)
        ud = dev(torch, u0)
        b = orc.scale_rhs(f)
        ref = u0.copy()
        nsw = min(6, len(w))
        for k in range(nsw):
            cj.cj_sweeps(p.handle, fd, ud, k, 1)
            ref = orc.sweep(st, ref, b, w[k])
            got = ud.cpu().numpy()
            np.testing.assert_array_equal(got, ref, err_msg="sweep %d" % k)


@pytest.mark.parametrize("st", STENCILS)
def test_fp64_sweeps_batched_launches(cj, torch, st):
    """Many sweeps in one call (ping-pong inside the library) equal the oracle's."""
    Nx, Ny = 203, 77
    f, u0 = rand_problem(Nx, Ny, st)
    with cj.Plan(Nx, Ny, st, 1e-6) as p:
        w = p.info()["w"]
        fd, ud = dev(torch, f), dev(torch, u0)
        count = min(33, len(w))
        cj.cj_sweeps(p.handle, fd, ud, 0, count)
        b = orc.scale_rhs(f)
        ref = u0.copy()
        for k in range(count):
            ref = orc.sweep(st, ref, b, w[k])
        np.testing.assert_array_equal(ud.cpu().numpy(), ref)


def test_fp64_sweeps_strided_caller_arrays(cj, torch):
    """Caller rows with ld > Nx are read and written at the right places only."""
    Nx, Ny, ld = 45, 20, 64
    f, u0 = rand_problem(Nx, Ny, 3)
    fbig = np.full((Ny, ld), 7.0)
    ubig = np.full((Ny, ld), -3.0)
    fbig[:, :Nx] = f
    ubig[:, :Nx] = u0
    with cj.Plan(Nx, Ny, 17, 1e-8) as p:
        w = p.info()["w"]
        fd, ud = dev(torch, fbig), dev(torch, ubig)
        cj.cj_sweeps(p.handle, fd[:, :Nx], ud[:, :Nx], 0, 3)
        ref = u0.copy()
        b = orc.scale_rhs(f)
        for k in range(3):
            ref = orc.sweep(17, ref, b, w[k])
        got = ud.cpu().numpy()
        np.testing.assert_array_equal(got[:, :Nx], ref)
        assert np.all(got[:, Nx:] == -3.0)


@pytest.mark.parametrize("st", STENCILS)
@pytest.mark.parametrize("Nx,Ny", [(1, 1), (5, 3), (130, 70), (257, 131)])
def test_fp32_sweeps_bit_exact(cj, torch, st, Nx, Ny):
    rng = np.random.default_rng(Nx + Ny + st)
    r = rng.standard_normal((Ny, Nx)).astype(np.float32)
    e = rng.standard_normal((Ny, Nx)).astype(np.float32)
    with cj.Plan(Nx, Ny, st, 1e-8, precision=cj.CJ_FP32_INNER, inner_cycle=16) as p:
        kmin, kmax = orc.kappa_bounds(st, Nx, Ny)
        w32 = orc.sweep_coeffs(st, kmin, kmax, 16).astype(np.float32)
        rd, ed = dev(torch, r), dev(torch, e)
        ref = e.copy()
        for k in range(5):
            cj.cj_sweeps_f32(p.handle, rd, ed, k, 1)
            ref = orc.sweep_f32(st, ref, r, w32[k])
            np.testing.assert_array_equal(ed.cpu().numpy(), ref, err_msg="sweep %d" % k)


# ----------------------------------------------------------------- residual

@pytest.mark.parametrize("st", STENCILS)
@pytest.mark.parametrize("Nx,Ny", [(1, 1), (17, 9), (300, 64)])
def test_residual_norms(cj, torch, st, Nx, Ny):
    f, u = rand_problem(Nx, Ny, 5 + st)
    with cj.Plan(Nx, Ny, st, 1e-8) as p:
        l2, linf, fl = cj.cj_residual(p.handle, dev(torch, f), dev(torch, u))
    b = orc.scale_rhs(f)
    s, m = orc.residual(st, u, b)
    assert l2 == pytest.approx(np.sqrt(s) / np.linalg.norm(b), rel=1e-12)
    assert linf == pytest.approx(m / np.abs(b).max(), rel=1e-14)
    assert fl == pytest.approx(2.0 ** -53 * orc.abs_coeff_sum(st) * np.linalg.norm(u) / np.linalg.norm(b),
                               rel=1e-12)


# ----------------------------------------------------------------- solves

@pytest.mark.parametrize("st", STENCILS)
@pytest.mark.parametrize("Nx,Ny,tol,kind", [(64, 64, 1e-10, "man"), (48, 40, 1e-10, "rnd"),
                                            (1, 1, 1e-10, "rnd"), (97, 33, 1e-8, "rnd"),
                                            (48, 40, 1e-15, "rnd")])
def test_fp64_solve_matches_oracle(cj, torch, st, Nx, Ny, tol, kind):
    f = workloads.manufactured_rhs(Nx, Ny) if kind == "man" else workloads.smooth_random_rhs(Nx, Ny, 2)
    ref = orc.solve(st, f, tol)
    with cj.Plan(Nx, Ny, st, tol) as p:
        ud = torch.zeros((Ny, Nx), dtype=torch.float64, device="cuda")
        res = cj.cj_solve(p.handle, dev(torch, f), ud)
    assert res["sweeps"] == ref["sweeps"] and res["cycles"] == ref["cycles"]
    assert {0: "converged", 1: "floor", 3: "stalled"}[res["status"]] == ref["status"]
    np.testing.assert_array_equal(ud.cpu().numpy(), ref["u"])
    assert res["rel_res_l2"] == pytest.approx(ref["rel_l2"], rel=1e-10)


def test_fp64_solve_warm_start(cj, torch):
    Nx, Ny, st = 70, 50, 9
    f = workloads.smooth_random_rhs(Nx, Ny, 4)
    u0 = np.random.default_rng(1).standard_normal((Ny, Nx)) * 1e-3
    ref = orc.solve(st, f, 1e-9, u0=u0)
    with cj.Plan(Nx, Ny, st, 1e-9) as p:
        ud = dev(torch, u0)
        res = cj.cj_solve(p.handle, dev(torch, f), ud)
    assert res["sweeps"] == ref["sweeps"]
    np.testing.assert_array_equal(ud.cpu().numpy(), ref["u"])


def test_fp64_solve_host_arrays(cj, torch):
    Nx, Ny, st = 64, 64, 5
    f = workloads.manufactured_rhs(Nx, Ny)
    ref = orc.solve(st, f, 1e-10)
    with cj.Plan(Nx, Ny, st, 1e-10) as p:
        u = np.zeros((Ny, Nx))
        res = cj.cj_solve_host(p.handle, np.ascontiguousarray(f), u)
    assert res["rc"] == cj.CJ_OK and res["sweeps"] == ref["sweeps"]
    np.testing.assert_array_equal(u, ref["u"])


def test_zero_rhs(cj, torch):
    with cj.Plan(9, 7, 17, 1e-10) as p:
        ud = torch.zeros((7, 9), dtype=torch.float64, device="cuda")
        res = cj.cj_solve(p.handle, torch.zeros_like(ud), ud)
    assert res["rc"] == cj.CJ_OK and res["sweeps"] == 0 and float(ud.abs().max()) == 0.0


def test_sweep_budget_exhausted(cj, torch):
    Nx, Ny = 40, 40
    f = workloads.smooth_random_rhs(Nx, Ny, 1)
    with cj.Plan(Nx, Ny, 5, 1e-10, max_sweeps=10) as p:
        ud = torch.zeros((Ny, Nx), dtype=torch.float64, device="cuda")
        res = cj.cj_solve(p.handle, dev(torch, f), ud)
    assert res["rc"] == cj.CJ_ERR_NOT_CONVERGED and res["sweeps"] == 0


@pytest.mark.parametrize("st", STENCILS)
@pytest.mark.parametrize("Nx,Ny,M_in", [(48, 40, 64), (130, 70, 128), (1, 1, 1)])
def test_mixed_solve_matches_oracle(cj, torch, st, Nx, Ny, M_in):
    f = workloads.smooth_random_rhs(Nx, Ny, 6)
    ref = orc.solve_mixed(st, f, 1e-10, M_in)
    with cj.Plan(Nx, Ny, st, 1e-10, precision=cj.CJ_FP32_INNER, inner_cycle=M_in) as p:
        ud = torch.zeros((Ny, Nx), dtype=torch.float64, device="cuda")
        res = cj.cj_solve(p.handle, dev(torch, f), ud)
    assert res["sweeps"] == ref["sweeps"] and res["cycles"] == ref["outer"]
    np.testing.assert_array_equal(ud.cpu().numpy(), ref["u"])


def test_mixed_solve_auto_inner_cycle_reaches_fp64_solution(cj, torch):
    Nx, Ny, st = 256, 200, 9
    f = workloads.smooth_random_rhs(Nx, Ny, 8)
    with cj.Plan(Nx, Ny, st, 1e-10) as p:
        u64 = torch.zeros((Ny, Nx), dtype=torch.float64, device="cuda")
        r64 = cj.cj_solve(p.handle, dev(torch, f), u64)
    with cj.Plan(Nx, Ny, st, 1e-10, precision=cj.CJ_FP32_INNER) as p:
        um = torch.zeros((Ny, Nx), dtype=torch.float64, device="cuda")
        rm = cj.cj_solve(p.handle, dev(torch, f), um)
    assert r64["rc"] == cj.CJ_OK and rm["rc"] == cj.CJ_OK
    err = float(torch.linalg.norm(um - u64) / torch.linalg.norm(u64))
    assert err < 1e-9


# ----------------------------------------------------------------- full-size cases

@pytest.mark.parametrize("st,N", [(9, 4096), (17, 8192)])
def test_full_size_sweeps_bit_exact(cj, torch, st, N):
    """Two sweeps of the 4096^2 (9-point) and 8192^2 (17-point) problems in the launch
    configuration the solver uses, against the oracle on the whole grid."""
    f = workloads.smooth_random_rhs(N, N, 1)
    u0 = np.zeros((N, N))
    with cj.Plan(N, N, st, 1e-10) as p:
        w = p.info()["w"]
        fd, ud = dev(torch, f), dev(torch, u0)
        cj.cj_sweeps(p.handle, fd, ud, 0, 2)
        got = ud.cpu().numpy()
    b = orc.scale_rhs(f)
    ref = orc.sweep(st, orc.sweep(st, u0, b, w[0]), b, w[1 % len(w)])
    np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("st", (5, 9))
def test_full_size_fp32_temporal_sweeps_bit_exact(cj, torch, st):
    """Nine FP32 inner sweeps of the 4096^2 grid at the solver's default depth for this size (the
    register wavefront, four sweeps per launch, then one), against the oracle's one-sweep-at-a-
    time FP32 sweeps on the whole grid."""
    N = 4096
    rng = np.random.default_rng(17 + st)
    r = rng.standard_normal((N, N)).astype(np.float32)
    e = rng.standard_normal((N, N)).astype(np.float32)
    with cj.Plan(N, N, st, 1e-10, precision=cj.CJ_FP32_INNER, inner_cycle=64) as p:
        kmin, kmax = orc.kappa_bounds(st, N, N)
        w32 = orc.sweep_coeffs(st, kmin, kmax, 64).astype(np.float32)
        ed = dev(torch, e)
        cj.cj_sweeps_f32(p.handle, dev(torch, r), ed, 7, 9)
        got = ed.cpu().numpy()
    ref = e
    for k in range(9):
        ref = orc.sweep_f32(st, ref, r, w32[(7 + k) % 64])
    np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("depth", (1, 2))
def test_full_size_fp32_17_point_8192_sweeps_bit_exact(cj, torch, depth):
    """Five FP32 inner sweeps of the 17-point 8192^2 grid (the high-order workload's hot kernel) at
    depth 1 (one sweep per launch, the default) and depth 2 (the register wavefront), against
    the oracle's one-sweep-at-a-time FP32 sweeps on the whole grid."""
    N, st = 8192, 17
    rng = np.random.default_rng(29 + depth)
    r = rng.standard_normal((N, N)).astype(np.float32)
    e = rng.standard_normal((N, N)).astype(np.float32)
    with cj.Plan(N, N, st, 1e-10, precision=cj.CJ_FP32_INNER, inner_cycle=64, temporal_depth=depth) as p:
        kmin, kmax = orc.kappa_bounds(st, N, N)
        w32 = orc.sweep_coeffs(st, kmin, kmax, 64).astype(np.float32)
        ed = dev(torch, e)
        cj.cj_sweeps_f32(p.handle, dev(torch, r), ed, 3, 5)
        got = ed.cpu().numpy()
    ref = e
    for k in range(5):
        ref = orc.sweep_f32(st, ref, r, w32[(3 + k) % 64])
    np.testing.assert_array_equal(got, ref)


def test_full_size_residual(cj, torch):
    N, st = 4096, 9
    f = workloads.smooth_random_rhs(N, N, 1)
    u = np.random.default_rng(2).standard_normal((N, N)) * 1e-4
    with cj.Plan(N, N, st, 1e-10) as p:
        l2, linf, _ = cj.cj_residual(p.handle, dev(torch, f), dev(torch, u))
    b = orc.scale_rhs(f)
    s, m = orc.residual(st, u, b)
    assert l2 == pytest.approx(np.sqrt(s) / np.linalg.norm(b), rel=1e-12)
    assert linf == pytest.approx(m / np.abs(b).max(), rel=1e-14)


@pytest.mark.parametrize("st,N", [(9, 4096), (17, 4096), (17, 8192)])
def test_full_size_mixed_dd_meets_the_tolerance_by_the_oracle(cj, torch, st, N):
    """The FP32-inner / double-FP64-outer solve to 1e-10 of the 4096^2 problems (9 points: the
    benchmark's problem; 17 points) and of the 17-point 8192^2 high-order problem: its relative
    residual as the oracle evaluates it, the double-FP64 defect of u_hi + u_lo, is within the
    tolerance and agrees with the library's own figure."""
    f = workloads.smooth_random_rhs(N, N, 2)
    with cj.Plan(N, N, st, 1e-10, precision=cj.CJ_FP32_INNER_DD) as p:
        u = torch.zeros((N, N), dtype=torch.float64, device="cuda")
        res = cj.cj_solve(p.handle, dev(torch, f), u)
        lo = torch.zeros_like(u)
        cj.cj_solution_lo(p.handle, lo)
    assert res["rc"] == cj.CJ_OK
    b = orc.scale_rhs(f)
    R = orc.residual_dd(st, u.cpu().numpy(), lo.cpu().numpy(), b)
    rho = np.linalg.norm(R) / np.linalg.norm(b)
    assert rho <= 1e-10
    assert rho == pytest.approx(res["rel_res_l2"], rel=1e-6)


# ----------------------------------------------------------------- double-FP64 outer form

@pytest.mark.parametrize("st", STENCILS)
@pytest.mark.parametrize("prec", [2, 3])
@pytest.mark.parametrize("Nx,Ny,M_in,tol", [(48, 40, 64, 1e-12), (130, 70, 128, 1e-10), (1, 1, 1, 1e-10),
                                            (257, 131, 256, 1e-13)])
def test_mixed_dd_solve_matches_oracle(cj, torch, st, prec, Nx, Ny, M_in, tol):
    """Double-FP64 outer steps with FP32 (prec 2) or FP64 (prec 3, reading R20) inner cycles:
    u_hi, u_lo and the sweep and step counts equal the oracle's bit for bit."""
    f = workloads.smooth_random_rhs(Nx, Ny, 12)
    solve = orc.solve_fp64_dd if prec == 3 else orc.solve_mixed_dd
    ref = solve(st, f, tol, M_in)
    with cj.Plan(Nx, Ny, st, tol, precision=prec, inner_cycle=M_in) as p:
        ud = torch.zeros((Ny, Nx), dtype=torch.float64, device="cuda")
        res = cj.cj_solve(p.handle, dev(torch, f), ud)
        lo = torch.empty_like(ud)
        cj.cj_solution_lo(p.handle, lo)
    assert res["sweeps"] == ref["sweeps"] and res["cycles"] == ref["outer"]
    assert {0: "converged", 1: "floor", 3: "stalled"}[res["status"]] == ref["status"]
    np.testing.assert_array_equal(ud.cpu().numpy(), ref["u"])
    np.testing.assert_array_equal(lo.cpu().numpy(), ref["u_lo"])
    assert res["rel_res_l2"] == pytest.approx(ref["rel_l2"], rel=1e-10)


@pytest.mark.parametrize("st", STENCILS)
def test_mixed_dd_goes_below_fp64_floor(cj, torch, st):
    N, tol = 160, 1e-13
    f = workloads.smooth_random_rhs(N, N, seed=4, kmax=40)
    with cj.Plan(N, N, st, tol, precision=cj.CJ_FP32_INNER, inner_cycle=512) as p:
        ud = torch.zeros((N, N), dtype=torch.float64, device="cuda")
        r32 = cj.cj_solve(p.handle, dev(torch, f), ud)
    with cj.Plan(N, N, st, tol, precision=cj.CJ_FP32_INNER_DD, inner_cycle=512) as p:
        ud = torch.zeros((N, N), dtype=torch.float64, device="cuda")
        rdd = cj.cj_solve(p.handle, dev(torch, f), ud)
    assert r32["rc"] in (cj.CJ_FLOOR, cj.CJ_STALLED) and r32["rel_res_l2"] > tol
    assert (r32["rc"] == cj.CJ_FLOOR) == (r32["rel_res_l2"] <= 4 * r32["floor_est"])
    assert rdd["rc"] == cj.CJ_OK and rdd["rel_res_l2"] <= tol


@pytest.mark.parametrize("st", STENCILS)
def test_fp64_dd_goes_below_where_plain_fp64_stops(cj, torch, st):
    """The all-FP64 path (R20) reaches a tolerance that plain FP64 cycles stall or floor above."""
    N, tol = 160, 1e-13
    f = workloads.smooth_random_rhs(N, N, seed=4, kmax=40)
    with cj.Plan(N, N, st, tol) as p:
        ud = torch.zeros((N, N), dtype=torch.float64, device="cuda")
        plain = cj.cj_solve(p.handle, dev(torch, f), ud)
    with cj.Plan(N, N, st, tol, precision=cj.CJ_FP64_INNER_DD, inner_cycle=512) as p:
        ud = torch.zeros((N, N), dtype=torch.float64, device="cuda")
        rdd = cj.cj_solve(p.handle, dev(torch, f), ud)
    assert plain["rc"] in (cj.CJ_FLOOR, cj.CJ_STALLED) and plain["rel_res_l2"] > tol
    assert rdd["rc"] == cj.CJ_OK and rdd["rel_res_l2"] <= tol


def test_full_size_fp64_dd_meets_the_tolerance_by_the_oracle(cj, torch):
    """The benchmark's FP64-arithmetic solve: 9-point 4096^2 to 1e-10 by FP64 inner cycles in
    double-FP64 defect correction at the planner's inner cycle; its relative residual as the oracle
    evaluates it (the double-FP64 defect of u_hi + u_lo) is within the tolerance and agrees with
    the library's figure; the inner cycle is a power of two no longer than the plan's cycle."""
    N, st = 4096, 9
    f = workloads.smooth_random_rhs(N, N, 1)
    with cj.Plan(N, N, st, 1e-10, precision=cj.CJ_FP64_INNER_DD) as p:
        info = p.info()
        u = torch.zeros((N, N), dtype=torch.float64, device="cuda")
        res = cj.cj_solve(p.handle, dev(torch, f), u)
        lo = torch.zeros_like(u)
        cj.cj_solution_lo(p.handle, lo)
    M_in = info["M_inner"]
    assert M_in & (M_in - 1) == 0 and M_in <= info["M"]
    assert res["rc"] == cj.CJ_OK and res["sweeps"] == res["cycles"] * M_in
    b = orc.scale_rhs(f)
    R = orc.residual_dd(st, u.cpu().numpy(), lo.cpu().numpy(), b)
    rho = np.linalg.norm(R) / np.linalg.norm(b)
    assert rho <= 1e-10
    assert rho == pytest.approx(res["rel_res_l2"], rel=1e-6)


def test_solution_lo_rejected_for_fp64_plans(cj, torch):
    with cj.Plan(8, 8, 5, 1e-8) as p:
        with pytest.raises(cj.CJError):
            cj.cj_solution_lo(p.handle, torch.zeros((8, 8), dtype=torch.float64, device="cuda"))


# ----------------------------------------------------------------- temporal blocking

@pytest.mark.parametrize("st", STENCILS)
@pytest.mark.parametrize("depth", [2, 3, 4, 8])
@pytest.mark.parametrize("Nx,Ny", [(1, 1), (5, 3), (2, 40), (130, 70), (257, 33), (300, 97)])
def test_fp32_temporal_blocking_bit_exact(cj, torch, st, depth, Nx, Ny):
    """depth sweeps per launch equal one sweep per launch bit for bit, over counts that are
    not multiples of the depth and tiles cut by the grid's edges."""
    rng = np.random.default_rng(7 * Nx + Ny + st + depth)
    r = rng.standard_normal((Ny, Nx)).astype(np.float32)
    e = rng.standard_normal((Ny, Nx)).astype(np.float32)
    count = 2 * depth + 1
    with cj.Plan(Nx, Ny, st, 1e-8, precision=cj.CJ_FP32_INNER, inner_cycle=32,
                 temporal_depth=depth) as p:
        kmin, kmax = orc.kappa_bounds(st, Nx, Ny)
        w32 = orc.sweep_coeffs(st, kmin, kmax, 32).astype(np.float32)
        rd, ed = dev(torch, r), dev(torch, e)
        cj.cj_sweeps_f32(p.handle, rd, ed, 3, count)
    ref = e.copy()
    for k in range(count):
        ref = orc.sweep_f32(st, ref, r, w32[(3 + k) % 32])
    np.testing.assert_array_equal(ed.cpu().numpy(), ref)


@pytest.mark.parametrize("st,depth", [(5, 2), (5, 4), (9, 2), (9, 4), (17, 2)])
@pytest.mark.parametrize("Nx,Ny", [(124, 9), (125, 40), (244, 17), (245, 3), (246, 66), (247, 33), (248, 129),
                                   (369, 250)])
def test_register_wavefront_strip_edges_bit_exact(cj, torch, st, depth, Nx, Ny):
    """The register wavefront kernel's 120-column strips (124 for the first) with the last
    column Nx at every position within a lane's four, one and several strips and row blocks:
    depth sweeps per launch equal the oracle's one-sweep-at-a-time FP32 result bit for bit."""
    rng = np.random.default_rng(3 * Nx + Ny + 11 * st + depth)
    r = rng.standard_normal((Ny, Nx)).astype(np.float32)
    e = rng.standard_normal((Ny, Nx)).astype(np.float32)
    count = 3 * depth
    with cj.Plan(Nx, Ny, st, 1e-8, precision=cj.CJ_FP32_INNER, inner_cycle=64, temporal_depth=depth) as p:
        kmin, kmax = orc.kappa_bounds(st, Nx, Ny)
        w32 = orc.sweep_coeffs(st, kmin, kmax, 64).astype(np.float32)
        ed = dev(torch, e)
        cj.cj_sweeps_f32(p.handle, dev(torch, r), ed, 5, count)
    ref = e.copy()
    for k in range(count):
        ref = orc.sweep_f32(st, ref, r, w32[(5 + k) % 64])
    np.testing.assert_array_equal(ed.cpu().numpy(), ref)


@pytest.mark.parametrize("st", STENCILS)
def test_mixed_solve_with_temporal_blocking_matches_oracle(cj, torch, st):
    Nx, Ny, M_in = 200, 150, 128
    f = workloads.smooth_random_rhs(Nx, Ny, 13)
    ref = orc.solve_mixed_dd(st, f, 1e-11, M_in)
    with cj.Plan(Nx, Ny, st, 1e-11, precision=cj.CJ_FP32_INNER_DD, inner_cycle=M_in,
                 temporal_depth=4) as p:
        ud = torch.zeros((Ny, Nx), dtype=torch.float64, device="cuda")
        res = cj.cj_solve(p.handle, dev(torch, f), ud)
    assert res["sweeps"] == ref["sweeps"] and res["cycles"] == ref["outer"]
    np.testing.assert_array_equal(ud.cpu().numpy(), ref["u"])


# ----------------------------------------------------------------- autotuner, history

def test_autotune_depth_records_the_fastest(cj, torch):
    out = cj.cj_autotune_depth(1024, 1024, 9, sweeps=32)
    rates = out["gupd"]
    assert out["best"] in (1, 2, 4, 8) and all(v > 0 for v in rates.values())
    assert rates[out["best"]] == max(rates.values())


def test_solve_history_records_every_residual_test(cj, torch):
    Nx, Ny, st = 96, 80, 9
    f = workloads.smooth_random_rhs(Nx, Ny, 21)
    with cj.Plan(Nx, Ny, st, 1e-10, precision=cj.CJ_FP32_INNER_DD, inner_cycle=64) as p:
        ud = torch.zeros((Ny, Nx), dtype=torch.float64, device="cuda")
        res = cj.cj_solve_history(p.handle, dev(torch, f), ud)
    h = res["history"]
    assert len(h) == res["cycles"] + 1 and h[0] == pytest.approx(1.0) and h[-1] == res["rel_res_l2"]
    assert res["rc"] == cj.CJ_OK and h[-1] <= 1e-10


# ----------------------------------------------------------------- Dirichlet data (Sec. 3.3)

def _ring(torch, Nx, Ny, g, ld_extra=3):
    G = orc.ghost_ring(Nx, Ny, g)
    Gd = torch.zeros((Ny + 4, Nx + 4 + ld_extra), dtype=torch.float64, device="cuda")
    Gd[:, :Nx + 4] = torch.from_numpy(G).cuda()
    return G, Gd


@pytest.mark.parametrize("st", STENCILS)
@pytest.mark.parametrize("Nx,Ny", [(1, 1), (17, 9), (130, 70)])
def test_dirichlet_data_sweeps_bit_exact(cj, torch, st, Nx, Ny):
    f, _, g = workloads.paper_problem(Nx, Ny)
    u0 = np.random.default_rng(Nx + st).standard_normal((Ny, Nx))
    G, Gd = _ring(torch, Nx, Ny, g)
    with cj.Plan(Nx, Ny, st, 1e-8, bc=cj.CJ_BC_DIRICHLET) as p:
        cj.cj_set_boundary(p.handle, Gd)
        w = p.info()["w"]
        fd, ud = dev(torch, f), dev(torch, u0)
        b = orc.scale_rhs(f)
        ref = u0.copy()
        for k in range(min(5, len(w))):
            cj.cj_sweeps(p.handle, fd, ud, k, 1)
            ref = orc.sweep_bc(st, ref, G, b, w[k])
            np.testing.assert_array_equal(ud.cpu().numpy(), ref, err_msg="sweep %d" % k)


@pytest.mark.parametrize("st", STENCILS)
@pytest.mark.parametrize("N,tol", [(64, 1e-10), (33, 1e-8)])
def test_dirichlet_data_solve_matches_oracle(cj, torch, st, N, tol):
    f, u_exact, g = workloads.paper_problem(N, N)
    G, Gd = _ring(torch, N, N, g)
    ref = orc.solve_bc(st, f, G, tol)
    with cj.Plan(N, N, st, tol, bc=cj.CJ_BC_DIRICHLET) as p:
        cj.cj_set_boundary(p.handle, Gd)
        ud = torch.zeros((N, N), dtype=torch.float64, device="cuda")
        res = cj.cj_solve(p.handle, dev(torch, f), ud)
    assert res["sweeps"] == ref["sweeps"] and res["cycles"] == ref["cycles"]
    np.testing.assert_array_equal(ud.cpu().numpy(), ref["u"])
    # and it is the paper's problem: close to u = -e^{xy}
    assert np.abs(ud.cpu().numpy() - u_exact).max() < 1e-3


def test_dirichlet_data_argument_checks(cj, torch):
    g = torch.zeros((20, 20), dtype=torch.float64, device="cuda")
    with cj.Plan(16, 16, 9, 1e-8) as p:
        with pytest.raises(cj.CJError):
            cj.cj_set_boundary(p.handle, g)
    with cj.Plan(16, 16, 9, 1e-8, bc=cj.CJ_BC_DIRICHLET) as p:
        with pytest.raises(cj.CJError):
            cj.cj_set_boundary(p.handle, g[:, :19])


# ----------------------------------------------------------------- real-error stop (Sec. 3.4)

@pytest.mark.parametrize("st", STENCILS)
@pytest.mark.parametrize("N,every,data", [(40, 0, True), (40, 37, True), (33, 16, False), (1, 0, True)])
def test_solve_to_error_matches_oracle(cj, torch, st, N, every, data):
    if data:
        f, ue, g = workloads.paper_problem(N, N)
        G, Gd = _ring(torch, N, N, g)
        ref_u = orc.solve_bc(st, f, G, 1e-13)["u"]
    else:
        f, ue, G = workloads.manufactured_rhs(N, N), workloads.manufactured_solution(N, N), None
        ref_u = orc.solve(st, f, 1e-13)["u"]
    err_tol = orc.real_error(ref_u, ue) * 1.05 + 1e-9
    ref = orc.solve_to_error(st, f, ue, 1e-4, err_tol, G=G, check_every=every)
    with cj.Plan(N, N, st, 1e-4, bc=cj.CJ_BC_DIRICHLET if data else cj.CJ_BC_DIRICHLET0) as p:
        if data:
            cj.cj_set_boundary(p.handle, Gd)
        ud = torch.zeros((N, N), dtype=torch.float64, device="cuda")
        res = cj.cj_solve_to_error(p.handle, dev(torch, f), ud, dev(torch, ue), err_tol, every)
    assert ref["status"] == "converged" and res["rc"] == cj.CJ_OK
    assert res["sweeps"] == ref["sweeps"] and res["cycles"] == ref["cycles"]
    assert res["tests"] == ref["tests"]
    np.testing.assert_array_equal(res["history"], ref["history"])
    np.testing.assert_array_equal(ud.cpu().numpy(), ref["u"])
    assert res["real_error"] == ref["err"]
    assert res["rel_res_l2"] == pytest.approx(ref["rel_l2"], rel=1e-10)


def test_solve_to_error_goal_below_discretisation_error(cj, torch):
    N, st = 31, 5
    f, ue, g = workloads.paper_problem(N, N)
    G, Gd = _ring(torch, N, N, g)
    disc = orc.real_error(orc.solve_bc(st, f, G, 1e-13)["u"], ue)
    ref = orc.solve_to_error(st, f, ue, 1e-8, disc / 2, G=G)
    with cj.Plan(N, N, st, 1e-8, bc=cj.CJ_BC_DIRICHLET) as p:
        cj.cj_set_boundary(p.handle, Gd)
        ud = torch.zeros((N, N), dtype=torch.float64, device="cuda")
        res = cj.cj_solve_to_error(p.handle, dev(torch, f), ud, dev(torch, ue), disc / 2)
    assert ref["status"] in ("floor", "stalled")
    assert {1: "floor", 3: "stalled"}[res["rc"]] == ref["status"]
    assert res["sweeps"] == ref["sweeps"]
    np.testing.assert_array_equal(ud.cpu().numpy(), ref["u"])


def test_solve_to_error_argument_checks(cj, torch):
    z = torch.zeros((8, 8), dtype=torch.float64, device="cuda")
    with cj.Plan(8, 8, 9, 1e-6, precision=cj.CJ_FP32_INNER) as p:
        with pytest.raises(cj.CJError):
            cj.cj_solve_to_error(p.handle, z, z.clone(), z, 1e-3, check_every=4)
    with cj.Plan(8, 8, 9, 1e-6) as p:
        with pytest.raises(cj.CJError):
            cj.cj_solve_to_error(p.handle, z, z.clone(), z, -1.0)
        with pytest.raises(cj.CJError):
            cj.cj_solve_to_error(p.handle, z, z.clone(), z, 1e-3, check_every=-2)


# ----------------------------------------------------------------- classical Jacobi (Sec. 3.4)

@pytest.mark.parametrize("st", STENCILS)
@pytest.mark.parametrize("Nx,Ny,tol,data", [(30, 21, 1e-6, False), (33, 33, 1e-5, True), (1, 1, 1e-8, False)])
def test_jacobi_solve_matches_oracle(cj, torch, st, Nx, Ny, tol, data):
    if data:
        f, _, g = workloads.paper_problem(Nx, Ny)
        G, Gd = _ring(torch, Nx, Ny, g)
    else:
        f, G = workloads.smooth_random_rhs(Nx, Ny, 8), None
    ref = orc.solve_jacobi(st, f, tol, G=G)
    with cj.Plan(Nx, Ny, st, tol, method=cj.CJ_JACOBI,
                 bc=cj.CJ_BC_DIRICHLET if data else cj.CJ_BC_DIRICHLET0) as p:
        assert set(p.info()["w"]) == {1.0 / orc.centre(st)}
        if data:
            cj.cj_set_boundary(p.handle, Gd)
        ud = torch.zeros((Ny, Nx), dtype=torch.float64, device="cuda")
        res = cj.cj_solve(p.handle, dev(torch, f), ud)
    assert res["sweeps"] == ref["sweeps"] and res["cycles"] == ref["cycles"]
    assert {0: "converged", 1: "floor", 3: "stalled"}[res["status"]] == ref["status"]
    np.testing.assert_array_equal(ud.cpu().numpy(), ref["u"])


def test_jacobi_argument_checks(cj, torch):
    with pytest.raises(cj.CJError):
        cj.cj_plan_create(8, 8, 9, 1e-6, method=2)
    with pytest.raises(cj.CJError):
        cj.cj_plan_create(8, 8, 9, 1e-6, method=cj.CJ_JACOBI, precision=cj.CJ_FP32_INNER)
    z = torch.zeros((8, 8), dtype=torch.float64, device="cuda")
    with cj.Plan(8, 8, 9, 1e-6, method=cj.CJ_JACOBI) as p:
        with pytest.raises(cj.CJError):
            cj.cj_solve_to_error(p.handle, z, z.clone(), z, 1e-3)


# ----------------------------------------------------------------- graph-launched cycles

@pytest.mark.parametrize("st", STENCILS)
@pytest.mark.parametrize("method,data", [(0, False), (0, True), (1, False)])
def test_launch_modes_give_identical_solves(cj, torch, st, method, data):
    """A cycle issued as one launch per sweep, as the CUDA graph of the cycle, or by the automatic
    choice gives the same bits, equal to the oracle's."""
    Nx, Ny, tol = 75, 52, 1e-7
    if data:
        f, _, g = workloads.paper_problem(Nx, Ny)
        G, Gd = _ring(torch, Nx, Ny, g)
        ref = orc.solve_bc(st, f, G, tol)
    else:
        f = workloads.smooth_random_rhs(Nx, Ny, 12)
        ref = orc.solve_jacobi(st, f, tol) if method else orc.solve(st, f, tol)
    outs = []
    for launch in (cj.CJ_LAUNCH_STREAM, cj.CJ_LAUNCH_GRAPH, cj.CJ_LAUNCH_AUTO):
        with cj.Plan(Nx, Ny, st, tol, method=method, launch=launch,
                     bc=cj.CJ_BC_DIRICHLET if data else cj.CJ_BC_DIRICHLET0) as p:
            if data:
                cj.cj_set_boundary(p.handle, Gd)
            ud = torch.zeros((Ny, Nx), dtype=torch.float64, device="cuda")
            res = cj.cj_solve(p.handle, dev(torch, f), ud)
            # a second solve on the same plan replays the graph from the start of the table
            ud2 = torch.zeros_like(ud)
            res2 = cj.cj_solve(p.handle, dev(torch, f), ud2)
        assert res["sweeps"] == res2["sweeps"] == ref["sweeps"]
        assert torch.equal(ud, ud2)
        outs.append(ud.cpu().numpy())
    for u in outs:
        np.testing.assert_array_equal(u, ref["u"])


# ----------------------------------------------------------------- the largest sides

@pytest.mark.parametrize("st", (5, 9))
@pytest.mark.parametrize("Nx,Ny", [(1 << 20, 1), (1, 1 << 20)])
def test_largest_side_sweeps_bit_exact(cj, torch, st, Nx, Ny):
    """Grids at the largest side the plan accepts (2^20 nodes): FP64 sweeps and FP32 sweeps (four
    per launch by the register wavefront, then one) equal the oracle's (a tolerance of 0.5 keeps
    the cycle within the 2^24-sweep limit)."""
    f, u0 = rand_problem(Nx, Ny, 4)
    with cj.Plan(Nx, Ny, st, 0.5, launch=cj.CJ_LAUNCH_STREAM) as p:
        w = p.info()["w"]
        ud = dev(torch, u0)
        cj.cj_sweeps(p.handle, dev(torch, f), ud, 0, 2)
    b = orc.scale_rhs(f)
    ref = orc.sweep(st, orc.sweep(st, u0, b, w[0]), b, w[1 % len(w)])
    np.testing.assert_array_equal(ud.cpu().numpy(), ref)
    r = np.random.default_rng(5).standard_normal((Ny, Nx)).astype(np.float32)
    e0 = np.random.default_rng(6).standard_normal((Ny, Nx)).astype(np.float32)
    with cj.Plan(Nx, Ny, st, 0.5, precision=cj.CJ_FP32_INNER, inner_cycle=4, temporal_depth=4) as p:
        kmin, kmax = orc.kappa_bounds(st, Nx, Ny)
        w32 = orc.sweep_coeffs(st, kmin, kmax, 4).astype(np.float32)
        ed = torch.from_numpy(e0).cuda()
        cj.cj_sweeps_f32(p.handle, torch.from_numpy(r).cuda(), ed, 0, 5)
    ref32 = e0
    for k in range(5):
        ref32 = orc.sweep_f32(st, ref32, r, w32[k % 4])
    np.testing.assert_array_equal(ed.cpu().numpy(), ref32)


@pytest.mark.parametrize("st", STENCILS)
@pytest.mark.parametrize("prec", [1, 2, 3])
@pytest.mark.parametrize("Nx,Ny,M_in", [(40, 33, 32), (130, 70, 64)])
def test_mixed_with_dirichlet_data_matches_oracle(cj, torch, st, prec, Nx, Ny, M_in):
    """FP32 inner cycles in FP64 / double-FP64 defect correction, and FP64 inner cycles in
    double-FP64 defect correction, on the paper's problem with its data ring: every bit of u (and
    u_lo) and the sweep count equal the oracle's."""
    f, _, g = workloads.paper_problem(Nx, Ny)
    G, Gd = _ring(torch, Nx, Ny, g)
    tol = 1e-10
    solve = {1: orc.solve_mixed, 2: orc.solve_mixed_dd, 3: orc.solve_fp64_dd}[prec]
    ref = solve(st, f, tol, M_in, G=G, max_outer=64)
    with cj.Plan(Nx, Ny, st, tol, precision=prec, inner_cycle=M_in, bc=cj.CJ_BC_DIRICHLET) as p:
        cj.cj_set_boundary(p.handle, Gd)
        ud = torch.zeros((Ny, Nx), dtype=torch.float64, device="cuda")
        res = cj.cj_solve(p.handle, dev(torch, f), ud)
        if prec >= 2:
            lo = torch.zeros_like(ud)
            cj.cj_solution_lo(p.handle, lo)
            np.testing.assert_array_equal(lo.cpu().numpy(), ref["u_lo"])
    assert res["sweeps"] == ref["sweeps"] and res["cycles"] == ref["outer"]
    assert {0: "converged", 1: "floor", 3: "stalled"}[res["status"]] == ref["status"]
    np.testing.assert_array_equal(ud.cpu().numpy(), ref["u"])


@pytest.mark.parametrize("st", STENCILS)
@pytest.mark.parametrize("prec,data", [(1, True), (2, True), (3, True), (1, False), (2, False), (3, False)])
def test_mixed_solve_to_error_matches_oracle(cj, torch, st, prec, data):
    """The real-error stop on the defect-correction plans (tested at every outer step): sweeps,
    outer steps, every (sweeps, error) test and the bits of u equal the oracle's."""
    N, M_in = 37, 32
    if data:
        f, ue, g = workloads.paper_problem(N, N)
        G, Gd = _ring(torch, N, N, g)
        disc = orc.real_error(orc.solve_bc(st, f, G, 1e-13)["u"], ue)
    else:
        f, ue, G = workloads.manufactured_rhs(N, N), workloads.manufactured_solution(N, N), None
        disc = orc.real_error(orc.solve(st, f, 1e-13)["u"], ue)
    goal = disc * 1.5 + 1e-12
    ref = orc.solve_mixed_to_error(st, f, ue, goal, M_in, dd=prec - 1, G=G, max_outer=64)
    with cj.Plan(N, N, st, 1e-10, precision=prec, inner_cycle=M_in,
                 bc=cj.CJ_BC_DIRICHLET if data else cj.CJ_BC_DIRICHLET0) as p:
        if data:
            cj.cj_set_boundary(p.handle, Gd)
        ud = torch.zeros((N, N), dtype=torch.float64, device="cuda")
        res = cj.cj_solve_to_error(p.handle, dev(torch, f), ud, dev(torch, ue), goal)
    assert ref["status"] == "converged" and res["rc"] == cj.CJ_OK
    assert res["sweeps"] == ref["sweeps"] and res["cycles"] == ref["outer"] and res["tests"] == ref["tests"]
    np.testing.assert_array_equal(res["history"], ref["history"])
    np.testing.assert_array_equal(ud.cpu().numpy(), ref["u"])
    assert res["real_error"] == ref["err"]


# ----------------------------------------------------------------- whole solves in one cluster

@pytest.mark.parametrize("st", STENCILS)
@pytest.mark.parametrize("Nx,Ny", [(64, 64), (1, 1), (1, 100), (100, 1), (17, 9), (128, 128), (33, 65), (3, 40)])
@pytest.mark.parametrize("method", [0, 1])
def test_cluster_solve_equals_launched_sweeps_and_the_oracle(cj, torch, st, Nx, Ny, method):
    """The single-launch cluster solve (launch 3) gives the bits, sweep count and status of one
    launch per sweep (launch 1) and of the oracle, for CJM and classical Jacobi."""
    f = workloads.smooth_random_rhs(Nx, Ny, 3, kmax=min(20, Nx, Ny))
    tol = 1e-10 if method == 0 else 1e-4
    out = {}
    for launch in (3, 1):
        with cj.Plan(Nx, Ny, st, tol, launch=launch, method=method) as p:
            u = torch.zeros((Ny, Nx), dtype=torch.float64, device="cuda")
            out[launch] = (cj.cj_solve(p.handle, dev(torch, f), u), u.cpu().numpy())
    r3, u3 = out[3]
    r1, u1 = out[1]
    assert r3["launches"] == 4 and (r3["sweeps"], r3["cycles"], r3["rc"]) == (r1["sweeps"], r1["cycles"], r1["rc"])
    np.testing.assert_array_equal(u3, u1)
    assert r3["rel_res_l2"] == pytest.approx(r1["rel_res_l2"], rel=1e-12)
    ref = orc.solve(st, f, tol) if method == 0 else orc.solve_jacobi(st, f, tol)
    assert r3["sweeps"] == ref["sweeps"]
    assert {0: "converged", 1: "floor", 3: "stalled"}[r3["rc"]] == ref["status"]
    np.testing.assert_array_equal(u3, ref["u"])


@pytest.mark.parametrize("st", STENCILS)
def test_cluster_solve_with_dirichlet_data(cj, torch, st):
    N = 90
    f, _, g = workloads.paper_problem(N, N)
    G, Gd = _ring(torch, N, N, g)
    ref = orc.solve_bc(st, f, G, 1e-10)
    for launch in (3, 1):
        with cj.Plan(N, N, st, 1e-10, bc=cj.CJ_BC_DIRICHLET, launch=launch) as p:
            cj.cj_set_boundary(p.handle, Gd)
            u = torch.zeros((N, N), dtype=torch.float64, device="cuda")
            r = cj.cj_solve(p.handle, dev(torch, f), u)
        assert r["sweeps"] == ref["sweeps"] and {0: "converged", 1: "floor", 3: "stalled"}[r["rc"]] == ref["status"]
        np.testing.assert_array_equal(u.cpu().numpy(), ref["u"])


def test_cluster_solve_repeats_and_warm_starts(cj, torch):
    """A second solve on the same plan, and a warm start, give the launched sweeps' results."""
    Nx, Ny, st = 80, 70, 9
    f = workloads.smooth_random_rhs(Nx, Ny, 8)
    u0 = np.random.default_rng(1).standard_normal((Ny, Nx)) * 1e-3
    res = {}
    for launch in (3, 1):
        with cj.Plan(Nx, Ny, st, 1e-9, launch=launch) as p:
            for k in range(2):
                u = dev(torch, u0)
                r = cj.cj_solve(p.handle, dev(torch, f), u)
            res[launch] = (r["sweeps"], u.cpu().numpy())
    assert res[3][0] == res[1][0]
    np.testing.assert_array_equal(res[3][1], res[1][1])


def test_cluster_launch_refused_where_it_does_not_fit(cj):
    with pytest.raises(cj.CJError):
        cj.Plan(200, 200, 9, 1e-8, launch=3)
    with pytest.raises(cj.CJError):
        cj.Plan(64, 64, 9, 1e-8, launch=3, precision=cj.CJ_FP32_INNER)
