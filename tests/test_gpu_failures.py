"""Failures injected on the host: non-finite input data and malformed requests.

Nothing here faults, traps or hangs the GPU.  A NaN or an Inf placed in the right-hand side (or
the initial guess) makes the relative residual non-finite, which every stop test reports as
CJ_ERR_DIVERGED; the tests check that status, that the plan (or the batch, or the server) stays
usable, and that the problems solved beside the failing one keep the oracle's bits.
"""
import time

import numpy as np
import pytest

from oracle import oracle as orc
import workloads

pytestmark = pytest.mark.gpu


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


def _poisoned(f, bad, where=(5, 7)):
    g = f.copy()
    g[where] = bad
    return g


def _oracle(st, f, tol, prec, M_in):
    if prec == 0:
        return orc.solve(st, f, tol)
    return {1: orc.solve_mixed, 2: orc.solve_mixed_dd, 3: orc.solve_fp64_dd}[prec](st, f, tol, M_in)


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
@pytest.mark.parametrize("bad", [np.nan, np.inf, -np.inf])
@pytest.mark.parametrize("st", [5, 17])
def test_non_finite_rhs_diverges_and_the_plan_stays_usable(cj, torch, prec, bad, st):
    Nx, Ny, tol, M_in = 40, 33, 1e-10, 32
    f = workloads.smooth_random_rhs(Nx, Ny, 3, kmax=20)
    kw = {} if prec == 0 else dict(precision=prec, inner_cycle=M_in)
    with cj.Plan(Nx, Ny, st, tol, **kw) as p:
        u = torch.zeros((Ny, Nx), dtype=torch.float64, device="cuda")
        res = cj.cj_solve(p.handle, dev(torch, _poisoned(f, bad)), u)
        assert res["rc"] == cj.CJ_ERR_DIVERGED and res["sweeps"] == 0
        # the same plan then solves a clean problem to the oracle's bits
        u.zero_()
        res = cj.cj_solve(p.handle, dev(torch, f), u)
    ref = _oracle(st, f, tol, prec, M_in)
    assert res["sweeps"] == ref["sweeps"]
    assert {0: "converged", 1: "floor", 3: "stalled"}[res["rc"]] == ref["status"]
    np.testing.assert_array_equal(u.cpu().numpy(), ref["u"])


@pytest.mark.parametrize("prec", [0, 2])
def test_non_finite_initial_guess_diverges(cj, torch, prec):
    Nx, Ny = 30, 20
    f = workloads.smooth_random_rhs(Nx, Ny, 4, kmax=10)
    u0 = np.zeros((Ny, Nx))
    u0[3, 3] = np.nan
    kw = {} if prec == 0 else dict(precision=prec, inner_cycle=16)
    with cj.Plan(Nx, Ny, 9, 1e-8, **kw) as p:
        res = cj.cj_solve(p.handle, dev(torch, f), dev(torch, u0))
    assert res["rc"] == cj.CJ_ERR_DIVERGED


def test_non_finite_rhs_in_solve_host_and_to_error(cj, torch):
    N, st = 24, 9
    f, ue, _ = workloads.paper_problem(N, N)
    with cj.Plan(N, N, st, 1e-8) as p:
        res = cj.cj_solve_host(p.handle, _poisoned(f, np.nan), np.zeros((N, N)))
        assert res["rc"] == cj.CJ_ERR_DIVERGED
        u = torch.zeros((N, N), dtype=torch.float64, device="cuda")
        res = cj.cj_solve_to_error(p.handle, dev(torch, _poisoned(f, np.inf)), u, dev(torch, ue), 1e-6)
        assert res["rc"] == cj.CJ_ERR_DIVERGED


MATES = [  # (Nx, Ny, stencil, tol, precision, inner cycle)
    (33, 20, 5, 1e-8, 1, 64),
    (130, 70, 9, 1e-8, 1, 128),
    (64, 64, 17, 1e-10, 2, 64),
    (90, 41, 9, 1e-9, 2, 64),
]


def test_batch_with_a_diverging_problem_keeps_its_mates_exact(cj, torch):
    fs, probs = [], []
    for k, (Nx, Ny, st, tol, prec, M_in) in enumerate(MATES):
        f = workloads.smooth_random_rhs(Nx, Ny, 50 + k, kmax=30)
        fs.append(f)
        probs.append(dict(Nx=Nx, Ny=Ny, st=st, tol=tol, precision=prec, inner_cycle=M_in,
                          f=dev(torch, f), u=torch.zeros((Ny, Nx), dtype=torch.float64, device="cuda")))
    bad_f = _poisoned(workloads.smooth_random_rhs(100, 60, 9, kmax=30), np.nan, (30, 40))
    bad = dict(Nx=100, Ny=60, st=9, tol=1e-8, precision=1, inner_cycle=64, f=dev(torch, bad_f),
               u=torch.zeros((60, 100), dtype=torch.float64, device="cuda"))
    res = cj.cj_solve_batch(probs[:2] + [bad] + probs[2:])
    assert res[2]["rc"] == cj.CJ_ERR_DIVERGED
    for k, (Nx, Ny, st, tol, prec, M_in) in enumerate(MATES):
        r = res[k if k < 2 else k + 1]
        ref = _oracle(st, fs[k], tol, prec, M_in)
        assert r["sweeps"] == ref["sweeps"] and r["cycles"] == ref["outer"], (k, r, ref["sweeps"])
        np.testing.assert_array_equal(probs[k]["u"].cpu().numpy(), ref["u"], err_msg="problem %d" % k)


def _serve(srv, reqs, timeout=120.0):
    out, t0, pending = {}, time.time(), dict(reqs)
    while pending and time.time() - t0 < timeout:
        for t, shape in list(pending.items()):
            got = srv.poll(t, shape)
            if got is not None:
                out[t] = got
                del pending[t]
        time.sleep(0.002)
    assert not pending, "requests did not finish"
    return out


def test_server_survives_a_diverging_and_a_malformed_request(cj, torch):
    """In a live stream: a request whose f holds a NaN ends with CJ_ERR_DIVERGED, a malformed one
    (bad stencil, bad tolerance, empty grid) is refused at submit and never queued, and the
    requests around them complete with the oracle's bits."""
    good = [(60, 40, 5, 1e-8), (90, 70, 9, 1e-9)]
    fs = [workloads.smooth_random_rhs(Nx, Ny, 70 + k, kmax=30) for k, (Nx, Ny, st, tol) in enumerate(good)]
    with cj.Server(1 << 30, 4) as srv:
        t0 = srv.submit(fs[0], good[0][2], good[0][3])
        tb = srv.submit(_poisoned(workloads.smooth_random_rhs(50, 50, 5), np.nan), 9, 1e-8)
        with pytest.raises(cj.CJError):
            srv.submit(np.zeros((8, 8)), 7, 1e-8)
        with pytest.raises(cj.CJError):
            srv.submit(np.zeros((8, 8)), 9, 0.0)
        with pytest.raises(cj.CJError):
            srv.submit(np.zeros((0, 8)), 9, 1e-8)
        t1 = srv.submit(fs[1], good[1][2], good[1][3])
        got = _serve(srv, {t0: fs[0].shape, tb: (50, 50), t1: fs[1].shape})
        stats = srv.stats()
    assert got[tb][1]["rc"] == cj.CJ_ERR_DIVERGED
    assert stats["completed"] == 3 and stats["active"] == 0 and stats["bytes_in_use"] == 0
    for t, f, (Nx, Ny, st, tol) in ((t0, fs[0], good[0]), (t1, fs[1], good[1])):
        with cj.Plan(Nx, Ny, st, tol, precision=1) as p:
            M_in = p.info()["M_inner"]
        ref = orc.solve_mixed(st, f, tol, M_in, max_outer=64)
        u, r = got[t]
        assert r["sweeps"] == ref["sweeps"]
        np.testing.assert_array_equal(u, ref["u"])
