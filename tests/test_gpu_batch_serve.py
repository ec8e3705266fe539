"""Batched and served solves (the step engine) against the FP64 oracle, through the C ABI.

Each problem in a batch runs the mixed-precision CJM with its own plan; its arithmetic is
evaluated per node in the oracle's order, and its residual sums are reduced within its own
tiles in a fixed order, so results are compared bit for bit with the oracle's mixed solves
and with the same problem solved alone or among others.
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


MIX = [  # (Nx, Ny, stencil, tol, precision, inner cycle, temporal depth)
    (33, 20, 5, 1e-8, 1, 64, 1),
    (130, 70, 9, 1e-8, 1, 128, 1),
    (64, 64, 17, 1e-10, 2, 64, 1),
    (257, 100, 9, 1e-9, 1, 128, 4),
    (1, 1, 5, 1e-8, 1, 1, 1),
    (200, 199, 17, 1e-8, 1, 256, 2),
    (3, 300, 9, 1e-8, 2, 128, 3),
    # depth 4 of 5 and 9 points: the register wavefront (several strips and row blocks, ragged)
    (300, 260, 5, 1e-8, 1, 64, 4),
    (130, 129, 9, 1e-9, 2, 128, 4),
    (1, 200, 5, 1e-8, 1, 64, 4),
    (200, 3, 9, 1e-8, 1, 64, 4),
]


def _oracle(Nx, Ny, st, tol, prec, M_in, f):
    if prec == 2:
        return orc.solve_mixed_dd(st, f, tol, M_in, max_outer=64)
    return orc.solve_mixed(st, f, tol, M_in, max_outer=64)


def _problem(torch, Nx, Ny, st, tol, prec, M_in, depth, seed):
    f = workloads.smooth_random_rhs(Nx, Ny, seed, kmax=min(40, max(Nx, Ny)))
    return f, dict(Nx=Nx, Ny=Ny, st=st, tol=tol, precision=prec, inner_cycle=M_in,
                   temporal_depth=depth, f=torch.from_numpy(f).cuda(),
                   u=torch.zeros((Ny, Nx), dtype=torch.float64, device="cuda"))


def test_batch_matches_oracle(cj, torch):
    fs, probs = [], []
    for k, (Nx, Ny, st, tol, prec, M_in, depth) in enumerate(MIX):
        f, pr = _problem(torch, Nx, Ny, st, tol, prec, M_in, depth, 40 + k)
        fs.append(f)
        probs.append(pr)
    res = cj.cj_solve_batch(probs)
    for k, (Nx, Ny, st, tol, prec, M_in, depth) in enumerate(MIX):
        ref = _oracle(Nx, Ny, st, tol, prec, M_in, fs[k])
        assert res[k]["sweeps"] == ref["sweeps"] and res[k]["cycles"] == ref["outer"], (k, res[k], ref["sweeps"])
        assert {0: "converged", 1: "floor", 3: "stalled"}[res[k]["rc"]] == ref["status"]
        np.testing.assert_array_equal(probs[k]["u"].cpu().numpy(), ref["u"], err_msg="problem %d" % k)
        assert res[k]["rel_res_l2"] == pytest.approx(ref["rel_l2"], rel=1e-10)


def test_batch_result_independent_of_batch_mates(cj, torch):
    Nx, Ny, st, tol, prec, M_in, depth = 150, 90, 9, 1e-9, 1, 128, 1
    f, alone = _problem(torch, Nx, Ny, st, tol, prec, M_in, depth, 77)
    cj.cj_solve_batch([alone])
    _, again = _problem(torch, Nx, Ny, st, tol, prec, M_in, depth, 77)
    others = [_problem(torch, *m, 90 + k)[1] for k, m in enumerate(MIX)]
    cj.cj_solve_batch(others[:3] + [again] + others[3:])
    assert torch.equal(alone["u"], again["u"])


def test_batch_warm_start_and_strided(cj, torch):
    Nx, Ny, ld = 45, 30, 64
    f = workloads.smooth_random_rhs(Nx, Ny, 5)
    u0 = np.random.default_rng(3).standard_normal((Ny, Nx)) * 1e-3
    fbig = torch.full((Ny, ld), 9.0, dtype=torch.float64, device="cuda")
    ubig = torch.full((Ny, ld), -1.0, dtype=torch.float64, device="cuda")
    fbig[:, :Nx] = torch.from_numpy(f).cuda()
    ubig[:, :Nx] = torch.from_numpy(u0).cuda()
    res = cj.cj_solve_batch([dict(Nx=Nx, Ny=Ny, st=17, tol=1e-9, precision=1, inner_cycle=64,
                                  f=fbig[:, :Nx], u=ubig[:, :Nx])])
    ref = orc.solve_mixed(17, f, 1e-9, 64, u0=u0, max_outer=64)
    assert res[0]["sweeps"] == ref["sweeps"]
    np.testing.assert_array_equal(ubig[:, :Nx].cpu().numpy(), ref["u"])
    assert float(ubig[:, Nx:].min()) == -1.0 and float(ubig[:, Nx:].max()) == -1.0


def test_batch_rejects_bad_problem(cj, torch):
    f = torch.zeros((4, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(cj.CJError):
        cj.cj_solve_batch([dict(Nx=4, Ny=4, st=7, tol=1e-8, f=f, u=f.clone())])


def _serve(cj, srv, reqs, timeout=120.0):
    out = {}
    t0 = time.time()
    pending = dict(reqs)
    while pending and time.time() - t0 < timeout:
        for t, shape in list(pending.items()):
            got = srv.poll(t, shape)
            if got is not None:
                out[t] = got
                del pending[t]
        time.sleep(0.002)
    assert not pending, "requests did not finish"
    return out


def test_server_results_match_oracle_and_alone(cj, torch):
    cases = [(60, 40, 5, 1e-8), (130, 90, 9, 1e-9), (80, 80, 17, 1e-10), (200, 33, 9, 1e-6), (17, 17, 17, 1e-8)]
    fs = [workloads.smooth_random_rhs(Nx, Ny, 60 + k, kmax=30) for k, (Nx, Ny, st, tol) in enumerate(cases)]
    with cj.Server(2 << 30, 4) as srv:
        tickets = {srv.submit(f, st, tol): (Ny, Nx) for f, (Nx, Ny, st, tol) in zip(fs, cases)}
        mixed = _serve(cj, srv, tickets)
        st_ = srv.stats()
    assert st_["completed"] == len(cases) and st_["active"] == 0 and st_["bytes_in_use"] == 0
    results = [mixed[t] for t in sorted(mixed)]
    for k, ((u, r), (Nx, Ny, st, tol)) in enumerate(zip(results, cases)):
        # the server picks precision and inner cycle as a plan of that problem would
        prec = 2 if 4 * 2.0 ** -53 * orc.abs_coeff_sum(st) / (orc.centre(st) * orc.kappa_bounds(st, Nx, Ny)[0]) > tol else 1
        with cj.Plan(Nx, Ny, st, tol, precision=prec) as p:
            M_in = p.info()["M_inner"]
        ref = _oracle(Nx, Ny, st, tol, prec, M_in, fs[k])
        assert r["rc"] in (cj.CJ_OK, cj.CJ_FLOOR, cj.CJ_STALLED) and r["sweeps"] == ref["sweeps"], (k, r, ref["sweeps"])
        np.testing.assert_array_equal(u, ref["u"], err_msg="request %d" % k)
        assert r["seconds"] > 0
    # the same request alone gives the same bits
    with cj.Server(2 << 30, 4) as srv:
        t = srv.submit(fs[1], cases[1][2], cases[1][3])
        alone = _serve(cj, srv, {t: (cases[1][1], cases[1][0])})[t]
    np.testing.assert_array_equal(alone[0], results[1][0])


def test_server_admission_by_footprint(cj, torch):
    """A budget that holds one problem at a time still completes every request (the rest
    wait in the queue); a problem larger than the whole budget is refused."""
    f = workloads.smooth_random_rhs(100, 100, 3, kmax=20)
    with cj.Server(2_000_000, 8) as srv:   # ~2 MB: one 100x100 problem (~0.4 MB) ... a few
        ts = {srv.submit(f, 9, 1e-8): (100, 100) for _ in range(6)}
        big = srv.submit(np.zeros((400, 400)), 9, 1e-8)
        want = dict(ts)
        want[big] = (400, 400)
        res = _serve(cj, srv, want)
        stats = srv.stats()
    us = [res[t][0] for t in ts]
    for u in us[1:]:
        np.testing.assert_array_equal(u, us[0])
    assert res[big][1]["rc"] == cj.CJ_ERR_BUDGET
    assert stats["peak_bytes"] <= 2_000_000


def test_server_rejects_bad_request(cj):
    with cj.Server(1 << 26, 2) as srv:
        with pytest.raises(cj.CJError):
            srv.submit(np.zeros((4, 4)), 6, 1e-8)
        with pytest.raises(cj.CJError):
            srv.submit(np.zeros((4, 4)), 5, 2.0)


def test_engine_autotune_records_and_uses_its_choice(cj, torch):
    """The engine autotuner times tile rows x depth on a problem of the size class, records the
    fastest, and a batch of that class then runs with it -- to the oracle's bits.  (Run last in
    this file: the choice stays in the process's table.)"""
    # both sides >= 512: depth 4 (the register wavefront) is a candidate
    r = cj.cj_autotune_engine(600, 520, 5)
    assert all(v > 0 for v in r["gupd"].values())
    assert r["gupd"][(r["tile_rows"], r["depth"])] == max(r["gupd"].values())
    Nx, Ny, st = 300, 200, 9
    r = cj.cj_autotune_engine(Nx, Ny, st)
    assert r["tile_rows"] in (16, 32, 64) and r["depth"] in (1, 2)
    assert all((v > 0) == (d != 4) for (ty, d), v in r["gupd"].items())  # a side under 512: no depth 4
    assert r["gupd"][(r["tile_rows"], r["depth"])] == max(r["gupd"].values())
    f, pr = _problem(torch, Nx, Ny, st, 1e-8, 1, 128, 0, 31)  # temporal_depth 0: the tuned one
    res = cj.cj_solve_batch([pr])
    ref = _oracle(Nx, Ny, st, 1e-8, 1, 128, f)
    assert res[0]["sweeps"] == ref["sweeps"] and res[0]["cycles"] == ref["outer"]
    np.testing.assert_array_equal(pr["u"].cpu().numpy(), ref["u"])
    with pytest.raises(cj.CJError):
        cj.cj_autotune_engine(0, 10, 9)


def test_server_lanes_give_the_batch_engines_bits(cj, torch):
    """Requests in all three size lanes (up to 2^20 nodes, up to 2^23, larger) give the bits the
    batch engine gives for the same problems (the batch engine is checked against the oracle
    above); a small request submitted after a large one finishes first."""
    cases = [(3000, 2900, 9, 1e-6), (1100, 1000, 5, 1e-6), (100, 80, 17, 1e-8), (64, 64, 9, 1e-10)]
    fs = [workloads.smooth_random_rhs(Nx, Ny, 80 + k, kmax=30) for k, (Nx, Ny, st, tol) in enumerate(cases)]
    done_at = {}
    with cj.Server(8 << 30, 8) as srv:
        tickets = {srv.submit(f, st, tol): k for k, (f, (Nx, Ny, st, tol)) in enumerate(zip(fs, cases))}
        got, t0 = {}, time.time()
        while len(got) < len(cases) and time.time() - t0 < 300:
            for t, k in tickets.items():
                if k not in got:
                    g = srv.poll(t, fs[k].shape)
                    if g is not None:
                        got[k] = g
                        done_at[k] = len(done_at)
            time.sleep(0.001)
    assert len(got) == len(cases)
    assert done_at[3] < done_at[0] and done_at[2] < done_at[0]
    probs = [dict(Nx=Nx, Ny=Ny, st=st, tol=tol, f=torch.from_numpy(f).cuda(),
                  u=torch.zeros((Ny, Nx), dtype=torch.float64, device="cuda"))
             for f, (Nx, Ny, st, tol) in zip(fs, cases)]
    res = cj.cj_solve_batch(probs)
    for k in range(len(cases)):
        u, r = got[k]
        assert r["rc"] == res[k]["rc"] and r["sweeps"] == res[k]["sweeps"], (k, r, res[k])
        np.testing.assert_array_equal(u, probs[k]["u"].cpu().numpy(), err_msg="request %d" % k)
        assert 0 < r["sweep_seconds"] <= r["seconds"]
