"""Coefficient-mask plans (Sec. 3.2) on the GPU against the oracle, through the C ABI: every
sweep and whole solves bit for bit, for the four patterns, broadcast coefficient layouts, a
node factor, and Dirichlet data."""
import numpy as np
import pytest

from oracle import oracle as orc
from workloads import masks

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


def _dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _kappa(P, Nx, Ny):
    """Spectrum bounds of D^-1 A from the dense matrix (small grids)."""
    offs = orc.mask_offsets(P["pattern"])
    coef = np.broadcast_to(P["coef"], (len(offs) + 1, Ny, Nx))
    n = Nx * Ny
    A = np.zeros((n, n))
    for j in range(Ny):
        for i in range(Nx):
            A[j * Nx + i, j * Nx + i] = coef[0, j, i]
            for k, (dx, dy) in enumerate(offs):
                if 0 <= i + dx < Nx and 0 <= j + dy < Ny:
                    A[j * Nx + i, (j + dy) * Nx + i + dx] = coef[k + 1, j, i]
    ev = np.linalg.eigvals(A / np.diag(A)[:, None]).real
    return ev.min(), ev.max()


def _problem(name, Nx, Ny, pat=5):
    if name == "random":
        return masks.random_dominant(pat, Nx, Ny, 100 + pat + Nx)
    return {"polar": masks.polar, "bipolar": masks.bipolar, "stretched": masks.cartesian_stretched}[name](Nx, Ny)


def _ring(P, Nx, Ny):
    if P["g"] is None:
        G = np.random.default_rng(Nx * Ny).standard_normal((Ny + 4, Nx + 4))
        G[2:Ny + 2, 2:Nx + 2] = 0.0
        return G
    return orc.ghost_ring(Nx, Ny, P["g"])


CASES = [("random", 5, 1, 1), ("random", 9, 7, 5), ("random", 17, 33, 20), ("random", 25, 130, 70),
         ("random", 25, 3, 9), ("polar", 5, 40, 31), ("bipolar", 5, 37, 41), ("stretched", 5, 29, 35)]


@pytest.mark.parametrize("name,pat,Nx,Ny", CASES)
def test_mask_sweeps_bit_exact(cj, torch, name, pat, Nx, Ny):
    P = _problem(name, Nx, Ny, pat)
    G = _ring(P, Nx, Ny)
    kmin, kmax = 0.01, 1.99
    scale = None if P["scale"] is None else _dev(torch, P["scale"])
    with cj.Plan.mask(Nx, Ny, pat, _dev(torch, P["coef"]), kmin, kmax, 1e-6, scale=scale) as p:
        cj.cj_set_boundary(p.handle, _dev(torch, G))
        info = p.info()
        w = info["w"]
        np.testing.assert_array_equal(w, orc.mask_weights(kmin, kmax, info["M"]))
        chat, dC = orc.mask_normalize(pat, P["coef"], P["scale"], Nx, Ny)
        bhat = P["f"] / dC
        u = np.random.default_rng(7).standard_normal((Ny, Nx))
        fd, ud = _dev(torch, P["f"]), _dev(torch, u)
        for k in range(4):
            cj.cj_sweeps(p.handle, fd, ud, k, 1)
            u = orc.sweep_mask(pat, u, G, bhat, chat, w[k])
            np.testing.assert_array_equal(ud.cpu().numpy(), u, err_msg="sweep %d" % k)
        # the residual norms of the normalised system
        rel, _, _ = cj.cj_residual(p.handle, fd, ud)
        sq, _ = orc.residual_mask(pat, u, G, bhat, chat)
        assert rel == pytest.approx(np.sqrt(sq) / np.linalg.norm(bhat), rel=1e-12)


@pytest.mark.parametrize("name,method", [("polar", 0), ("bipolar", 0), ("stretched", 0), ("random", 1),
                                         ("polar", 1)])
def test_mask_solves_match_oracle(cj, torch, name, method):
    Nx, Ny = 26, 21
    pat = 9 if name == "random" else 5
    P = _problem(name, Nx, Ny, pat)
    G = _ring(P, Nx, Ny)
    kmin, kmax = (0.04, 1.96) if name == "random" else _kappa(P, Nx, Ny)
    kmin, kmax = 0.999 * kmin, 1.001 * kmax
    tol = 1e-10
    ref = orc.solve_mask(pat, P["f"], P["coef"], kmin, kmax, tol, scale=P["scale"], G=G, method=method)
    scale = None if P["scale"] is None else _dev(torch, P["scale"])
    with cj.Plan.mask(Nx, Ny, pat, _dev(torch, P["coef"]), kmin, kmax, tol, scale=scale, method=method) as p:
        cj.cj_set_boundary(p.handle, _dev(torch, G))
        ud = torch.zeros((Ny, Nx), dtype=torch.float64, device="cuda")
        res = cj.cj_solve(p.handle, _dev(torch, P["f"]), ud)
    assert res["sweeps"] == ref["sweeps"] and res["cycles"] == ref["cycles"]
    assert {0: "converged", 1: "floor", 3: "stalled"}[res["status"]] == ref["status"]
    np.testing.assert_array_equal(ud.cpu().numpy(), ref["u"])
    if P["u_exact"] is not None:
        np.testing.assert_allclose(ref["u"], P["u_exact"], rtol=0, atol=1e-7 * np.abs(P["u_exact"]).max())


def test_mask_broadcast_layouts_equal_full_planes(cj, torch):
    """A polar mask given with planes that vary along x only, and the same mask expanded to full
    planes, give the same bits."""
    Nx, Ny = 45, 30
    P = masks.polar(Nx, Ny)
    G = _dev(torch, _ring(P, Nx, Ny))
    outs = []
    for coef in (P["coef"], np.broadcast_to(P["coef"], (5, Ny, Nx))):
        with cj.Plan.mask(Nx, Ny, 5, _dev(torch, coef), 0.001, 1.999, 1e-8) as p:
            cj.cj_set_boundary(p.handle, G)
            ud = torch.zeros((Ny, Nx), dtype=torch.float64, device="cuda")
            cj.cj_solve(p.handle, _dev(torch, P["f"]), ud)
            outs.append(ud.cpu().numpy())
    np.testing.assert_array_equal(outs[0], outs[1])


def test_mask_argument_checks(cj, torch):
    c = _dev(torch, masks.random_dominant(9, 6, 5, 1)["coef"])
    bad = [dict(pattern=7), dict(kmin=0.0), dict(kmin=2.0, kmax=1.0)]
    for kw in bad:
        args = dict(pattern=9, kmin=0.1, kmax=1.9)
        args.update(kw)
        with pytest.raises(cj.CJError):
            cj.cj_plan_create_mask(6, 5, args["pattern"], c, args["kmin"], args["kmax"], 1e-6)
    z = c.clone()
    z[0, 2, 3] = 0.0
    with pytest.raises(cj.CJError, match="centre"):
        cj.cj_plan_create_mask(6, 5, 9, z, 0.1, 1.9, 1e-6)


def test_mask_host_solve_and_history_equal_the_device_solve(cj, torch):
    """cj_solve_host (one copy in, one out) and cj_solve_history give the device solve's bits on
    a mask plan, and the history ends at the reported residual."""
    Nx, Ny = 31, 27
    P = masks.polar(Nx, Ny, solution="harmonic")
    G = _dev(torch, _ring(P, Nx, Ny))
    kmin, kmax = _kappa(P, Nx, Ny)
    outs = []
    for how in ("device", "host", "history"):
        with cj.Plan.mask(Nx, Ny, 5, _dev(torch, P["coef"]), 0.999 * kmin, 1.001 * kmax, 1e-9) as p:
            cj.cj_set_boundary(p.handle, G)
            if how == "host":
                u = np.zeros((Ny, Nx))
                res = cj.cj_solve_host(p.handle, np.ascontiguousarray(P["f"]), u)
            else:
                ud = torch.zeros((Ny, Nx), dtype=torch.float64, device="cuda")
                if how == "device":
                    res = cj.cj_solve(p.handle, _dev(torch, P["f"]), ud)
                else:
                    res = cj.cj_solve_history(p.handle, _dev(torch, P["f"]), ud)
                    assert res["history"][-1] == res["rel_res_l2"]
                u = ud.cpu().numpy()
            outs.append((res["sweeps"], u))
    for sweeps, u in outs[1:]:
        assert sweeps == outs[0][0]
        np.testing.assert_array_equal(u, outs[0][1])
