"""2-D domain decomposition (the host logic of paper_1705_00103_gb300/dd.py) on the CPU.

The partition, the halo bookkeeping, the two-phase exchange and the cross-rank stop test are
checked with the blocks' compute done by the oracle (a test backend below: its sweep and
residual on a box of the extended array are the oracle's Dirichlet-ring sweep and residual with
the ring cut from that array), one process holding several blocks and two gloo ranks holding one
each; the result must be the oracle's undecomposed solve bit for bit.  The GPU test at the end
runs the product backend (libcj's box kernels) on one GPU.
"""
import os
import socket

import numpy as np
import pytest
import torch

from oracle import oracle as orc
from paper_1705_00103_gb300 import dd
import workloads


class OracleBlocks:
    """Block compute by the oracle on host float64 tensors (test infrastructure only)."""

    def zeros(self, shape):
        return torch.zeros(shape, dtype=torch.float64)

    def empty_like(self, t):
        return torch.empty(tuple(t.shape), dtype=t.dtype)

    def copy(self, dst, src):
        dst.copy_(src)

    def load_rhs(self, sd, f, B, h2):
        B[sd.interior()] = torch.from_numpy(h2 * np.asarray(f))

    @staticmethod
    def _cut(A, box):
        row0, col0, nyb, nxb, _ = box
        return A[row0 - 2:row0 + nyb + 2, col0 - 2:col0 + nxb + 2].copy(), A[row0:row0 + nyb, col0:col0 + nxb].copy()

    def sweep(self, sd, src, dst, B, box, w):
        row0, col0, nyb, nxb, edges = box
        G, u = self._cut(src.numpy(), box)
        b = B.numpy()[row0:row0 + nyb, col0:col0 + nxb].copy()
        v = orc.sweep_bc(sd.st, u, G, b, w)
        D = dst.numpy()
        D[row0:row0 + nyb, col0:col0 + nxb] = v
        if sd.st == 17:  # the odd-reflection ghosts beyond the grid's boundary sides (R6)
            rs, cs = slice(row0, row0 + nyb), slice(col0, col0 + nxb)
            if edges & 1:
                D[rs, col0 - 2] = -v[:, 0]
            if edges & 2:
                D[rs, col0 + nxb + 1] = -v[:, -1]
            for bit, row, src_row in ((4, row0 - 2, 0), (8, row0 + nyb + 1, -1)):
                if edges & bit:
                    D[row, cs] = -v[src_row, :]
                    if edges & 1:
                        D[row, col0 - 2] = v[src_row, 0]
                    if edges & 2:
                        D[row, col0 + nxb + 1] = v[src_row, -1]

    def residual(self, sd, U, B):
        box = sd.box(0)
        row0, col0, nyb, nxb, _ = box
        G, u = self._cut(U.numpy(), box)
        b = B.numpy()[row0:row0 + nyb, col0:col0 + nxb]
        s, m = orc.residual_bc(sd.st, u, G, b)
        return [s, m, float(np.sum(u * u)), float(np.sum(b * b)), float(np.abs(b).max())]

    def block(self, sd, U):
        return U[sd.interior()]


STATUS = {0: "converged", 1: "floor", 3: "stalled"}


def _blocks(part, f, ranks):
    out = {}
    for r in ranks:
        i0, nx, j0, ny = part.block(r)
        out[r] = np.ascontiguousarray(f[j0:j0 + ny, i0:i0 + nx])
    return out


def _assemble(part, blocks):
    u = np.zeros((part.Ny, part.Nx))
    for r, b in blocks.items():
        i0, nx, j0, ny = part.block(r)
        u[j0:j0 + ny, i0:i0 + nx] = np.asarray(b)
    return u


def test_split_is_balanced_and_tiles():
    for n in (1, 7, 64, 101):
        for p in range(1, min(n, 9) + 1):
            parts = dd.split(n, p)
            assert sum(c for _, c in parts) == n and parts[0][0] == 0
            assert max(c for _, c in parts) - min(c for _, c in parts) <= 1
            assert all(parts[k][0] + parts[k][1] == parts[k + 1][0] for k in range(p - 1))
    with pytest.raises(ValueError):
        dd.split(3, 4)


def test_partition_neighbours_are_symmetric_and_blocks_tile():
    part = dd.Partition(50, 37, 3, 2)
    cover = np.zeros((37, 50), dtype=int)
    for r in range(part.size):
        i0, nx, j0, ny = part.block(r)
        cover[j0:j0 + ny, i0:i0 + nx] += 1
        for dx, dy in ((1, 0), (0, 1), (1, 1), (-1, 1)):
            n = part.neighbour(r, dx, dy)
            if n is not None:
                assert part.neighbour(n, -dx, -dy) == r
    assert np.all(cover == 1)


@pytest.mark.parametrize("st,K", [(5, 1), (9, 2), (17, 1), (17, 3)])
def test_halo_entries_pair_up(st, K):
    """Every strip a block sends has the shape of the strip its neighbour receives, under the
    tag the neighbour expects; the width is r K and the strips span the full array."""
    part = dd.Partition(40, 33, 3, 2)
    subs = {r: dd.Subdomain(part, r, st, K) for r in range(part.size)}
    for r, sd in subs.items():
        assert sd.h == (2 if st == 17 else 1) * K and sd.H == sd.h + 2
        for phase in (0, 1):
            for nb, stag, send, rtag, recv in sd.halo(phase):
                A = np.zeros(sd.shape)
                peer = [e for e in subs[nb].halo(phase) if e[0] == r]
                assert len(peer) == 1
                _, pstag, psend, prtag, precv = peer[0]
                assert pstag == rtag and prtag == stag
                Bn = np.zeros(subs[nb].shape)
                assert A[send].shape == Bn[precv].shape and A[recv].shape == Bn[psend].shape
                assert min(A[send].shape) == sd.h


@pytest.mark.parametrize("st", [5, 9, 17])
@pytest.mark.parametrize("Px,Py,K", [(2, 2, 1), (3, 1, 1), (1, 3, 2), (2, 3, 4)])
def test_blocks_in_one_process_give_the_oracles_bits(st, Px, Py, K):
    Nx, Ny, tol = 37, 29, 1e-10
    f = workloads.smooth_random_rhs(Nx, Ny, 5, kmax=20)
    part = dd.Partition(Nx, Ny, Px, Py)
    blocks, res = dd.solve(part, st, tol, _blocks(part, f, range(part.size)), OracleBlocks(), dd.LocalComm(), K=K)
    ref = orc.solve(st, f, tol)
    assert res["sweeps"] == ref["sweeps"] and res["cycles"] == ref["cycles"]
    assert STATUS[res["status"]] == ref["status"]
    np.testing.assert_array_equal(_assemble(part, blocks), ref["u"])
    assert res["rel_res_l2"] == pytest.approx(ref["rel_l2"], rel=1e-12)
    assert res["exchanges"] == 1 + res["cycles"] * (-(-len(dd.plan_weights(Nx, Ny, st, tol)[0]) // K)) + 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, st, Px, Py, K, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        Nx, Ny = 41, 30
        f = workloads.smooth_random_rhs(Nx, Ny, 6, kmax=20)
        part = dd.Partition(Nx, Ny, Px, Py)
        blocks, res = dd.solve(part, st, 1e-10, _blocks(part, f, [rank]), OracleBlocks(), dd.DistComm(dist), K=K)
        q.put((rank, np.asarray(blocks[rank]).copy(), res))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("st,Px,Py,K", [(9, 2, 1, 1), (17, 1, 2, 2), (5, 2, 1, 3), (9, 2, 2, 1), (17, 2, 2, 1)])
def test_gloo_ranks_give_the_single_rank_bits(st, Px, Py, K):
    """World size Px x Py (2 or 4) over gloo: each rank holds one block, halos travel as messages
    (with a 2 x 2 split the corner values reach the diagonal neighbour through the two-phase
    exchange), the stop test reduces across ranks; the assembled u, the sweep count and the status
    are the undecomposed oracle solve's."""
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    world = Px * Py
    procs = [ctx.Process(target=_rank, args=(r, world, port, st, Px, Py, K, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = {}
    for _ in procs:
        r, u, res = q.get(timeout=300)
        out[r] = (u, res)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    Nx, Ny = 41, 30
    f = workloads.smooth_random_rhs(Nx, Ny, 6, kmax=20)
    part = dd.Partition(Nx, Ny, Px, Py)
    ref = orc.solve(st, f, 1e-10)
    u = _assemble(part, {r: out[r][0] for r in out})
    np.testing.assert_array_equal(u, ref["u"])
    for r in out:
        res = out[r][1]
        assert res["sweeps"] == ref["sweeps"] and STATUS[res["status"]] == ref["status"]
        assert res["rel_res_l2"] == out[0][1]["rel_res_l2"]


def test_blocks_narrower_than_the_halo_are_refused():
    part = dd.Partition(10, 10, 5, 1)
    with pytest.raises(ValueError):
        dd.Subdomain(part, 0, 17, 2)


@pytest.mark.gpu
@pytest.mark.parametrize("st,Px,Py,K", [(9, 2, 2, 1), (17, 3, 2, 2), (5, 1, 4, 4)])
def test_device_blocks_give_the_undecomposed_solves_bits(st, Px, Py, K):
    """The product backend (libcj's box kernels on one GPU), blocks held by one process: u, the
    sweep count and the status equal cj_solve's for the whole grid (and so the oracle's)."""
    import paper_1705_00103_gb300 as cj
    cj.build.build()
    Nx, Ny, tol = 150, 97, 1e-9
    f = workloads.smooth_random_rhs(Nx, Ny, 7, kmax=30)
    part = dd.Partition(Nx, Ny, Px, Py)
    fb = {r: torch.from_numpy(b).cuda() for r, b in _blocks(part, f, range(part.size)).items()}
    blocks, res = dd.solve(part, st, tol, fb, dd.Device(), dd.LocalComm(), K=K)
    u = _assemble(part, {r: b.cpu().numpy() for r, b in blocks.items()})
    with cj.Plan(Nx, Ny, st, tol) as p:
        ud = torch.zeros((Ny, Nx), dtype=torch.float64, device="cuda")
        ref = cj.cj_solve(p.handle, torch.from_numpy(f).cuda(), ud)
    assert res["sweeps"] == ref["sweeps"] and res["status"] == ref["rc"]
    np.testing.assert_array_equal(u, ud.cpu().numpy())
    assert res["rel_res_l2"] == pytest.approx(ref["rel_res_l2"], rel=1e-12)


@pytest.mark.parametrize("st", [5, 9, 17])
@pytest.mark.parametrize("Nx,Ny,tol", [(1, 1, 1e-6), (64, 64, 1e-10), (4096, 4096, 1e-10), (8192, 8192, 1e-10),
                                       (300, 17, 1e-8)])
def test_host_plan_weights_equal_the_oracles(st, Nx, Ny, tol):
    """cj_plan_weights (host arithmetic only, no GPU needed): kappa bounds, M and every weight
    bit-equal to the oracle's."""
    w, M, kmin, kmax = dd.plan_weights(Nx, Ny, st, tol)
    a, b = orc.kappa_bounds(st, Nx, Ny)
    assert (kmin, kmax) == (a, b) and M == orc.cycle_length(a, b, tol)
    np.testing.assert_array_equal(np.array(w), orc.sweep_coeffs(st, a, b, M))


def test_host_plan_weights_argument_checks():
    import ctypes
    from paper_1705_00103_gb300 import cj
    L = cj._lib()
    buf = (ctypes.c_double * 4)()
    M = ctypes.c_longlong()
    assert L.cj_plan_weights(0, 4, 5, 1e-6, 0, None, 0, None, None, None) == cj.CJ_ERR_INVALID_ARG
    assert L.cj_plan_weights(4, 4, 7, 1e-6, 0, None, 0, None, None, None) == cj.CJ_ERR_INVALID_ARG
    assert L.cj_plan_weights(4, 4, 5, 1.5, 0, None, 0, None, None, None) == cj.CJ_ERR_INVALID_ARG
    assert L.cj_plan_weights(64, 64, 5, 1e-10, 0, None, 0, ctypes.byref(M), None, None) == cj.CJ_OK and M.value > 4
    assert L.cj_plan_weights(64, 64, 5, 1e-10, 0, buf, 4, None, None, None) == cj.CJ_ERR_INVALID_ARG
