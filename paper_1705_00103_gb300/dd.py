"""Two-dimensional domain decomposition of one CJM solve across ranks (host logic).

The paper solves each grid on one GPU (Sec. 3.2).  A grid too large for one device, or one
spread over several to cut its time, splits into Px x Py blocks of nearly equal size, one per
rank.  Each rank keeps its block in an extended array with a margin of H = h + 2 nodes on every
side, h = r K (r the stencil radius, K the sweeps between exchanges):

  - on a side shared with a neighbouring block the margin's first h nodes hold the neighbour's
    halo, refreshed by an exchange before every K sweeps;
  - on a side that is the grid's boundary it holds the homogeneous ghosts (0 at distance 1 and,
    for the 17-point stencil, the odd reflection at distance 2, written by the sweep kernel with
    each boundary node).

K sweeps after an exchange run on shrinking boxes (sweep s updates the block extended by
h - r s nodes on its shared sides), so the block is exact after the K-th, with the redundant
halo work of temporal blocking in place of K - 1 exchanges.  The exchange has two phases: left
and right strips of the full array height, then top and bottom strips of the full array width,
which carries the corner regions (the diagonal neighbours' nodes) along without diagonal
messages.  The stop test of R8 needs the global relative residual: every rank reduces
(sum r^2, max |r|, sum u^2, sum b^2, max |b|) over its block, and one all-reduce (sums and
maxima) gives every rank the same numbers, so all take the same decision.

Each node's arithmetic and its order are those of the undecomposed sweep (the box kernels of
libcj), and the halo holds exact copies, so a decomposed solve gives the undecomposed solve's
u bit for bit; only the residual sums are reduced in another order.

Compute goes through a backend (the product one, `Device`, calls libcj's kernels on the current
CUDA device); messages go through a communicator (`LocalComm` for blocks held by one process,
`DistComm` for one block per torch.distributed rank: gloo on host tensors, NCCL on device
tensors).  Halo strips are copied, never read from a peer's memory by a kernel.
"""
from __future__ import annotations

import ctypes
import math

from . import cj as _cj

_EPS = 2.0 ** -53
# sum of the absolute stencil coefficients in units of 1/h^2 (Table 3, Eq. 1, Eq. 2): the S of
# the rounding-floor estimate of R8
_ABS_COEFF_SUM = {5: 8.0, 9: 40.0 / 6.0, 17: 640.0 / 72.0}
# message tags: the side of the sender the strip leaves from
_TO_LEFT, _TO_RIGHT, _TO_BOTTOM, _TO_TOP = 0, 1, 2, 3


def split(n: int, p: int) -> list:
    """(first, count) of p nearly equal parts of n nodes, the first n mod p parts one longer."""
    if p < 1 or p > n:
        raise ValueError("cannot split %d nodes into %d parts" % (n, p))
    q, rem = divmod(n, p)
    out, first = [], 0
    for k in range(p):
        c = q + (1 if k < rem else 0)
        out.append((first, c))
        first += c
    return out


class Partition:
    """Px x Py blocks of an Nx x Ny interior; rank = py * Px + px, block (px, py) covers
    interior columns i0 .. i0 + nx - 1 and rows j0 .. j0 + ny - 1 (0-based)."""

    def __init__(self, Nx: int, Ny: int, Px: int, Py: int):
        self.Nx, self.Ny, self.Px, self.Py = Nx, Ny, Px, Py
        self.xs, self.ys = split(Nx, Px), split(Ny, Py)
        self.size = Px * Py

    def coords(self, rank: int):
        return rank % self.Px, rank // self.Px

    def rank_at(self, px: int, py: int):
        if 0 <= px < self.Px and 0 <= py < self.Py:
            return py * self.Px + px
        return None

    def neighbour(self, rank: int, dx: int, dy: int):
        px, py = self.coords(rank)
        return self.rank_at(px + dx, py + dy)

    def block(self, rank: int):
        """(i0, nx, j0, ny) of a rank's block."""
        px, py = self.coords(rank)
        (i0, nx), (j0, ny) = self.xs[px], self.ys[py]
        return i0, nx, j0, ny


class Subdomain:
    """One rank's block: the extended-array geometry, its boxes and its halo bookkeeping."""

    def __init__(self, part: Partition, rank: int, st: int, K: int = 1):
        if st not in (5, 9, 17) or K < 1:
            raise ValueError("bad stencil or sweeps per exchange")
        self.part, self.rank, self.st, self.K = part, rank, st, K
        self.r = 2 if st == 17 else 1
        self.h = self.r * K
        self.H = self.h + 2
        self.i0, self.nx, self.j0, self.ny = part.block(rank)
        if min(self.nx, self.ny) < self.h:
            raise ValueError("blocks must be at least r K = %d nodes wide" % self.h)
        self.shape = (self.ny + 2 * self.H, self.nx + 2 * self.H)
        self.nb = {"left": part.neighbour(rank, -1, 0), "right": part.neighbour(rank, 1, 0),
                   "bottom": part.neighbour(rank, 0, -1), "top": part.neighbour(rank, 0, 1)}
        self.edges = ((self.nb["left"] is None) * 1 | (self.nb["right"] is None) * 2 |
                      (self.nb["bottom"] is None) * 4 | (self.nb["top"] is None) * 8)

    def box(self, ext: int):
        """(row0, col0, nyb, nxb, edges): the block extended by ext nodes on its shared sides."""
        H = self.H
        el = 0 if self.nb["left"] is None else ext
        er = 0 if self.nb["right"] is None else ext
        eb = 0 if self.nb["bottom"] is None else ext
        et = 0 if self.nb["top"] is None else ext
        return H - eb, H - el, self.ny + eb + et, self.nx + el + er, self.edges

    def sweep_box(self, s: int):
        """Box of the s-th sweep (1-based) after an exchange of width h."""
        return self.box(self.h - self.r * s)

    def interior(self):
        return (slice(self.H, self.H + self.ny), slice(self.H, self.H + self.nx))

    def halo(self, phase: int):
        """Exchange entries of a phase (0: left/right, 1: bottom/top): (neighbour, send tag,
        send slices, recv tag, recv slices); the receive tag is the tag the neighbour sends
        with towards this block."""
        H, h, nx, ny = self.H, self.h, self.nx, self.ny
        rows, cols = slice(0, ny + 2 * H), slice(0, nx + 2 * H)
        out = []
        if phase == 0:
            if self.nb["left"] is not None:
                out.append((self.nb["left"], _TO_LEFT, (rows, slice(H, H + h)), _TO_RIGHT, (rows, slice(H - h, H))))
            if self.nb["right"] is not None:
                out.append((self.nb["right"], _TO_RIGHT, (rows, slice(H + nx - h, H + nx)), _TO_LEFT,
                            (rows, slice(H + nx, H + nx + h))))
        else:
            if self.nb["bottom"] is not None:
                out.append((self.nb["bottom"], _TO_BOTTOM, (slice(H, H + h), cols), _TO_TOP, (slice(H - h, H), cols)))
            if self.nb["top"] is not None:
                out.append((self.nb["top"], _TO_TOP, (slice(H + ny - h, H + ny), cols), _TO_BOTTOM,
                            (slice(H + ny, H + ny + h), cols)))
        return out


class LocalComm:
    """Every block held by this process: halos move by array copies, reductions are local."""

    def exchange(self, subs: dict, arrays: dict, backend) -> None:
        for phase in (0, 1):
            for rank, sd in subs.items():
                for nb, _stag, _send, rtag, recv in sd.halo(phase):
                    # the strip the neighbour sends towards this block, with that tag
                    src = next(e for e in subs[nb].halo(phase) if e[0] == rank and e[1] == rtag)
                    backend.copy(arrays[rank][recv], arrays[nb][src[2]])

    def allreduce(self, sums, maxes):
        return list(sums), list(maxes)


class DistComm:
    """One block per torch.distributed rank (block rank = process rank): halo strips by
    point-to-point messages (gloo for host arrays, NCCL for device arrays), the residual
    statistics by one all-reduce each for the sums and the maxima."""

    def __init__(self, dist, device=None):
        self.dist, self.device = dist, device

    def exchange(self, subs: dict, arrays: dict, backend) -> None:
        (rank, sd), = subs.items()
        A = arrays[rank]
        for phase in (0, 1):
            reqs, landing = [], []
            for nb, _stag, _send, rtag, recv in sd.halo(phase):
                buf = backend.empty_like(A[recv])
                reqs.append(self.dist.irecv(buf, src=nb, tag=4 * phase + rtag))
                landing.append((recv, buf))
            for nb, stag, send, _rtag, _recv in sd.halo(phase):
                reqs.append(self.dist.isend(A[send].contiguous(), dst=nb, tag=4 * phase + stag))
            for q in reqs:
                q.wait()
            for recv, buf in landing:
                backend.copy(A[recv], buf)

    def allreduce(self, sums, maxes):
        import torch
        s = torch.tensor(list(sums), dtype=torch.float64, device=self.device)
        m = torch.tensor(list(maxes), dtype=torch.float64, device=self.device)
        self.dist.all_reduce(s, op=self.dist.ReduceOp.SUM)
        self.dist.all_reduce(m, op=self.dist.ReduceOp.MAX)
        return s.tolist(), m.tolist()


class Device:
    """Block compute on the current CUDA device by libcj's box kernels (torch tensors hold the
    extended arrays)."""

    def __init__(self, stream=None):
        import torch
        self.torch = torch
        self.stream = _cj._stream(stream)
        self._scratch = {}
        self._out = torch.zeros(5, dtype=torch.float64, device="cuda")

    def zeros(self, shape):
        return self.torch.zeros(shape, dtype=self.torch.float64, device="cuda")

    def empty_like(self, t):
        return self.torch.empty(tuple(t.shape), dtype=t.dtype, device=t.device)

    def copy(self, dst, src):
        dst.copy_(src)

    @staticmethod
    def _at(t, row0, col0):
        return t.data_ptr() + 8 * (row0 * t.stride(0) + col0)

    def load_rhs(self, sd: Subdomain, f, B, h2: float) -> None:
        """B's block = h^2 f (f: the block's Ny x Nx device array)."""
        fp, ldf = _cj._grid(f, "float64")
        rc = _cj._lib().cj_box_scale(sd.nx, sd.ny, h2, fp, ldf, self._at(B, sd.H, sd.H), B.stride(0), self.stream)
        if rc != _cj.CJ_OK:
            raise _cj.CJError(rc, "cj_box_scale")

    def sweep(self, sd: Subdomain, src, dst, B, box, w: float) -> None:
        row0, col0, nyb, nxb, edges = box
        ld = src.stride(0)
        rc = _cj._lib().cj_box_sweep(nxb, nyb, sd.st, w, self._at(src, row0, col0), ld, self._at(B, row0, col0), ld,
                                     self._at(dst, row0, col0), ld, edges, self.stream)
        if rc != _cj.CJ_OK:
            raise _cj.CJError(rc, "cj_box_sweep")

    def residual(self, sd: Subdomain, U, B):
        """(sum r^2, max |r|, sum u^2, sum b^2, max |b|) over the block."""
        row0, col0, nyb, nxb, _ = sd.box(0)
        n = _cj._lib().cj_box_residual_slots(nxb, nyb)
        if self._scratch.get(n) is None:
            self._scratch = {n: self.torch.empty(n, dtype=self.torch.float64, device="cuda")}
        ld = U.stride(0)
        rc = _cj._lib().cj_box_residual(nxb, nyb, sd.st, self._at(U, row0, col0), ld, self._at(B, row0, col0), ld,
                                        self._scratch[n].data_ptr(), n, self._out.data_ptr(), self.stream)
        if rc != _cj.CJ_OK:
            raise _cj.CJError(rc, "cj_box_residual")
        return self._out.tolist()

    def block(self, sd: Subdomain, U):
        return U[sd.interior()]


def plan_weights(Nx: int, Ny: int, st: int, tol: float):
    """(w, M, kmin, kmax) of the whole grid's plan (cj_plan_weights: host arithmetic only)."""
    L = _cj._lib()
    M, a, b = ctypes.c_longlong(), ctypes.c_double(), ctypes.c_double()
    rc = L.cj_plan_weights(Nx, Ny, st, tol, 0, None, 0, ctypes.byref(M), ctypes.byref(a), ctypes.byref(b))
    if rc != _cj.CJ_OK:
        raise _cj.CJError(rc, "cj_plan_weights")
    w = (ctypes.c_double * M.value)()
    rc = L.cj_plan_weights(Nx, Ny, st, tol, 0, w, M.value, None, None, None)
    if rc != _cj.CJ_OK:
        raise _cj.CJError(rc, "cj_plan_weights")
    return list(w), M.value, a.value, b.value


def stop_rule(rho: float, fl: float, prev: float, cycles: int, tol: float, stall: int):
    """R8 for plain cycles (patience 1), as cj_solve: (status or None, stall count)."""
    if rho <= tol:
        return _cj.CJ_OK, stall
    if not (rho == rho) or rho > 1e300:
        return _cj.CJ_ERR_DIVERGED, stall
    if rho <= 4.0 * fl:
        return _cj.CJ_FLOOR, stall
    if cycles > 0:
        stall = stall + 1 if rho > 0.5 * prev else 0
        if stall >= 1:
            return _cj.CJ_STALLED, stall
    return None, stall


def solve(part: Partition, st: int, tol: float, f_blocks: dict, backend, comm, K: int = 1,
          max_cycles: int = 64):
    """Plain FP64 CJM of the whole grid by the blocks this process holds (f_blocks: rank ->
    that block's right-hand side, ny x nx, in the backend's arrays), from u = 0.  Returns
    (rank -> the block of u, result dict as cj_solve's: sweeps, cycles, status, rel_res_l2,
    rel_res_inf, floor_est, exchanges)."""
    w, M, _, _ = plan_weights(part.Nx, part.Ny, st, tol)
    h = 1.0 / (part.Nx + 1)
    subs = {rank: Subdomain(part, rank, st, K) for rank in f_blocks}
    B = {rank: backend.zeros(sd.shape) for rank, sd in subs.items()}
    U = [{rank: backend.zeros(sd.shape) for rank, sd in subs.items()} for _ in range(2)]
    for rank, sd in subs.items():
        backend.load_rhs(sd, f_blocks[rank], B[rank], h * h)
    comm.exchange(subs, B, backend)  # b on the halo, once
    S = _ABS_COEFF_SUM[st]
    cur, sweeps, cycles, exchanges, prev, stall = 0, 0, 0, 1, 0.0, 0
    while True:
        comm.exchange(subs, U[cur], backend)
        exchanges += 1
        stats = [backend.residual(sd, U[cur][rank], B[rank]) for rank, sd in subs.items()]
        sums, maxes = comm.allreduce([sum(s[0] for s in stats), sum(s[2] for s in stats), sum(s[3] for s in stats)],
                                     [max(s[1] for s in stats), max(s[4] for s in stats)])
        rn, un, bn = math.sqrt(sums[0]), math.sqrt(sums[1]), math.sqrt(sums[2])
        rho = rn / bn if bn > 0 else rn
        rinf = maxes[0] / maxes[1] if maxes[1] > 0 else maxes[0]
        fl = _EPS * S * un / bn if bn > 0 else _EPS * S * un
        status, stall = stop_rule(rho, fl, prev, cycles, tol, stall)
        if status is not None:
            break
        if cycles >= max_cycles:
            status = _cj.CJ_ERR_NOT_CONVERGED
            break
        for n0 in range(0, M, K):
            if n0 > 0:
                comm.exchange(subs, U[cur], backend)
                exchanges += 1
            for s in range(1, min(K, M - n0) + 1):
                for rank, sd in subs.items():
                    backend.sweep(sd, U[cur][rank], U[1 - cur][rank], B[rank], sd.sweep_box(s), w[n0 + s - 1])
                cur = 1 - cur
        sweeps += M
        cycles += 1
        prev = rho
    blocks = {rank: backend.block(sd, U[cur][rank]) for rank, sd in subs.items()}
    return blocks, {"sweeps": sweeps, "cycles": cycles, "status": status, "rel_res_l2": rho, "rel_res_inf": rinf,
                    "floor_est": fl, "exchanges": exchanges}
