"""Seeded problem sets and request streams of the batched and served workloads.

Draws come from the splitmix64 uniform stream of :mod:`workloads.rhs` (one stream per
purpose, seeded from the workload seed), so every run regenerates the same problems.
"""
from __future__ import annotations

import numpy as np

from .rhs import uniform_stream


def log_uniform_int(u: np.ndarray, lo: int, hi: int) -> np.ndarray:
    """Integers log-uniform in [lo, hi] from uniforms in (0, 1]."""
    v = np.exp(np.log(lo) + (np.log(hi) - np.log(lo)) * (1.0 - u))
    return np.clip(np.rint(v).astype(np.int64), lo, hi)


def batch_problems(n: int = 512, seed: int = 3, lo: int = 64, hi: int = 2048,
                   stencils=(5, 9), tol: float = 1e-8):
    """The batched workload: n independent Dirichlet problems, Nx and Ny drawn independently
    log-uniform in [lo, hi], stencil uniform over `stencils`, smooth random right-hand side
    with per-problem seed seed * 10**6 + index, tolerance tol.  Returns a list of dicts
    (Nx, Ny, st, tol, rhs_seed)."""
    u = uniform_stream(seed, 3 * n).reshape(n, 3)
    nx = log_uniform_int(u[:, 0], lo, hi)
    ny = log_uniform_int(u[:, 1], lo, hi)
    st = np.array(stencils)[np.minimum((u[:, 2] * len(stencils)).astype(int), len(stencils) - 1)]
    return [dict(Nx=int(nx[k]), Ny=int(ny[k]), st=int(st[k]), tol=tol, rhs_seed=seed * 10 ** 6 + k)
            for k in range(n)]


def request_stream(n: int = 10000, seed: int = 4, rate: float = 2000.0, lo: int = 32, hi: int = 8192,
                   stencils=(5, 9, 17), tols=(1e-6, 1e-10)):
    """The served workload: n requests of a Poisson process of `rate` per second
    (exponential inter-arrival times), sides log-uniform in [lo, hi] (Nx, Ny independent),
    stencil uniform over `stencils`, tolerance uniform over `tols`.  Returns a list of dicts
    (t_arrival [s], Nx, Ny, st, tol, rhs_seed)."""
    u = uniform_stream(seed, 5 * n).reshape(n, 5)
    gaps = -np.log(u[:, 0]) / rate
    t = np.cumsum(gaps)
    nx = log_uniform_int(u[:, 1], lo, hi)
    ny = log_uniform_int(u[:, 2], lo, hi)
    st = np.array(stencils)[np.minimum((u[:, 3] * len(stencils)).astype(int), len(stencils) - 1)]
    tl = np.array(tols)[np.minimum((u[:, 4] * len(tols)).astype(int), len(tols) - 1)]
    return [dict(t_arrival=float(t[k]), Nx=int(nx[k]), Ny=int(ny[k]), st=int(st[k]), tol=float(tl[k]),
                 rhs_seed=seed * 10 ** 6 + k) for k in range(n)]
