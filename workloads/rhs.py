"""Right-hand sides f of Delta u = f on the uniform mesh of the Chebyshev-Jacobi solver.

Mesh: interior nodes i = 1..Nx, j = 1..Ny, spacing h = 1/(Nx+1) in both directions
(uniform mesh, Sec. 2.1 of the paper), so the domain is [0, 1] x [0, Ly], Ly = (Ny+1) h.
Arrays are interior-only, shape (Ny, Nx), row-major: f[j-1, i-1] = f(i h, j h).

Random numbers: splitmix64 (Steele, Lea and Flood, 2014) feeding a Box-Muller transform,
both written here from their published definitions, so any language can regenerate the
same stream.
"""
from __future__ import annotations

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def grid_h(Nx: int) -> float:
    return 1.0 / (Nx + 1)


def splitmix64_stream(seed: int, n: int) -> np.ndarray:
    """n outputs of splitmix64 started from state ``seed`` (uint64)."""
    with np.errstate(over="ignore"):
        k = np.arange(1, n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform_stream(seed: int, n: int) -> np.ndarray:
    """n doubles in (0, 1]: top 53 bits of splitmix64, mapped away from zero."""
    z = splitmix64_stream(seed, n)
    return 1.0 - (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def gaussian_stream(seed: int, n: int) -> np.ndarray:
    """n standard normal deviates by Box-Muller on consecutive uniform pairs."""
    u = uniform_stream(seed, 2 * n)
    u1, u2 = u[0::2], u[1::2]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def manufactured_solution(Nx: int, Ny: int) -> np.ndarray:
    """u = sin(pi x) sin(pi y / Ly) at the interior nodes (sin(pi x) sin(pi y) on the unit
    square when Nx == Ny)."""
    h = grid_h(Nx)
    Ly = (Ny + 1) * h
    x = np.arange(1, Nx + 1) * h
    y = np.arange(1, Ny + 1) * h
    return np.outer(np.sin(np.pi * y / Ly), np.sin(np.pi * x))


def manufactured_rhs(Nx: int, Ny: int) -> np.ndarray:
    """f = Delta u of :func:`manufactured_solution`: -pi^2 (1 + 1/Ly^2) sin sin, which is
    -2 pi^2 sin(pi x) sin(pi y) on the unit square."""
    h = grid_h(Nx)
    Ly = (Ny + 1) * h
    return -(np.pi ** 2) * (1.0 + 1.0 / (Ly * Ly)) * manufactured_solution(Nx, Ny)


def smooth_random_modes(Nx: int, Ny: int, seed: int, kmax: int = 64):
    """Sine modes (k, l), k, l >= 1, k^2 + l^2 <= kmax^2, k <= Nx, l <= Ny, in (k, l)
    lexicographic order, with amplitudes a_kl = g_kl / (k^2 + l^2), g ~ N(0, 1) from the
    seeded stream.  Returns (k, l, a) as arrays."""
    ks, ls = [], []
    for k in range(1, min(kmax, Nx) + 1):
        for l in range(1, min(kmax, Ny) + 1):
            if k * k + l * l <= kmax * kmax:
                ks.append(k)
                ls.append(l)
    k = np.array(ks, dtype=np.int64)
    l = np.array(ls, dtype=np.int64)
    g = gaussian_stream(seed, len(k))
    a = g / (k * k + l * l).astype(np.float64)
    return k, l, a


def smooth_random_rhs(Nx: int, Ny: int, seed: int, kmax: int = 64) -> np.ndarray:
    """f(x_i, y_j) = sum_kl a_kl sin(k pi i/(Nx+1)) sin(l pi j/(Ny+1)) for the modes of
    :func:`smooth_random_modes` (amplitude decaying as |k|^-2 up to |k| <= kmax)."""
    k, l, a = smooth_random_modes(Nx, Ny, seed, kmax)
    if len(k) == 0:
        return np.zeros((Ny, Nx))
    K, L = int(k.max()), int(l.max())
    A = np.zeros((L, K))
    A[l - 1, k - 1] = a
    i = np.arange(1, Nx + 1)
    j = np.arange(1, Ny + 1)
    Sx = np.sin(np.pi * np.outer(np.arange(1, K + 1), i) / (Nx + 1))   # (K, Nx)
    Sy = np.sin(np.pi * np.outer(j, np.arange(1, L + 1)) / (Ny + 1))   # (Ny, L)
    return np.ascontiguousarray(Sy @ A @ Sx)


def paper_problem(Nx: int, Ny: int):
    """The paper's test problem (Sec. 3.3): Delta u = -(x^2 + y^2) e^{xy} with the Dirichlet
    data of its analytic solution u = -e^{xy}, on the uniform mesh x_i = i h, y_j = j h,
    h = 1/(Nx+1) (the unit square when Nx == Ny).  Returns (f, u_exact, g): f and u_exact at
    the interior nodes, and g(i, j) = u(i h, j h) for any node (the boundary data, also at the
    second ring the 17-point stencil reaches)."""
    h = grid_h(Nx)
    x = np.arange(1, Nx + 1) * h
    y = np.arange(1, Ny + 1) * h
    X, Y = np.meshgrid(x, y)
    f = -(X * X + Y * Y) * np.exp(X * Y)
    u = -np.exp(X * Y)

    def g(i, j):
        return -np.exp((i * h) * (j * h))

    return f, u, g
