"""Problems posed with position-dependent coefficient masks (Sec. 3.2 of the paper): the
5-point Laplacian in Cartesian coordinates on uniform and non-uniform meshes, in polar and in
bipolar coordinates (the three masks of the paper's table of examples), each with an analytic
solution for Dirichlet data.

Every problem is returned as a dict: `pattern` (5), `coef` (planes: centre, then the
off-centre offsets (0,-1), (-1,0), (1,0), (0,1) -- south, west, east, north -- with trailing
axes of length Ny / Nx or 1 where a plane does not vary along that axis), optional `scale`
s(i, j) multiplying every coefficient, `f`, `u_exact` (interior nodes), and `g(i, j)`
(vectorised) giving the analytic solution at any node index, for the Dirichlet ring.
Node (i, j) sits at coordinates (x1_i, x2_j) with i = 1..Nx, j = 1..Ny; the ring nodes
i, j in {-1, 0, N+1, N+2} continue the same coordinate formulas.  Inputs only: these are
problem definitions, not solver arithmetic.
"""
from __future__ import annotations

import numpy as np


def _planes(C, S, W, E, N):
    return np.stack(np.broadcast_arrays(C, S, W, E, N))


def cartesian_uniform(Nx: int, Ny: int, hx: float, hy: float, u, lap_u):
    """Uniform Cartesian 5-point mask (Table 3, Cartesian) on x_i = i hx, y_j = j hy."""
    i = np.arange(1, Nx + 1)
    j = np.arange(1, Ny + 1)
    X, Y = np.meshgrid(i * hx, j * hy)
    coef = _planes(np.full((1, 1), -2 / hx ** 2 - 2 / hy ** 2), np.full((1, 1), 1 / hy ** 2),
                   np.full((1, 1), 1 / hx ** 2), np.full((1, 1), 1 / hx ** 2), np.full((1, 1), 1 / hy ** 2))
    return dict(pattern=5, coef=coef, scale=None, f=lap_u(X, Y), u_exact=u(X, Y),
                g=lambda ii, jj: u(ii * hx, jj * hy))


def cartesian_stretched(Nx: int, Ny: int, beta: float = 0.6):
    """Non-uniform Cartesian mesh on [0, 1]^2: x(t) = t + beta t (1 - t) / 2 (and y likewise),
    t = i / (Nx + 1), with the three-point second differences of a non-uniform mesh (exact for
    quadratics).  Analytic solution u = x^2 + y^2 (Delta u = 4)."""
    def xmap(t):
        return t + 0.5 * beta * t * (1.0 - t)

    def coords(n, idx):
        return xmap(idx / (n + 1.0))

    i = np.arange(1, Nx + 1)
    j = np.arange(1, Ny + 1)
    x, xm, xp = coords(Nx, i), coords(Nx, i - 1), coords(Nx, i + 1)
    y, ym, yp = coords(Ny, j), coords(Ny, j - 1), coords(Ny, j + 1)
    hw, he = x - xm, xp - x
    hs, hn = y - ym, yp - y
    W = (2.0 / (hw * (hw + he)))[None, :]
    E = (2.0 / (he * (hw + he)))[None, :]
    S = (2.0 / (hs * (hs + hn)))[:, None]
    N = (2.0 / (hn * (hs + hn)))[:, None]
    C = -(2.0 / (hw * he))[None, :] - (2.0 / (hs * hn))[:, None]
    X, Y = np.meshgrid(x, y)

    def u(a, b):
        return a * a + b * b

    return dict(pattern=5, coef=_planes(C, S, W, E, N), scale=None, f=np.full((Ny, Nx), 4.0),
                u_exact=u(X, Y), g=lambda ii, jj: u(coords(Nx, ii), coords(Ny, jj)))


def polar(Nx: int, Ny: int, r0: float = 1.0, r1: float = 2.0, th0: float = 0.0,
          th1: float = 0.5 * np.pi, solution: str = "r2"):
    """Polar 5-point mask (Table 3, polar): r_i = r0 + i dr, theta_j = th0 + j dth on the annulus
    sector [r0, r1] x [th0, th1]; W/E = 1/dr^2 -+ 1/(2 r_i dr), S/N = 1/(r_i^2 dth^2),
    C = -2/dr^2 - 2/(r_i^2 dth^2) -- planes that depend on r (i) only.
    solution "r2": u = r^2, Delta u = 4 (the discrete operator is exact for it);
    "harmonic": u = r^3 cos(3 theta), Delta u = 0."""
    dr = (r1 - r0) / (Nx + 1)
    dth = (th1 - th0) / (Ny + 1)
    r = r0 + np.arange(1, Nx + 1) * dr
    W = (1 / dr ** 2 - 1 / (2 * r * dr))[None, :]
    E = (1 / dr ** 2 + 1 / (2 * r * dr))[None, :]
    S = (1 / (r * r * dth ** 2))[None, :]
    C = (-2 / dr ** 2 - 2 / (r * r * dth ** 2))[None, :]
    if solution == "r2":
        def u(rr, tt):
            return rr * rr + 0.0 * tt
        lap = 4.0
    else:
        def u(rr, tt):
            return rr ** 3 * np.cos(3 * tt)
        lap = 0.0
    R, T = np.meshgrid(r, th0 + np.arange(1, Ny + 1) * dth)
    return dict(pattern=5, coef=_planes(C, S, W, E, S), scale=None, f=np.full((Ny, Nx), lap),
                u_exact=u(R, T), g=lambda ii, jj: u(r0 + ii * dr, th0 + jj * dth))


def bipolar(Nx: int, Ny: int, a: float = 1.0, mu0: float = 0.5, mu1: float = 2.5, nu0: float = 0.3,
            nu1: float = 1.5):
    """Bipolar 5-point mask (Table 3, bipolar) on mu_i = mu0 + i dmu, nu_j = nu0 + j dnu: a
    constant mask (C = -2/dmu^2 - 2/dnu^2, W/E = 1/dmu^2, S/N = 1/dnu^2) times the node factor
    s = (cosh nu_j - cos mu_i) / a^2, as printed.  With that operator the analytic solution
    u = mu^2 + nu^2 has A u = 4 s (the mask is exact for quadratics in (mu, nu))."""
    dmu = (mu1 - mu0) / (Nx + 1)
    dnu = (nu1 - nu0) / (Ny + 1)
    mu = mu0 + np.arange(1, Nx + 1) * dmu
    nu = nu0 + np.arange(1, Ny + 1) * dnu
    MU, NU = np.meshgrid(mu, nu)
    s = (np.cosh(NU) - np.cos(MU)) / (a * a)
    one = np.ones((1, 1))
    coef = _planes(one * (-2 / dmu ** 2 - 2 / dnu ** 2), one / dnu ** 2, one / dmu ** 2, one / dmu ** 2,
                   one / dnu ** 2)

    def u(m, n):
        return m * m + n * n

    return dict(pattern=5, coef=coef, scale=s, f=4.0 * s, u_exact=u(MU, NU),
                g=lambda ii, jj: u(mu0 + ii * dmu, nu0 + jj * dnu))


def random_dominant(pattern: int, Nx: int, Ny: int, seed: int):
    """Random position-dependent coefficients of a given pattern (full planes): off-centre
    entries uniform in [0.1, 1], centre -(1.05 .. 1.5) x the sum of the off-centre ones, so
    the Jacobi-normalised operator has its spectrum in (0, 2).  f uniform in [-1, 1]."""
    from .rhs import uniform_stream
    K = {5: 4, 9: 8, 17: 16, 25: 24}[pattern]
    n = Nx * Ny
    v = uniform_stream(seed, (K + 2) * n)
    off = 0.1 + 0.9 * v[:K * n].reshape(K, Ny, Nx)
    C = -(1.05 + 0.45 * v[K * n:(K + 1) * n].reshape(Ny, Nx)) * off.sum(axis=0)
    f = 2.0 * v[(K + 1) * n:(K + 2) * n].reshape(Ny, Nx) - 1.0
    return dict(pattern=pattern, coef=np.concatenate([C[None], off]), scale=None, f=f,
                u_exact=None, g=None)
