"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: every expected value comes from the
paper's printed coefficients and bounds (tests/golden/), from a closed form (Chebyshev
polynomials, the stencil symbol, the discrete sine transform), from a dense linear-algebra
routine on a small grid, or from the continuum solution of a manufactured problem.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as orc
import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
STENCILS = (5, 9, 17)


def _golden_coeffs():
    tab = {}
    with open(os.path.join(GOLDEN, "stencil_coefficients.txt")) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if not line:
                continue
            st, dx, dy, v = line.split()
            tab.setdefault(int(st), {})[(int(dx), int(dy))] = float(Fraction(v))
    return tab


COEF = _golden_coeffs()


def symbol(st, theta, phi):
    """Fourier symbol of h^2 Delta_h built from the paper's printed coefficients."""
    return sum(c * np.cos(dx * theta + dy * phi) for (dx, dy), c in COEF[st].items())


def kappa_sym(st, theta, phi):
    """Eigenvalue of D^-1 A for the mode (theta, phi), D = centre coefficient."""
    return symbol(st, theta, phi) / COEF[st][(0, 0)]


def dense_L(st, Nx, Ny):
    n = Nx * Ny
    A = np.zeros((n, n))
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        A[:, k] = orc.apply_L(st, e.reshape(Ny, Nx)).ravel()
    return A


def sine_mode(Nx, Ny, k, l):
    i = np.arange(1, Nx + 1)
    j = np.arange(1, Ny + 1)
    return np.outer(np.sin(l * np.pi * j / (Ny + 1)), np.sin(k * np.pi * i / (Nx + 1)))


def cheb_T(M, x):
    x = float(x)
    if abs(x) <= 1.0:
        return np.cos(M * np.arccos(x))
    s = 1.0 if x > 0 or M % 2 == 0 else -1.0
    return s * np.cosh(M * np.arccosh(abs(x)))


# ----------------------------------------------------------------- stencils

@pytest.mark.parametrize("st", STENCILS)
def test_stencil_matches_paper_coefficients(st):
    """A unit impulse far from the boundary returns the printed coefficients (L is
    symmetric, so the response at offset (dx, dy) is the coefficient there)."""
    N = 9
    u = np.zeros((N, N))
    u[4, 4] = 1.0
    Lu = orc.apply_L(st, u)
    expect = np.zeros((N, N))
    for (dx, dy), c in COEF[st].items():
        expect[4 + dy, 4 + dx] = c
    np.testing.assert_allclose(Lu, expect, rtol=0, atol=1e-15)
    assert orc.centre(st) == pytest.approx(-COEF[st][(0, 0)], rel=1e-15)
    assert orc.radius(st) == max(max(abs(dx), abs(dy)) for dx, dy in COEF[st])


@pytest.mark.parametrize("st", STENCILS)
@pytest.mark.parametrize("Nx,Ny", [(7, 5), (6, 9), (11, 8)])
def test_sine_modes_are_eigenvectors(st, Nx, Ny):
    """With the Dirichlet / odd-reflection boundary every discrete sine mode is an exact
    eigenvector of L with eigenvalue symbol(k pi/(Nx+1), l pi/(Ny+1))."""
    for k, l in [(1, 1), (2, 3), (Nx, 1), (1, Ny), (Nx, Ny), (3, 2)]:
        s = sine_mode(Nx, Ny, k, l)
        lam = symbol(st, k * np.pi / (Nx + 1), l * np.pi / (Ny + 1))
        np.testing.assert_allclose(orc.apply_L(st, s), lam * s, rtol=0, atol=1e-13)


@pytest.mark.parametrize("st", STENCILS)
def test_dense_L_symmetric(st):
    A = dense_L(st, 6, 5)
    np.testing.assert_allclose(A, A.T, rtol=0, atol=1e-15)


# ----------------------------------------------------------------- kappa bounds

@pytest.mark.parametrize("st", STENCILS)
@pytest.mark.parametrize("Nx,Ny", [(4, 4), (7, 5), (10, 12), (12, 9)])
def test_kappa_bounds_vs_dense_eigenvalues(st, Nx, Ny):
    """kmin is the smallest eigenvalue of D^-1 A exactly; kmax bounds the largest."""
    kmin, kmax = orc.kappa_bounds(st, Nx, Ny)
    ev = np.linalg.eigvalsh(dense_L(st, Nx, Ny) / COEF[st][(0, 0)])
    assert kmin == pytest.approx(ev.min(), rel=1e-12)
    assert ev.max() <= kmax * (1 + 1e-14)


@pytest.mark.parametrize("st", STENCILS)
@pytest.mark.parametrize("Nx,Ny", [(16, 16), (64, 64), (1023, 1023), (4096, 4096), (8192, 8192),
                                   (100, 37), (37, 2048)])
def test_kappa_min_formula_equals_symbol(st, Nx, Ny):
    """The paper's sin^2 expressions (N -> Nx+1) equal the symbol at the lowest mode (the
    symbol summed in 40-digit arithmetic: in doubles its cosines cancel badly)."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    kmin, _ = orc.kappa_bounds(st, Nx, Ny)
    th, ph = mp.pi / (Nx + 1), mp.pi / (Ny + 1)
    sym = sum(mp.mpf(c) * mp.cos(dx * th + dy * ph) for (dx, dy), c in COEF[st].items())
    ref = float(sym / mp.mpf(COEF[st][(0, 0)]))
    assert kmin == pytest.approx(ref, rel=1e-12)


@pytest.mark.parametrize("st", STENCILS)
def test_kappa_max_is_symbol_supremum(st):
    _, kmax = orc.kappa_bounds(st, 64, 64)
    t = np.linspace(0, np.pi, 1201)
    T, P = np.meshgrid(t, t)
    sup = kappa_sym(st, T, P).max()
    assert kmax == pytest.approx(sup, rel=1e-12)
    with open(os.path.join(GOLDEN, "kappa_max.txt")) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if line and int(line.split()[0]) == st:
                assert kmax == pytest.approx(float(Fraction(line.split()[1])), rel=1e-15)


def test_kappa_literal_n_convention_differs():
    """The paper-literal N = Nx variant is kept for ablation; it is not the exact bound."""
    a, _ = orc.kappa_bounds(9, 63, 63)
    b, _ = orc.kappa_bounds(9, 63, 63, literal_n=True)
    ref = kappa_sym(9, np.pi / 64, np.pi / 64)
    assert a == pytest.approx(ref, rel=1e-12)
    assert b > a * 1.02


# ----------------------------------------------------------------- weights / plan

@pytest.mark.parametrize("M", [1, 2, 4, 8, 64, 256])
def test_weight_product_is_scaled_chebyshev(M):
    """prod_n (1 - omega_n lam) = T_M((kmax+kmin-2 lam)/(kmax-kmin)) / T_M(sigma)."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    st = 9
    kmin, kmax = orc.kappa_bounds(st, 40, 30)
    omega = orc.sweep_coeffs(st, kmin, kmax, M) * orc.centre(st)
    sig = (kmax + kmin) / (kmax - kmin)
    rng = np.random.default_rng(M)
    lams = [kmin, kmax, 0.5 * (kmin + kmax), 0.5 * kmin, 1.2 * kmax] + list(rng.uniform(kmin, kmax, 6))
    for lam in lams:
        prod = mp.mpf(1)
        for w in omega:
            prod *= 1 - mp.mpf(float(w)) * mp.mpf(lam)
        x = (mp.mpf(kmax) + kmin - 2 * mp.mpf(lam)) / (mp.mpf(kmax) - kmin)
        ref = mp.chebyt(M, x) / mp.chebyt(M, mp.mpf(sig))
        assert abs(prod - ref) <= 1e-8 * max(abs(ref), mp.mpf(1) / mp.chebyt(M, mp.mpf(sig)))


def test_single_weight_is_optimal_stationary_jacobi():
    """M = 1 reduces to weighted Jacobi with omega = 2/(kmin + kmax)."""
    for st in STENCILS:
        kmin, kmax = orc.kappa_bounds(st, 20, 20)
        w = orc.sweep_coeffs(st, kmin, kmax, 1)
        assert w[0] * orc.centre(st) == pytest.approx(2.0 / (kmin + kmax), rel=1e-15)


@pytest.mark.parametrize("M", [1, 2, 4, 16, 512, 8192])
def test_order_is_mirror_paired_permutation(M):
    o = orc.order(M)
    assert sorted(o.tolist()) == list(range(1, M + 1))
    if M >= 2:
        assert np.all(o[0::2] + o[1::2] == M + 1)


def test_order_rejects_non_power_of_two():
    with pytest.raises(ValueError):
        orc.order(12)


def test_order_keeps_partial_products_bounded():
    """Rounding amplification (max partial product over the spectrum) stays modest in the
    pairing order; in sorted order it is astronomically large."""
    st = 5
    kmin, kmax = orc.kappa_bounds(st, 64, 64)
    M = 512
    w = orc.sweep_coeffs(st, kmin, kmax, M) * orc.centre(st)
    lam = np.concatenate([np.linspace(kmin, kmax, 3000), [kmin, kmax]])

    def growth(ws):
        p = np.ones_like(lam)
        g = 0.0
        for x in ws:
            p *= 1 - x * lam
            g = max(g, np.abs(p).max())
        return g

    # prefix products (w) and suffix products (w reversed) both stay bounded ...
    assert growth(w) < 1e4 and growth(w[::-1]) < 1e4
    # ... while sorted order has astronomically large suffix products
    assert growth(np.sort(w)[::-1]) > 1e100


@pytest.mark.parametrize("st", STENCILS)
@pytest.mark.parametrize("N,tol", [(64, 1e-10), (4096, 1e-10), (8192, 1e-10), (300, 1e-6), (33, 1e-8)])
def test_cycle_length_is_minimal_chebyshev_degree(st, N, tol):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    kmin, kmax = orc.kappa_bounds(st, N, N)
    sig = (mp.mpf(kmax) + kmin) / (mp.mpf(kmax) - kmin)
    M0 = orc.cycle_length_min(kmin, kmax, tol)
    assert 1 / mp.cosh(M0 * mp.acosh(sig)) <= tol
    assert M0 == 1 or 1 / mp.cosh((M0 - 1) * mp.acosh(sig)) > tol
    M = orc.cycle_length(kmin, kmax, tol)
    assert M & (M - 1) == 0 and M >= M0 and (M == 1 or M // 2 < M0)


def test_cycle_lengths_of_the_workloads():
    """M of the 5-point 64^2, 9-point 4096^2 and 17-point 8192^2 problems at tol 1e-10."""
    for st, N, M0_range, M in [(5, 64, (400, 600), 512), (9, 4096, (20000, 32768), 32768),
                               (17, 8192, (40000, 65536), 65536)]:
        kmin, kmax = orc.kappa_bounds(st, N, N)
        M0 = orc.cycle_length_min(kmin, kmax, 1e-10)
        assert M0_range[0] <= M0 <= M0_range[1]
        assert orc.cycle_length(kmin, kmax, 1e-10) == M


# ----------------------------------------------------------------- sweeps

@pytest.mark.parametrize("st", [5, 9])
def test_unit_weight_sweep_is_classical_jacobi(st):
    """omega = 1 (w = 1/c) is classical Jacobi: u_i <- (b_i - sum_{j!=i} A_ij u_j) / A_ii."""
    Nx, Ny = 7, 6
    A = dense_L(st, Nx, Ny)
    rng = np.random.default_rng(3)
    u = rng.standard_normal((Ny, Nx))
    b = rng.standard_normal((Ny, Nx))
    d = np.diag(A)
    ref = (b.ravel() - (A - np.diag(d)) @ u.ravel()) / d
    out = orc.sweep(st, u, b, 1.0 / orc.centre(st))
    np.testing.assert_allclose(out.ravel(), ref, rtol=0, atol=1e-13)


def test_17pt_jacobi_uses_constant_centre():
    """For the 17-point stencil the Jacobi D is the constant centre -c (reading R7), not the
    dense diagonal that folds in the reflected ghost."""
    st, Nx, Ny = 17, 7, 6
    A = dense_L(st, Nx, Ny)
    rng = np.random.default_rng(4)
    u = rng.standard_normal((Ny, Nx))
    b = rng.standard_normal((Ny, Nx))
    c = -COEF[st][(0, 0)]
    ref = (b.ravel() - (A + c * np.eye(A.shape[0])) @ u.ravel()) / (-c)
    out = orc.sweep(st, u, b, 1.0 / orc.centre(st))
    np.testing.assert_allclose(out.ravel(), ref, rtol=0, atol=1e-13)
    assert not np.allclose(np.diag(A), -c)


@pytest.mark.parametrize("st", STENCILS)
def test_residual_norms_vs_dense(st):
    Nx, Ny = 9, 7
    A = dense_L(st, Nx, Ny)
    rng = np.random.default_rng(5)
    u = rng.standard_normal((Ny, Nx))
    b = rng.standard_normal((Ny, Nx))
    s, m = orc.residual(st, u, b)
    r = A @ u.ravel() - b.ravel()
    assert s == pytest.approx(np.sum(r * r), rel=1e-13)
    assert m == pytest.approx(np.abs(r).max(), rel=1e-13)


@pytest.mark.parametrize("st", STENCILS)
def test_one_cycle_on_a_sine_mode(st):
    """With b = 0, one cycle multiplies the mode s_kl by T_M(x_kl)/T_M(sigma) exactly."""
    Nx, Ny, M = 20, 16, 64
    kmin, kmax = orc.kappa_bounds(st, Nx, Ny)
    w = orc.sweep_coeffs(st, kmin, kmax, M)
    sig = (kmax + kmin) / (kmax - kmin)
    for k, l in [(1, 1), (3, 5), (Nx, Ny), (7, 2)]:
        s = sine_mode(Nx, Ny, k, l)
        u = s.copy()
        zero = np.zeros_like(s)
        for wn in w:
            u = orc.sweep(st, u, zero, wn)
        kap = kappa_sym(st, k * np.pi / (Nx + 1), l * np.pi / (Ny + 1))
        g = cheb_T(M, (kmax + kmin - 2 * kap) / (kmax - kmin)) / cheb_T(M, sig)
        np.testing.assert_allclose(u, g * s, rtol=0, atol=1e-11)


@pytest.mark.parametrize("st", STENCILS)
def test_one_cycle_residual_bound(st):
    Nx, Ny = 40, 33
    f = workloads.smooth_random_rhs(Nx, Ny, seed=11, kmax=40)
    b = orc.scale_rhs(f)
    kmin, kmax = orc.kappa_bounds(st, Nx, Ny)
    M = orc.cycle_length(kmin, kmax, 1e-6)
    w = orc.sweep_coeffs(st, kmin, kmax, M)
    u = np.zeros_like(b)
    for wn in w:
        u = orc.sweep(st, u, b, wn)
    s, _ = orc.residual(st, u, b)
    rho = np.sqrt(s) / np.linalg.norm(b)
    sig = (kmax + kmin) / (kmax - kmin)
    assert rho <= 1.0 / np.cosh(M * np.arccosh(sig)) * (1 + 1e-6) + 1e-13


def test_scale_rhs_is_h_squared():
    f = np.arange(12.0).reshape(3, 4)
    np.testing.assert_array_equal(orc.scale_rhs(f), f * (1.0 / 5.0) ** 2)


# ----------------------------------------------------------------- converged solutions

@pytest.mark.parametrize("st", STENCILS)
@pytest.mark.parametrize("Nx,Ny", [(1, 1), (3, 2), (7, 5), (12, 9), (16, 16)])
def test_solve_matches_dense_lu(st, Nx, Ny):
    rng = np.random.default_rng(Nx * 100 + Ny)
    f = rng.standard_normal((Ny, Nx))
    out = orc.solve(st, f, 1e-13)
    assert out["converged"] and out["rel_l2"] <= 1e-13
    h = 1.0 / (Nx + 1)
    ref = np.linalg.solve(dense_L(st, Nx, Ny), (h * h * f).ravel()).reshape(Ny, Nx)
    np.testing.assert_allclose(out["u"], ref, rtol=0, atol=1e-11 * np.abs(ref).max())


@pytest.mark.parametrize("st", STENCILS)
def test_solve_matches_discrete_sine_closed_form(st):
    """u* = sum_kl h^2 a_kl / symbol(theta_k, phi_l) s_kl for f = sum_kl a_kl s_kl."""
    Nx, Ny = 48, 40
    k, l, a = workloads.smooth_random_modes(Nx, Ny, seed=7, kmax=30)
    f = workloads.smooth_random_rhs(Nx, Ny, seed=7, kmax=30)
    h = 1.0 / (Nx + 1)
    ustar = np.zeros((Ny, Nx))
    for kk, ll, aa in zip(k, l, a):
        lam = symbol(st, kk * np.pi / (Nx + 1), ll * np.pi / (Ny + 1))
        ustar += h * h * aa / lam * sine_mode(Nx, Ny, kk, ll)
    out = orc.solve(st, f, 1e-11)
    assert out["converged"]
    err = np.linalg.norm(out["u"] - ustar) / np.linalg.norm(ustar)
    assert err < 1e-9


@pytest.mark.parametrize("st,order", [(5, 2.0), (9, 2.0), (17, 4.0)])
def test_manufactured_solution_order(st, order):
    """Error against sin(pi x) sin(pi y) falls at the stencil's formal order."""
    errs = []
    Ns = (15, 31, 63)
    for N in Ns:
        f = workloads.manufactured_rhs(N, N)
        out = orc.solve(st, f, 1e-13)
        errs.append(np.abs(out["u"] - workloads.manufactured_solution(N, N)).max())
    rates = [np.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    for r in rates:
        assert abs(r - order) < 0.25, (errs, rates)


def _closed_form(st, Nx, Ny, seed, kmax):
    k, l, a = workloads.smooth_random_modes(Nx, Ny, seed=seed, kmax=kmax)
    h = 1.0 / (Nx + 1)
    K, L = int(k.max()), int(l.max())
    lam = symbol(st, k * np.pi / (Nx + 1), l * np.pi / (Ny + 1))
    A = np.zeros((L, K))
    A[l - 1, k - 1] = h * h * a / lam
    i = np.arange(1, Nx + 1)
    j = np.arange(1, Ny + 1)
    Sx = np.sin(np.pi * np.outer(np.arange(1, K + 1), i) / (Nx + 1))
    Sy = np.sin(np.pi * np.outer(j, np.arange(1, L + 1)) / (Ny + 1))
    return Sy @ A @ Sx


@pytest.mark.parametrize("st", STENCILS)
def test_rounding_floor_estimate(st):
    """The FP64-rounded exact discrete solution (closed form) has a relative residual of
    the order of eps * S * ||u|| / ||b||: the floor the stop rule uses."""
    N = 384
    ustar = _closed_form(st, N, N, seed=1, kmax=64)
    b = orc.scale_rhs(workloads.smooth_random_rhs(N, N, seed=1, kmax=64))
    s, _ = orc.residual(st, ustar, b)
    rho = np.sqrt(s) / np.linalg.norm(b)
    est = 2.0 ** -53 * orc.abs_coeff_sum(st) * np.linalg.norm(ustar) / np.linalg.norm(b)
    assert 0.1 * est < rho < 4.0 * est


def _floor_estimate(st, u, f, eps=2.0 ** -53):
    """fl = eps S ||u||_2 / ||b||_2 of reading R8, from the returned u (S from the printed
    coefficients' absolute sum, pinned by the impulse-response test)."""
    b = f / (f.shape[1] + 1) ** 2
    return eps * orc.abs_coeff_sum(st) * np.linalg.norm(u) / np.linalg.norm(b)


@pytest.mark.parametrize("st,Nx,Ny,want", [(5, 8, 8, "floor"), (5, 48, 40, "stalled"), (9, 64, 64, "stalled"),
                                           (17, 64, 64, "stalled")])
def test_solve_below_reach_ends_at_floor_or_stall(st, Nx, Ny, want):
    """A tolerance below what FP64 cycles reach ends the solve, not an endless loop: with 'floor'
    when the residual is within 4x of the FP64 floor of the returned u, and with 'stalled' when a
    cycle failed to halve it while it was still above that (the cycle's own rounding, amplified
    by its partial products)."""
    f = workloads.smooth_random_rhs(Nx, Ny, seed=7, kmax=min(30, Nx, Ny))
    out = orc.solve(st, f, 1e-17)
    fl = _floor_estimate(st, out["u"], f)
    assert out["rel_l2"] < 1e-10 and out["cycles"] >= 1
    assert out["status"] == ("floor" if out["rel_l2"] <= 4 * fl else "stalled") == want


def test_too_short_inner_cycle_stalls():
    """Inner cycles too short to contract (M_in = 2, 4, 8 on 64^2) leave the residual near 1 after
    the two outer steps the defect-correction patience allows: 'stalled', far above the floor."""
    f = workloads.smooth_random_rhs(64, 64, seed=7)
    for M_in in (2, 4, 8):
        out = orc.solve_mixed(9, f, 1e-10, M_in)
        assert out["status"] == "stalled" and out["outer"] == 2 and out["rel_l2"] > 0.5
        assert out["rel_l2"] > 1e6 * _floor_estimate(9, out["u"], f)


def test_zero_rhs_converges_immediately():
    out = orc.solve(9, np.zeros((5, 6)), 1e-10)
    assert out["converged"] and out["sweeps"] == 0 and np.all(out["u"] == 0)


def test_solve_rejects_bad_tolerance():
    with pytest.raises(ValueError):
        orc.solve(5, np.ones((4, 4)), 0.0)
    with pytest.raises(ValueError):
        orc.solve(5, np.ones((4, 4)), 1.0)


# ----------------------------------------------------------------- FP32 inner form

def test_fp32_sweep_exact_on_integers():
    """5-point FP32 sweep with small-integer data and w = 1/4: all arithmetic is exact, so
    the result equals the FP64 sweep bit for bit."""
    rng = np.random.default_rng(9)
    e = rng.integers(-50, 50, (11, 13)).astype(np.float32)
    r = rng.integers(-50, 50, (11, 13)).astype(np.float32)
    out32 = orc.sweep_f32(5, e, r, 0.25)
    out64 = orc.sweep(5, e.astype(np.float64), r.astype(np.float64), 0.25)
    np.testing.assert_array_equal(out32.astype(np.float64), out64)


@pytest.mark.parametrize("st", STENCILS)
def test_fp32_impulse_response_is_the_printed_stencil(st):
    """The FP32 sweep (second-difference form) of a unit impulse with r = 0 and w = 1 gives, at
    every node within reach, the coefficient of Fig. 1 / Table 3 at that offset (zero where the
    paper prints none, e.g. the 17-point stencil's knight-move offsets), to FP32 rounding: each
    coefficient's FP32 quotient and the rounding of the centre's 1 + c."""
    n = 11
    e = np.zeros((n, n), dtype=np.float32)
    c = n // 2
    e[c, c] = 1.0
    out = orc.sweep_f32(st, e, np.zeros_like(e), np.float32(1.0)).astype(np.float64)
    out[c, c] -= 1.0
    for dy in range(-3, 4):
        for dx in range(-3, 4):
            # node (c + dx, c + dy) sees the impulse at offset (-dx, -dy); the stencils are symmetric
            want = COEF[st].get((-dx, -dy), 0.0)
            assert abs(out[c + dy, c + dx] - want) <= 4e-7, (dx, dy, out[c + dy, c + dx], want)


@pytest.mark.parametrize("st", STENCILS)
@pytest.mark.parametrize("N", [1024, 8192])
def test_fp32_sweep_keeps_the_lowest_mode(st, N):
    """On the smoothest mode of a fine grid, where L e is ~1e-7 of the values that cancel in
    it, the FP32 sweep's increment w (L e - r) matches the FP64 one to 1e-3 (difference form;
    the pair-sum form is off by ~40 % at 8192^2).  Checked on a 24 x 24 patch of the mode,
    with a weight large enough (1e4, the size of the cycle's largest weights) that the
    increment is not lost in the FP32 rounding of the updated value itself."""
    i = np.arange(1, N + 1)
    mode = np.sin(np.pi * i / (N + 1))
    lo = N // 2 - 12
    e = np.outer(mode[lo:lo + 24], mode[lo:lo + 24]).astype(np.float32)
    # interior nodes of the patch only: embed it so its own boundary does not matter
    r = np.zeros_like(e)
    w = 1.0e4
    out32 = orc.sweep_f32(st, e, r, np.float32(w)).astype(np.float64) - e
    out64 = orc.sweep(st, e.astype(np.float64), r.astype(np.float64), w) - e.astype(np.float64)
    core = (slice(4, 20), slice(4, 20))
    ref = out64[core]
    assert np.abs(out32[core] - ref).max() <= 1e-3 * np.abs(ref).max()


@pytest.mark.parametrize("st", STENCILS)
def test_fp32_sweep_close_to_fp64(st):
    rng = np.random.default_rng(10 + st)
    e = rng.standard_normal((12, 15)).astype(np.float32)
    r = rng.standard_normal((12, 15)).astype(np.float32)
    w = 0.3
    out32 = orc.sweep_f32(st, e, r, np.float32(w))
    out64 = orc.sweep(st, e.astype(np.float64), r.astype(np.float64), float(np.float32(w)))
    np.testing.assert_allclose(out32, out64, rtol=0, atol=2e-6 * np.abs(out64).max())


@pytest.mark.parametrize("st", STENCILS)
def test_defect_is_negated_residual(st):
    rng = np.random.default_rng(20 + st)
    u = rng.standard_normal((9, 10))
    b = rng.standard_normal((9, 10))
    rt, s, m = orc.defect(st, u, b)
    r = b - orc.apply_L(st, u)
    np.testing.assert_array_equal(rt, r.astype(np.float32))
    assert s == pytest.approx(np.sum(r * r), rel=1e-13)


@pytest.mark.parametrize("st", STENCILS)
def test_mixed_precision_reaches_fp64_solution(st):
    Nx, Ny = 48, 40
    f = workloads.smooth_random_rhs(Nx, Ny, seed=3, kmax=30)
    ref = orc.solve(st, f, 1e-11)
    out = orc.solve_mixed(st, f, 1e-10, M_in=64)
    assert out["converged"] and out["rel_l2"] <= 1e-10 and out["outer"] > 1
    err = np.linalg.norm(out["u"] - ref["u"]) / np.linalg.norm(ref["u"])
    assert err < 1e-9


# ----------------------------------------------------------------- double-FP64 outer form

def _exact_residual(st, uh, ul, b):
    """L (uh + ul) - b in exact rational arithmetic, from the printed coefficients and the
    Dirichlet / odd-reflection boundary."""
    Ny, Nx = uh.shape
    coef = {k: Fraction(v).limit_denominator(1000) for k, v in COEF[st].items()}

    def val(i, j):  # node (i, j), 1-based, with ghosts
        s = 1
        if i in (0, Nx + 1) or j in (0, Ny + 1):
            return Fraction(0)
        if i == -1:
            i, s = 1, -s
        elif i == Nx + 2:
            i, s = Nx, -s
        if j == -1:
            j, s = 1, -s
        elif j == Ny + 2:
            j, s = Ny, -s
        return s * (Fraction(float(uh[j - 1, i - 1])) + Fraction(float(ul[j - 1, i - 1])))

    R = [[None] * Nx for _ in range(Ny)]
    for j in range(1, Ny + 1):
        for i in range(1, Nx + 1):
            R[j - 1][i - 1] = sum(c * val(i + dx, j + dy) for (dx, dy), c in coef.items()) \
                - Fraction(float(b[j - 1, i - 1]))
    return R


@pytest.mark.parametrize("st", STENCILS)
def test_double_fp64_residual_exact(st):
    """The double-FP64 residual equals the exact rational residual to FP64 rounding of the
    result, even when it is 1e-12 of the terms that cancel in it."""
    Nx, Ny = 9, 7
    rng = np.random.default_rng(30 + st)
    uh = rng.standard_normal((Ny, Nx))
    ul = uh * rng.uniform(-1e-16, 1e-16, (Ny, Nx))
    # b = L(uh + ul) + tiny perturbation, rounded: the residual is tiny relative to the terms
    Rx = _exact_residual(st, uh, ul, np.zeros_like(uh))
    b = np.array([[float(Rx[j][i]) for i in range(Nx)] for j in range(Ny)])
    b = b + 1e-12 * rng.standard_normal((Ny, Nx)) * np.abs(b)
    ex = _exact_residual(st, uh, ul, b)
    got = orc.residual_dd(st, uh, ul, b)
    for j in range(Ny):
        for i in range(Nx):
            e = ex[j][i]
            assert abs(Fraction(float(got[j, i])) - e) <= abs(e) * Fraction(1, 2 ** 51) + Fraction(1, 10 ** 300)
    # the plain FP64 residual of the same data is far off (that is what the form is for)
    plain = orc.apply_L(st, uh) + orc.apply_L(st, ul) - b
    rel = max(abs(float(plain[j, i]) - float(ex[j][i])) / abs(float(ex[j][i]))
              for j in range(Ny) for i in range(Nx))
    assert rel > 1e-8


def _longdouble_residual(st, uh, ul, b):
    """||L (uh + ul) - b||_2 in numpy long double (64-bit mantissa on x86) from the printed
    coefficients; a check of the double-FP64 claims independent of the oracle's code."""
    LD = np.longdouble
    Ny, Nx = uh.shape
    u = uh.astype(LD) + ul.astype(LD)
    g = np.zeros((Ny + 4, Nx + 4), dtype=LD)
    g[2:-2, 2:-2] = u
    g[0, 2:-2] = -u[1 - 1]      # j = -1 mirrors j = 1
    g[-1, 2:-2] = -u[Ny - 1]    # j = Ny+2 mirrors j = Ny
    g[:, 0] = -g[:, 2]          # i = -1 mirrors i = 1 (corners pick up the second sign)
    g[:, -1] = -g[:, -3]        # i = Nx+2 mirrors i = Nx
    R = -b.astype(LD)
    for (dx, dy), c in COEF[st].items():
        fr = Fraction(c).limit_denominator(1000)
        R = R + (LD(fr.numerator) / LD(fr.denominator)) * g[2 + dy:2 + dy + Ny, 2 + dx:2 + dx + Nx]
    return float(np.sqrt(np.sum(R * R)))


@pytest.mark.parametrize("st", STENCILS)
def test_double_fp64_outer_goes_below_the_fp64_floor(st):
    if np.finfo(np.longdouble).nmant < 63:
        pytest.skip("needs an extended long double for the independent check")
    N, tol = 160, 1e-13
    f = workloads.smooth_random_rhs(N, N, seed=4, kmax=40)
    b = orc.scale_rhs(f)
    fp = orc.solve_mixed(st, f, tol, M_in=512)
    dd = orc.solve_mixed_dd(st, f, tol, M_in=512)
    assert fp["status"] in ("floor", "stalled") and fp["rel_l2"] > tol
    assert (fp["status"] == "floor") == (fp["rel_l2"] <= 4 * _floor_estimate(st, fp["u"], f))
    assert dd["converged"] and dd["rel_l2"] <= tol
    rho = _longdouble_residual(st, dd["u"], dd["u_lo"], b) / np.linalg.norm(b)
    assert rho <= 1.5 * tol
    # and the FP64 solution agrees with the double-FP64 one to FP64 accuracy
    assert np.abs(fp["u"] - dd["u"]).max() <= 1e-9 * np.abs(dd["u"]).max()


# ----------------------------------------------------------------- non-homogeneous Dirichlet

def _dense_zero_ghost(st, Nx, Ny):
    """L on the interior with every ghost value zero, from the printed coefficients."""
    n = Nx * Ny
    A = np.zeros((n, n))
    for j in range(Ny):
        for i in range(Nx):
            for (dx, dy), c in COEF[st].items():
                ii, jj = i + dx, j + dy
                if 0 <= ii < Nx and 0 <= jj < Ny:
                    A[j * Nx + i, jj * Nx + ii] += c
    return A


def _ghost_term(st, Nx, Ny, G):
    """Contribution of the fixed ghost data to L u at every interior node."""
    t = np.zeros((Ny, Nx))
    for j in range(1, Ny + 1):
        for i in range(1, Nx + 1):
            for (dx, dy), c in COEF[st].items():
                ii, jj = i + dx, j + dy
                if ii < 1 or ii > Nx or jj < 1 or jj > Ny:
                    t[j - 1, i - 1] += c * G[jj + 1, ii + 1]
    return t


@pytest.mark.parametrize("st", STENCILS)
@pytest.mark.parametrize("Nx,Ny", [(1, 1), (5, 4), (9, 7), (12, 12)])
def test_dirichlet_data_solve_matches_dense(st, Nx, Ny):
    """With Dirichlet data the solve equals the dense solution of the zero-ghost operator with
    the data moved to the right-hand side."""
    f, _, g = workloads.paper_problem(Nx, Ny)
    G = orc.ghost_ring(Nx, Ny, g)
    out = orc.solve_bc(st, f, G, 1e-13)
    assert out["status"] in ("converged", "floor") and out["rel_l2"] < 1e-12
    h = 1.0 / (Nx + 1)
    rhs = (h * h * f - _ghost_term(st, Nx, Ny, G)).ravel()
    ref = np.linalg.solve(_dense_zero_ghost(st, Nx, Ny), rhs).reshape(Ny, Nx)
    np.testing.assert_allclose(out["u"], ref, rtol=0, atol=1e-11 * np.abs(ref).max())


@pytest.mark.parametrize("st", STENCILS)
@pytest.mark.parametrize("N", [8, 16, 32])
def test_zero_ghost_spectrum_inside_the_kappa_bounds(st, N):
    """The error of a Dirichlet-data solve iterates with the zero-ghost operator; its
    eigenvalues lie inside the paper's [kmin, kmax], so the plan's weights stay valid."""
    ev = np.linalg.eigvalsh(_dense_zero_ghost(st, N, N) / COEF[st][(0, 0)])
    kmin, kmax = orc.kappa_bounds(st, N, N)
    assert ev.min() >= kmin * (1 - 1e-12) and ev.max() <= kmax * (1 + 1e-12)


def test_zero_data_equals_homogeneous_for_radius_one():
    f = workloads.smooth_random_rhs(20, 17, 3)
    G = np.zeros((21, 24))
    for st in (5, 9):
        a = orc.solve_bc(st, f, G, 1e-10)
        b = orc.solve(st, f, 1e-10)
        assert a["sweeps"] == b["sweeps"]
        np.testing.assert_array_equal(a["u"], b["u"])


@pytest.mark.parametrize("st,order", [(5, 2.0), (9, 2.0), (17, 4.0)])
def test_paper_problem_order(st, order):
    """The paper's test problem (Sec. 3.3, u = -e^{xy}): the error against the analytic
    solution falls at the stencil's order."""
    errs = []
    for N in (15, 31, 63):
        f, u, g = workloads.paper_problem(N, N)
        out = orc.solve_bc(st, f, orc.ghost_ring(N, N, g), 1e-13)
        errs.append(np.abs(out["u"] - u).max())
    rates = [np.log2(errs[k] / errs[k + 1]) for k in range(2)]
    for r in rates:
        assert abs(r - order) < 0.3, (errs, rates)


# ----------------------------------------------------------------- real-error stop (Sec. 3.4)

def _to_error_by_hand(st, f, ue, G, tol, err_tol, every):
    """The real-error-stopped solve written out with the pinned one-sweep primitive."""
    Ny, Nx = f.shape
    kmin, kmax = orc.kappa_bounds(st, Nx, Ny)
    M = orc.cycle_length(kmin, kmax, tol)
    w = orc.sweep_coeffs(st, kmin, kmax, M)
    b = orc.scale_rhs(f)
    u = np.zeros_like(f)
    hist, sweeps = [], 0
    while True:
        E = float(np.max(np.abs(u - ue)))
        hist.append((sweeps, E))
        if E <= err_tol:
            return u, sweeps, hist
        for s in range(M):
            u = orc.sweep(st, u, b, w[s]) if G is None else orc.sweep_bc(st, u, G, b, w[s])
            sweeps += 1
            if every and (s + 1) % every == 0 and s + 1 < M:
                E = float(np.max(np.abs(u - ue)))
                hist.append((sweeps, E))
                if E <= err_tol:
                    return u, sweeps, hist


@pytest.mark.parametrize("st", STENCILS)
@pytest.mark.parametrize("every", [0, 5, 16])
@pytest.mark.parametrize("data", [True, False])
def test_solve_to_error_follows_its_definition(st, every, data):
    Nx, Ny = 11, 9
    if data:
        f, ue, g = workloads.paper_problem(Nx, Ny)
        G = orc.ghost_ring(Nx, Ny, g)
    else:
        f, ue, G = workloads.manufactured_rhs(Nx, Ny), workloads.manufactured_solution(Nx, Ny), None
    # the discrete solution's real error plus a margin the iteration must close
    disc = orc.real_error(orc.solve_bc(st, f, G, 1e-13)["u"] if data else orc.solve(st, f, 1e-13)["u"], ue)
    err_tol = disc * 1.05 + 1e-9
    u, sweeps, hist = _to_error_by_hand(st, f, ue, G, 1e-2, err_tol, every)
    out = orc.solve_to_error(st, f, ue, 1e-2, err_tol, G=G, check_every=every)
    assert out["status"] == "converged"
    assert out["sweeps"] == sweeps and out["tests"] == len(hist)
    np.testing.assert_array_equal(out["history"], np.array(hist))
    np.testing.assert_array_equal(out["u"], u)
    assert out["err"] == hist[-1][1] <= err_tol < hist[-2][1]


def test_solve_to_error_below_the_discretisation_error_ends_at_the_floor():
    """A real-error goal below the discretisation error cannot be met: the solve runs until the
    residual stalls, and its real error is then that of the discrete solution."""
    N, st = 15, 5
    f, ue, g = workloads.paper_problem(N, N)
    G = orc.ghost_ring(N, N, g)
    disc = orc.real_error(orc.solve_bc(st, f, G, 1e-13)["u"], ue)
    out = orc.solve_to_error(st, f, ue, 1e-8, disc / 2, G=G)
    assert out["status"] in ("floor", "stalled")
    assert out["err"] == pytest.approx(disc, rel=1e-6)


def test_real_error_is_the_max_norm():
    rng = np.random.default_rng(5)
    u, v = rng.standard_normal((7, 13)), rng.standard_normal((7, 13))
    assert orc.real_error(u, v) == np.max(np.abs(u - v))
    u[3, 4] = np.nan
    assert np.isnan(orc.real_error(u, v))


def test_high_order_reaches_a_real_error_on_a_coarser_mesh():
    """Sec. 3.4, Fig. 4 right, in miniature: the 17-point stencil meets a real-error goal on a
    mesh where the 5-point one cannot, and with fewer sweeps than the 5-point one needs on the
    mesh that can."""
    goal = 1e-6
    f, ue, g = workloads.paper_problem(31, 31)
    hi = orc.solve_to_error(17, f, ue, 1e-8, goal, G=orc.ghost_ring(31, 31, g))
    lo = orc.solve_to_error(5, f, ue, 1e-8, goal, G=orc.ghost_ring(31, 31, g))
    assert hi["status"] == "converged" and lo["status"] in ("floor", "stalled")
    f, ue, g = workloads.paper_problem(63, 63)
    lo = orc.solve_to_error(5, f, ue, 1e-8, goal, G=orc.ghost_ring(63, 63, g))
    assert lo["status"] == "converged" and lo["sweeps"] > hi["sweeps"]


# ----------------------------------------------------------------- classical Jacobi (Sec. 3.4)

@pytest.mark.parametrize("st", STENCILS)
@pytest.mark.parametrize("N,tol", [(15, 1e-6), (24, 1e-4)])
def test_jacobi_damps_the_lowest_mode_by_one_minus_kmin_per_sweep(st, N, tol):
    """omega = 1 multiplies the lowest sine mode by (1 - kmin) per sweep, kmin the paper's bound
    (exact for that mode), so the sweep count and the final residual follow in closed form."""
    h = 1.0 / (N + 1)
    x = np.arange(1, N + 1) * h
    f = np.outer(np.sin(np.pi * x), np.sin(np.pi * x))
    out = orc.solve_jacobi(st, f, tol)
    kmin, kmax = orc.kappa_bounds(st, N, N)
    M = orc.cycle_length(kmin, kmax, tol)
    q = 1.0 - kmin
    n = int(np.ceil(np.log(tol) / (M * np.log(q))))
    assert out["status"] == "converged" and out["sweeps"] == n * M and out["cycles"] == n
    assert out["rel_l2"] == pytest.approx(q ** (n * M), rel=1e-8)


@pytest.mark.parametrize("st", STENCILS)
def test_jacobi_solution_with_data_matches_dense(st):
    Nx, Ny = 7, 6
    f, _, g = workloads.paper_problem(Nx, Ny)
    G = orc.ghost_ring(Nx, Ny, g)
    out = orc.solve_jacobi(st, f, 1e-12, G=G)
    assert out["status"] in ("converged", "floor") and out["rel_l2"] < 1e-11
    h = 1.0 / (Nx + 1)
    rhs = (h * h * f - _ghost_term(st, Nx, Ny, G)).ravel()
    ref = np.linalg.solve(_dense_zero_ghost(st, Nx, Ny), rhs).reshape(Ny, Nx)
    np.testing.assert_allclose(out["u"], ref, rtol=0, atol=1e-10 * np.abs(ref).max())


def test_jacobi_needs_far_more_sweeps_than_cjm():
    f = workloads.smooth_random_rhs(31, 31, 4)
    j = orc.solve_jacobi(9, f, 1e-8)
    c = orc.solve(9, f, 1e-8)
    assert j["status"] == c["status"] == "converged"
    assert j["sweeps"] > 10 * c["sweeps"]
    np.testing.assert_allclose(j["u"], c["u"], rtol=0, atol=1e-7 * np.abs(c["u"]).max())


def test_jacobi_budget_and_argument_checks():
    f = workloads.smooth_random_rhs(20, 20, 1)
    out = orc.solve_jacobi(5, f, 1e-10, max_sweeps=100)
    assert out["status"] == "max_sweeps" and out["sweeps"] <= 100
    with pytest.raises(ValueError):
        orc.solve_jacobi(5, f, 0.0)


# ----------------------------------------------------------------- mixed precision with Dirichlet data

@pytest.mark.parametrize("st", STENCILS)
@pytest.mark.parametrize("dd", [False, True])
def test_mixed_with_data_reaches_the_dense_solution(st, dd):
    """FP32 inner cycles in FP64 (or double-FP64) defect correction with Dirichlet data converge
    to the dense solution of the zero-ghost system with the data moved to the right-hand side."""
    Nx, Ny = 11, 9
    f, _, g = workloads.paper_problem(Nx, Ny)
    G = orc.ghost_ring(Nx, Ny, g)
    solve = orc.solve_mixed_dd if dd else orc.solve_mixed
    out = solve(st, f, 1e-12, 16, G=G, max_outer=200)
    assert out["status"] in ("converged", "floor") and out["rel_l2"] < 1e-11
    h = 1.0 / (Nx + 1)
    rhs = (h * h * f - _ghost_term(st, Nx, Ny, G)).ravel()
    ref = np.linalg.solve(_dense_zero_ghost(st, Nx, Ny), rhs).reshape(Ny, Nx)
    np.testing.assert_allclose(out["u"], ref, rtol=0, atol=1e-10 * np.abs(ref).max())


def test_mixed_with_zero_data_equals_homogeneous_for_radius_one():
    f = workloads.smooth_random_rhs(20, 17, 3)
    G = np.zeros((21, 24))
    for st in (5, 9):
        for solve in (orc.solve_mixed, orc.solve_mixed_dd):
            a = solve(st, f, 1e-10, 32, G=G)
            b = solve(st, f, 1e-10, 32)
            assert a["sweeps"] == b["sweeps"] and a["outer"] == b["outer"]
            np.testing.assert_array_equal(a["u"], b["u"])


def test_mixed_dd_with_data_meets_the_paper_problem_to_its_discretisation_error():
    N, st = 63, 17
    f, ue, g = workloads.paper_problem(N, N)
    G = orc.ghost_ring(N, N, g)
    out = orc.solve_mixed_dd(st, f, 1e-12, 64, G=G, max_outer=300)
    ref = orc.solve_bc(st, f, G, 1e-13)
    assert out["status"] in ("converged", "floor")
    # both are the discrete solution: their real errors agree to a few percent of it
    e_mixed = np.abs(out["u"] - ue).max()
    e_fp64 = np.abs(ref["u"] - ue).max()
    assert e_mixed == pytest.approx(e_fp64, rel=1e-2)


# ----------------------------------------------------------------- real-error stop of defect correction

def _mixed_to_error_by_hand(st, f, ue, goal, M_in):
    """The FP64-outer defect correction stopped by the real error, written out with the pinned
    defect and FP32 sweep primitives (homogeneous boundary)."""
    Ny, Nx = f.shape
    kmin, kmax = orc.kappa_bounds(st, Nx, Ny)
    w32 = orc.sweep_coeffs(st, kmin, kmax, M_in).astype(np.float32)
    b = orc.scale_rhs(f)
    u = np.zeros_like(f)
    hist, sweeps = [], 0
    while True:
        rt, _, _ = orc.defect(st, u, b)
        E = float(np.max(np.abs(u - ue)))
        hist.append((sweeps, E))
        if E <= goal:
            return u, sweeps, hist
        e = np.zeros(f.shape, np.float32)
        for k in range(M_in):
            e = orc.sweep_f32(st, e, rt, w32[k])
        u = u + e.astype(np.float64)
        sweeps += M_in


@pytest.mark.parametrize("st", STENCILS)
def test_mixed_to_error_follows_its_definition(st):
    N, M_in = 23, 32
    f, ue = workloads.manufactured_rhs(N, N), workloads.manufactured_solution(N, N)
    disc = orc.real_error(orc.solve(st, f, 1e-13)["u"], ue)
    goal = disc * 1.05 + 1e-9
    u, sweeps, hist = _mixed_to_error_by_hand(st, f, ue, goal, M_in)
    out = orc.solve_mixed_to_error(st, f, ue, goal, M_in)
    assert out["status"] == "converged" and out["sweeps"] == sweeps
    np.testing.assert_array_equal(out["history"], np.array(hist))
    np.testing.assert_array_equal(out["u"], u)


@pytest.mark.parametrize("st", STENCILS)
def test_mixed_dd_to_error_stops_at_the_iterate_of_the_plain_loop(st):
    """With data and the double-FP64 outer steps: the real-error stop ends at the same iterate as
    the residual-stopped loop run for that many outer steps, with its real error at most the goal."""
    N, M_in = 31, 64
    f, ue, g = workloads.paper_problem(N, N)
    G = orc.ghost_ring(N, N, g)
    disc = orc.real_error(orc.solve_bc(st, f, G, 1e-13)["u"], ue)
    goal = disc * 1.5 + 1e-12
    out = orc.solve_mixed_to_error(st, f, ue, goal, M_in, dd=True, G=G)
    assert out["status"] == "converged" and out["err"] <= goal
    assert out["history"][-1, 1] == out["err"] == orc.real_error(out["u"], ue)
    ref = orc.solve_mixed_dd(st, f, 1e-15, M_in, G=G, max_outer=out["outer"])
    np.testing.assert_array_equal(out["u"], ref["u"])
    np.testing.assert_array_equal(out["u_lo"], ref["u_lo"])


def test_mixed_to_error_goal_below_discretisation_ends_at_the_floor():
    N, st = 23, 9
    f, ue, g = workloads.paper_problem(N, N)
    G = orc.ghost_ring(N, N, g)
    disc = orc.real_error(orc.solve_bc(st, f, G, 1e-13)["u"], ue)
    out = orc.solve_mixed_to_error(st, f, ue, disc / 2, 32, dd=True, G=G, max_outer=400)
    assert out["status"] in ("floor", "stalled")
    assert out["err"] == pytest.approx(disc, rel=1e-6)


# ----------------------------------------------------------------- FP64 inner cycles, double-FP64 outer (R20)

@pytest.mark.parametrize("st", STENCILS)
@pytest.mark.parametrize("Nx,Ny", [(1, 1), (7, 5), (12, 9), (16, 16)])
def test_fp64_dd_matches_dense_lu(st, Nx, Ny):
    """FP64 inner cycles in double-FP64 defect correction converge to the dense solution."""
    rng = np.random.default_rng(Nx * 31 + Ny)
    f = rng.standard_normal((Ny, Nx))
    out = orc.solve_fp64_dd(st, f, 1e-14, 16, max_outer=400)
    assert out["converged"] and out["rel_l2"] <= 1e-14
    h = 1.0 / (Nx + 1)
    ref = np.linalg.solve(dense_L(st, Nx, Ny), (h * h * f).ravel()).reshape(Ny, Nx)
    np.testing.assert_allclose(out["u"], ref, rtol=0, atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("st", STENCILS)
def test_fp64_dd_with_data_reaches_the_dense_solution(st):
    Nx, Ny = 11, 9
    f, _, g = workloads.paper_problem(Nx, Ny)
    G = orc.ghost_ring(Nx, Ny, g)
    out = orc.solve_fp64_dd(st, f, 1e-12, 16, G=G, max_outer=200)
    assert out["converged"] and out["rel_l2"] <= 1e-12
    h = 1.0 / (Nx + 1)
    rhs = (h * h * f - _ghost_term(st, Nx, Ny, G)).ravel()
    ref = np.linalg.solve(_dense_zero_ghost(st, Nx, Ny), rhs).reshape(Ny, Nx)
    np.testing.assert_allclose(out["u"], ref, rtol=0, atol=1e-10 * np.abs(ref).max())


@pytest.mark.parametrize("st", STENCILS)
def test_fp64_dd_goes_below_the_fp64_floor(st):
    """The all-FP64 path reaches a residual below what plain FP64 cycles reach (they stall or hit
    the floor above it), checked by the independent 80-bit residual of u_hi + u_lo."""
    if np.finfo(np.longdouble).nmant < 63:
        pytest.skip("needs an extended long double for the independent check")
    N, tol = 160, 1e-13
    f = workloads.smooth_random_rhs(N, N, seed=4, kmax=40)
    b = orc.scale_rhs(f)
    plain = orc.solve(st, f, tol)
    dd = orc.solve_fp64_dd(st, f, tol, 512)
    assert plain["status"] in ("floor", "stalled") and plain["rel_l2"] > tol
    assert dd["converged"] and dd["rel_l2"] <= tol
    rho = _longdouble_residual(st, dd["u"], dd["u_lo"], b) / np.linalg.norm(b)
    assert rho <= 1.5 * tol
    assert np.abs(plain["u"] - dd["u"]).max() <= 1e-9 * np.abs(dd["u"]).max()


def _two_sum(a, b):
    """Knuth's TwoSum on FP64 arrays: s + e = a + b exactly."""
    s = a + b
    z = s - a
    return s, (a - (s - z)) + (b - z)


@pytest.mark.parametrize("st", STENCILS)
def test_fp64_dd_follows_its_definition(st):
    """R20 written out from the pinned parts -- the double-FP64 defect (residual_dd, pinned
    against exact rational arithmetic), the FP64 sweep (pinned as classical Jacobi and by the
    sine-mode cycle), the cycle's weights, the TwoSum correction and the stop rule of R8 with
    patience 2 and the 2^-106 floor -- gives the oracle's u, u_lo, sweeps and status bit for bit."""
    Nx, Ny, M_in, tol = 23, 19, 32, 1e-13
    f = workloads.smooth_random_rhs(Nx, Ny, seed=9, kmax=12)
    b = orc.scale_rhs(f)
    kmin, kmax = orc.kappa_bounds(st, Nx, Ny)
    w = orc.sweep_coeffs(st, kmin, kmax, M_in)
    uh, ul = np.zeros_like(f), np.zeros_like(f)
    bn, S = np.linalg.norm(b), orc.abs_coeff_sum(st)
    prev, stall, outer, status = 0.0, 0, 0, None
    while True:
        R = orc.residual_dd(st, uh, ul, b)
        rho = np.sqrt(np.sum(R * R)) / bn
        fl = 2.0 ** -106 * S * np.linalg.norm(uh) / bn
        if rho <= tol:
            status = "converged"
        elif rho <= 4 * fl:
            status = "floor"
        elif outer > 0:
            stall = stall + 1 if rho > 0.5 * prev else 0
            status = "stalled" if stall >= 2 else None
        if status:
            break
        e = np.zeros_like(f)
        for n in range(M_in):
            e = orc.sweep(st, e, -R, w[n])
        hi, err = _two_sum(uh, e)
        uh, ul = _two_sum(hi, ul + err)
        prev, outer = rho, outer + 1
    out = orc.solve_fp64_dd(st, f, tol, M_in)
    assert out["status"] == status == "converged" and out["outer"] == outer >= 2
    assert out["sweeps"] == outer * M_in
    np.testing.assert_array_equal(out["u"], uh)
    np.testing.assert_array_equal(out["u_lo"], ul)


def test_fp64_dd_to_error_stops_at_the_iterate_of_the_plain_loop():
    """The real-error stop of R16 on the R20 loop (dd = 2) stops at the iterate the residual-
    stopped loop reaches after the same number of outer steps."""
    N, st, M_in = 31, 9, 64
    f, ue, g = workloads.paper_problem(N, N)
    G = orc.ghost_ring(N, N, g)
    disc = orc.real_error(orc.solve_bc(st, f, G, 1e-13)["u"], ue)
    goal = 2 * disc
    out = orc.solve_mixed_to_error(st, f, ue, goal, M_in, dd=2, G=G)
    assert out["status"] == "converged" and out["err"] <= goal
    assert out["history"][-1, 1] == out["err"] == orc.real_error(out["u"], ue)
    assert out["sweeps"] == out["outer"] * M_in
    ref = orc.solve_fp64_dd(st, f, 1e-15, M_in, G=G, max_outer=out["outer"])
    np.testing.assert_array_equal(out["u"], ref["u"])
    np.testing.assert_array_equal(out["u_lo"], ref["u_lo"])
