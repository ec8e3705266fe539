"""Pins of the oracle's coefficient-mask operator (Sec. 3.2, reading R19) against facts that do
not come from the oracle itself: dense matrices built from the mask's definition, the paper's
uniform stencils, and discrete operators that are exact for quadratic solutions."""
import numpy as np
import pytest

from oracle import oracle as orc
import workloads
from workloads import masks

PATTERNS = (5, 9, 17, 25)


def _dense(P, Nx, Ny):
    """Dense A (interior unknowns, zero ring) and diag, from the mask's definition."""
    offs = orc.mask_offsets(P["pattern"])
    coef = np.broadcast_to(P["coef"], (len(offs) + 1, Ny, Nx))
    s = np.ones((Ny, Nx)) if P["scale"] is None else np.broadcast_to(P["scale"], (Ny, Nx))
    n = Nx * Ny
    A = np.zeros((n, n))
    for j in range(Ny):
        for i in range(Nx):
            row = j * Nx + i
            A[row, row] = s[j, i] * coef[0, j, i]
            for k, (dx, dy) in enumerate(offs):
                ii, jj = i + dx, j + dy
                if 0 <= ii < Nx and 0 <= jj < Ny:
                    A[row, jj * Nx + ii] += s[j, i] * coef[k + 1, j, i]
    return A


def _ring_term(P, Nx, Ny, G):
    """Contribution of the Dirichlet ring to A u at each interior node."""
    offs = orc.mask_offsets(P["pattern"])
    coef = np.broadcast_to(P["coef"], (len(offs) + 1, Ny, Nx))
    s = np.ones((Ny, Nx)) if P["scale"] is None else np.broadcast_to(P["scale"], (Ny, Nx))
    t = np.zeros((Ny, Nx))
    for j in range(1, Ny + 1):
        for i in range(1, Nx + 1):
            for k, (dx, dy) in enumerate(offs):
                ii, jj = i + dx, j + dy
                if ii < 1 or ii > Nx or jj < 1 or jj > Ny:
                    t[j - 1, i - 1] += s[j - 1, i - 1] * coef[k + 1, j - 1, i - 1] * G[jj + 1, ii + 1]
    return t


def _kappa(A):
    ev = np.linalg.eigvals(A / np.diag(A)[:, None])
    assert np.abs(ev.imag).max() < 1e-9 * np.abs(ev).max()
    return ev.real.min(), ev.real.max()


def test_pattern_offsets():
    """Counts and membership of the four patterns; the 17-point one is the point set of Eq. 2."""
    got = {p: orc.mask_offsets(p) for p in PATTERNS}
    assert [len(got[p]) for p in PATTERNS] == [4, 8, 16, 24]
    assert set(got[17]) == {(1, 0), (-1, 0), (0, 1), (0, -1), (1, 1), (1, -1), (-1, 1), (-1, -1),
                            (2, 0), (-2, 0), (0, 2), (0, -2), (2, 2), (2, -2), (-2, 2), (-2, -2)}
    for p in PATTERNS:
        assert got[p] == sorted(got[p], key=lambda o: (o[1], o[0]))  # row-major order


@pytest.mark.parametrize("pat", PATTERNS)
def test_residual_equals_the_dense_normalised_operator(pat):
    Nx, Ny = 7, 6
    P = masks.random_dominant(pat, Nx, Ny, 3 + pat)
    chat, dC = orc.mask_normalize(pat, P["coef"], None, Nx, Ny)
    A = _dense(P, Nx, Ny)
    rng = np.random.default_rng(pat)
    u = rng.standard_normal((Ny, Nx))
    # rho^2 with bhat = 0 is ||D^-1 A u||^2; with one-hot u it gives each column
    for k in range(0, Nx * Ny, 5):
        e = np.zeros(Nx * Ny)
        e[k] = 1.0
        sq, mx = orc.residual_mask(pat, e.reshape(Ny, Nx), None, np.zeros((Ny, Nx)), chat)
        col = A[:, k] / np.diag(A)
        assert sq == pytest.approx(float(col @ col), rel=1e-13)
        assert mx == pytest.approx(np.abs(col).max(), rel=1e-15)
    out = orc.sweep_mask(pat, u, None, np.zeros((Ny, Nx)), chat, 0.7)
    ref = u.ravel() - 0.7 * (A @ u.ravel()) / np.diag(A)
    np.testing.assert_allclose(out.ravel(), ref, rtol=0, atol=1e-13)
    np.testing.assert_array_equal(dC, np.broadcast_to(P["coef"][0], (Ny, Nx)))


@pytest.mark.parametrize("pat", PATTERNS)
def test_jacobi_solve_with_data_equals_dense(pat):
    Nx, Ny = 6, 5
    P = masks.random_dominant(pat, Nx, Ny, 11 + pat)
    G = np.random.default_rng(pat).standard_normal((Ny + 4, Nx + 4))
    G[2:Ny + 2, 2:Nx + 2] = 0.0
    out = orc.solve_mask(pat, P["f"], P["coef"], 0.04, 1.96, 1e-12, G=G, method=1)
    assert out["status"] in ("converged", "floor") and out["rel_l2"] < 1e-11
    A = _dense(P, Nx, Ny)
    ref = np.linalg.solve(A, (P["f"] - _ring_term(P, Nx, Ny, G)).ravel()).reshape(Ny, Nx)
    np.testing.assert_allclose(out["u"], ref, rtol=0, atol=1e-10 * np.abs(ref).max())


@pytest.mark.parametrize("st", (5, 9, 17))
def test_constant_masks_reproduce_the_paper_stencils(st):
    """The uniform stencils written as constant masks (Table 3 Cartesian, Eq. 1, Eq. 2, times
    1/h^2) solve to the stencil solver's answer (zero ring: the data form of R15)."""
    N = 23
    h = 1.0 / (N + 1)
    offs = orc.mask_offsets(st)
    centre = {5: -4.0, 9: -20.0 / 6.0, 17: -300.0 / 72.0}[st]

    def c_of(dx, dy):
        a = max(abs(dx), abs(dy))
        if st == 5:
            return 1.0
        if st == 9:
            return 4.0 / 6.0 if abs(dx) + abs(dy) == 1 else 1.0 / 6.0
        if abs(dx) + abs(dy) == 1:
            return 64.0 / 72.0
        if a == 1:
            return 16.0 / 72.0
        return -4.0 / 72.0 if dx == 0 or dy == 0 else -1.0 / 72.0

    coef = np.array([centre] + [c_of(dx, dy) for dx, dy in offs])[:, None, None] / (h * h)
    f, _, g = workloads.paper_problem(N, N)
    G = orc.ghost_ring(N, N, g)
    kmin, kmax = orc.kappa_bounds(st, N, N)
    m = orc.solve_mask(st, f, coef, kmin, kmax, 1e-10, G=G)
    s = orc.solve_bc(st, f, G, 1e-10)
    assert m["status"] == s["status"] == "converged"
    assert m["sweeps"] == s["sweeps"]
    np.testing.assert_allclose(m["u"], s["u"], rtol=0, atol=1e-9 * np.abs(s["u"]).max())


@pytest.mark.parametrize("maker", ["polar", "stretched", "bipolar"])
def test_masks_exact_for_quadratics_solve_exactly(maker):
    """Polar (u = r^2), non-uniform Cartesian (u = x^2 + y^2) and bipolar (u = mu^2 + nu^2):
    each discrete operator is exact for its quadratic, so the solve returns the analytic
    solution to the solver tolerance."""
    Nx, Ny = 13, 11
    P = {"polar": masks.polar, "stretched": masks.cartesian_stretched, "bipolar": masks.bipolar}[maker](Nx, Ny)
    G = orc.ghost_ring(Nx, Ny, P["g"])
    A = _dense(P, Nx, Ny)
    kmin, kmax = _kappa(A)
    out = orc.solve_mask(5, P["f"], P["coef"], kmin * 0.999, kmax * 1.001, 1e-12, scale=P["scale"], G=G)
    assert out["status"] in ("converged", "floor")
    np.testing.assert_allclose(out["u"], P["u_exact"], rtol=0, atol=1e-9 * np.abs(P["u_exact"]).max())
    # and the dense system agrees (the ring term moved to the right-hand side)
    ref = np.linalg.solve(A, (P["f"] - _ring_term(P, Nx, Ny, G)).ravel()).reshape(Ny, Nx)
    np.testing.assert_allclose(ref, P["u_exact"], rtol=0, atol=1e-10 * np.abs(P["u_exact"]).max())


def test_polar_harmonic_converges_at_second_order():
    errs = []
    for N in (15, 31, 63):
        P = masks.polar(N, N, solution="harmonic")
        # kmin of the polar mask: the dense value on the 15 x 15 grid, scaled by h^2, less 10 %
        kmin = 0.9 * _kappa(_dense(masks.polar(15, 15), 15, 15))[0] * (16.0 / (N + 1)) ** 2
        out = orc.solve_mask(5, P["f"], P["coef"], kmin, 2.0, 1e-12, G=orc.ghost_ring(N, N, P["g"]))
        assert out["status"] in ("converged", "floor"), out["status"]
        errs.append(np.abs(out["u"] - P["u_exact"]).max())
    rates = [np.log2(errs[k] / errs[k + 1]) for k in range(2)]
    assert all(abs(r - 2.0) < 0.25 for r in rates), (errs, rates)


def test_bipolar_scale_cancels_in_the_normalised_operator():
    """With the node factor s the normalised coefficients are those of the constant mask, and
    bhat = f / (s c_C)."""
    Nx, Ny = 9, 8
    P = masks.bipolar(Nx, Ny)
    chat, dC = orc.mask_normalize(5, P["coef"], P["scale"], Nx, Ny)
    chat0, _ = orc.mask_normalize(5, P["coef"], None, Nx, Ny)
    np.testing.assert_array_equal(chat, chat0)
    np.testing.assert_array_equal(dC, P["scale"] * P["coef"][0, 0, 0])


def test_mask_weights_are_the_chebyshev_weights_with_c_one():
    kmin, kmax, M = 0.013, 1.9, 64
    w = orc.mask_weights(kmin, kmax, M)
    nat = orc.weights_natural(kmin, kmax, M)
    np.testing.assert_array_equal(w, nat[orc.order(M) - 1])


def test_mask_argument_checks():
    P = masks.random_dominant(9, 5, 4, 1)
    with pytest.raises(ValueError):
        orc.solve_mask(7, P["f"], P["coef"], 0.1, 1.9, 1e-6)
    with pytest.raises(ValueError):
        orc.solve_mask(9, P["f"], P["coef"], 0.0, 1.9, 1e-6)
    bad = P["coef"].copy()
    bad[0, 2, 3] = 0.0
    with pytest.raises(ValueError):
        orc.solve_mask(9, P["f"], bad, 0.1, 1.9, 1e-6)
