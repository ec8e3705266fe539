// Plan numerics of the Chebyshev-Jacobi method (Sec. 2.1): eigenvalue bounds, cycle
// length, Chebyshev weights and their application order.  Host FP64, compiled with
// -ffp-contract=off so each expression rounds exactly as written.
#include <cmath>
#include <vector>

#include "cj_internal.h"

namespace {
const double kPi = 3.14159265358979323846;
inline double sin2(double x) {
    double s = std::sin(x);
    return s * s;
}
}  // namespace

// c = -(centre coefficient of h^2 Delta_h): Table 3 (5-point), Eq. 1 (9-point: -20/6),
// Eq. 2 (17-point: -300/72).
double plan_centre(int st) {
    if (st == 5) return 4.0;
    if (st == 9) return 20.0 / 6.0;
    return 300.0 / 72.0;
}

// Sum of the absolute coefficients of h^2 Delta_h (the FP64 rounding-floor factor S).
double plan_abs_coeff_sum(int st) {
    if (st == 5) return 8.0;
    if (st == 9) return 40.0 / 6.0;
    return 640.0 / 72.0;
}

// [kmin, kmax] of D^-1 A.  nint_x, nint_y are the paper's N: Nx + 1 intervals for the
// exact bound, Nx for the paper-literal variant.  9- and 17-point: the closed forms
// printed after Eq. 1 and Eq. 2; 5-point: the same Fourier analysis of Table 3's stencil.
void plan_kappa_bounds(int st, double nint_x, double nint_y, double *kmin, double *kmax) {
    double hx = kPi / (2.0 * nint_x), hy = kPi / (2.0 * nint_y);  // pi / 2N
    if (st == 5) {
        *kmin = sin2(hx) + sin2(hy);
        *kmax = 2.0;
        return;
    }
    if (st == 9) {
        *kmin = (4.0 / 5.0) * (sin2(hx) + sin2(hy)) + (1.0 / 5.0) * (sin2(hx + hy) + sin2(hx - hy));
        *kmax = 8.0 / 5.0;
        return;
    }
    double fx = kPi / nint_x, fy = kPi / nint_y;  // pi / N
    *kmin = -(4.0 / 75.0) * (sin2(fx) + sin2(fy)) + (64.0 / 75.0) * (sin2(hx) + sin2(hy)) -
            (1.0 / 75.0) * (sin2(fx + fy) + sin2(fx - fy)) +
            (16.0 / 75.0) * (sin2(hx + hy) + sin2(hx - hy));
    *kmax = 128.0 / 75.0;
}

// Smallest power of two M with 1/T_M(sigma) <= tol, sigma = (kmax+kmin)/(kmax-kmin).
// acosh(sigma) is taken as log1p(d + sqrt(d (2 + d))), d = sigma - 1, to keep its digits
// when kmin << kmax.
long long plan_cycle_length(double kmin, double kmax, double tol) {
    double d = 2.0 * kmin / (kmax - kmin);
    double a = std::log1p(d + std::sqrt(d * (2.0 + d)));
    double need = std::log(1.0 / tol + std::sqrt(1.0 / (tol * tol) - 1.0));
    double m0 = std::ceil(need / a);
    long long m = 1;
    while ((double)m < m0) m *= 2;
    return m;
}

// Inner FP32 cycle length of the mixed-precision solve.  One outer step multiplies the
// error by about q(M) = max(2 exp(-M theta), eps32 G(M)): the Chebyshev factor of an M-sweep
// cycle (theta = acosh sigma) or the FP32 rounding amplified by the partial products of the
// mirror-pairing order, G(M) ~ 10^(2.6 + 0.62 log2(M / 512)) (measured growth: 10^2.6 at
// M = 512, 10^5.1 at 8192, 10^6.9 at 65536).  The rule takes the power of two that
// minimises sweeps per decade, M / log10(1/q(M)), and at most the FP64 cycle length M.
// On the 9-point 4096^2 problem it gives 4096, the measured best (53k FP32 sweeps to
// 1e-10 against 131k at 8192 and 51k-55k at 2048).
long long plan_inner_cycle(double kmin, double kmax, long long M) {
    const double d = 2.0 * kmin / (kmax - kmin);
    const double theta = std::log1p(d + std::sqrt(d * (2.0 + d)));
    const double eps32 = 5.9604644775390625e-08;  // 2^-24
    long long best = 1;
    double best_cost = 1e300;
    for (long long m = 2; m <= 65536 && m <= M; m *= 2) {
        const double cheb = 2.0 * std::exp(-(double)m * theta);
        const double growth = std::pow(10.0, 2.6 + 0.62 * std::log2((double)m / 512.0));
        const double q = std::fmax(cheb, eps32 * growth);
        if (q >= 0.5) continue;
        const double cost = (double)m / std::log10(1.0 / q);
        if (cost < best_cost) {
            best_cost = cost;
            best = m;
        }
    }
    if (best_cost == 1e300) best = M < 2 ? M : 2;
    return best;
}

// Inner FP64 cycle length of the double-FP64 defect correction with FP64 inner cycles.  One
// outer step multiplies the error by about q(M) = max(2 exp(-M theta), eps64 G(M)) (the
// Chebyshev factor, or FP64 rounding amplified by the partial products as in plan_inner_cycle);
// the solve from u = 0 then needs ceil(log(1/tol) / log(1/q)) steps.  The rule takes the power
// of two with the fewest sweeps in total, the shorter cycle on a tie (it restarts the
// contraction more often).  Measured on the 9-point 4096^2 problem to 1e-10 (FP64 sweeps,
// outer steps, time): 4096: 28,672 in 7 steps, 7.74 s; 8192: 32,768 in 4, 8.85 s; 16384:
// 32,768 in 2, 8.84 s; 32768: 65,536 in 2, 17.7 s -- the rule picks 4096.
long long plan_inner_cycle_fp64(double kmin, double kmax, long long M, double tol) {
    const double d = 2.0 * kmin / (kmax - kmin);
    const double theta = std::log1p(d + std::sqrt(d * (2.0 + d)));
    const double eps64 = 1.1102230246251565e-16;  // 2^-53
    const double need = std::log(1.0 / tol);
    long long best = M < 2 ? M : 2;
    double best_total = 1e300;
    for (long long m = 2; m <= (1LL << 20) && m <= M; m *= 2) {
        const double cheb = 2.0 * std::exp(-(double)m * theta);
        const double growth = std::pow(10.0, 2.6 + 0.62 * std::log2((double)m / 512.0));
        const double q = std::fmax(cheb, eps64 * growth);
        if (q >= 0.5) continue;
        const double total = (double)m * std::ceil(need / std::log(1.0 / q) - 1e-9);
        if (total < best_total) {
            best_total = total;
            best = m;
        }
    }
    return best;
}

// Per-sweep coefficients w_n = 1 / (c * lambda_{o(n)}), lambda_j = (kmax+kmin)/2 +
// (kmax-kmin)/2 * cos((2j-1) pi / 2M), applied in the mirror-pairing order o: o = (1)
// for M = 1; going from m to 2m, every entry j of o is followed by 2m+1-j.
void plan_sweep_coeffs(int st, double kmin, double kmax, long long M, std::vector<double> &w) {
    plan_sweep_coeffs_c(plan_centre(st), kmin, kmax, M, w);
}

void plan_sweep_coeffs_c(double c, double kmin, double kmax, long long M, std::vector<double> &w) {
    std::vector<long long> o(1, 1), next;
    for (long long m = 1; m < M; m *= 2) {
        next.resize(2 * m);
        for (long long k = 0; k < m; ++k) {
            next[2 * k] = o[k];
            next[2 * k + 1] = 2 * m + 1 - o[k];
        }
        o.swap(next);
    }
    double mid = 0.5 * (kmax + kmin), half = 0.5 * (kmax - kmin);
    w.resize(M);
    for (long long n = 0; n < M; ++n) {
        double x = std::cos((double)(2 * o[n] - 1) * kPi / (double)(2 * M));
        double lam = mid + half * x;
        w[n] = 1.0 / (c * lam);
    }
}
