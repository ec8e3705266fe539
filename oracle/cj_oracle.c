/*
 * cj_oracle.c -- plain, slow, single-threaded FP64 reference of the Chebyshev-Jacobi
 * method (CJM) for the 2-D finite-difference Poisson problem.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or calls
 * this file; only the test-suite, the smoke check and the CPU-baseline leg of the
 * benchmark use it.  It shares no code, header or constant table with the CUDA path.
 *
 * What it follows (Adsuara et al., "Speeding up a few orders of magnitude the Jacobi
 * method: high order Chebyshev-Jacobi over GPUs"):
 *   - Sec. 2.1: CJM = weighted Jacobi with a different weight at every iteration; the
 *     weights are precomputed from the zeros of a Chebyshev polynomial mapped onto the
 *     eigenvalue interval [kmin, kmax] of the Jacobi iteration matrix.
 *   - Table 3 (Cartesian row): the classical 5-point Laplacian.
 *   - Eq. 1 / Fig. 1 (left): the 9-point, first-family, alpha = 2/3 Laplacian.
 *   - Eq. 2 / Fig. 1 (right): the 17-point, second-family, alpha = 2/3 Laplacian.
 *   - Eqs. for kmin^(9), kmax^(9) and kmin^(17), kmax^(17) in Sec. 2.1.
 *   - Sec. 3.2: node indices 1 <= i <= Nx, 1 <= j <= Ny.
 *
 * Readings where the paper is silent (each one is listed, with its reason, in the
 * design notes of the repository):
 *   R1 weights: omega_j = 1/lambda_j, lambda_j = (kmax+kmin)/2 + (kmax-kmin)/2 *
 *      cos((2j-1) pi / 2M), j = 1..M  (Chebyshev-Richardson; the paper's "transformation
 *      of the zeros of a Chebyshev polynomial").  The sweep multiplies by w = omega/c.
 *   R2 cycle length: M0 = ceil(acosh(1/tol) / acosh(sigma)), sigma = (kmax+kmin)/(kmax-kmin);
 *      M = smallest power of two >= M0.
 *   R3 order of the weights: recursive mirror pairing (1), then each index j of the
 *      order for m is followed by its mirror 2m+1-j in the order for 2m.
 *   R4 N in the kappa formulas is the number of intervals, Nx+1 (nodes 1..Nx, h = 1/(Nx+1)).
 *   R5 5-point bounds: kmin = sin^2(pi/2(Nx+1)) + sin^2(pi/2(Ny+1)), kmax = 2.
 *   R6 boundary: homogeneous Dirichlet; nodes 0 and N+1 hold 0; the 17-point stencil's
 *      second ghost layer is the odd reflection u[-1] = -u[1], u[N+2] = -u[N].
 *   R7 D is the constant stencil centre (-c in units of 1/h^2).
 *   R8 stop test: relative L2 residual rho = ||b - L u||_2 / ||b||_2 <= tol, checked
 *      before every cycle; u0 = 0 unless given.  If ||b|| = 0 the absolute norm is used.
 *      rho cannot fall below the rounding floor of an FP64 u, about
 *      fl = eps * S * ||u||_2 / ||b||_2 (eps = 2^-53, S = sum of |coefficients|), which is
 *      ~5e-10 for the 9-point stencil on 4096^2; so the solve also stops: with the status
 *      "floor" once rho <= 4 fl, and with the status "stalled" once `patience`
 *      consecutive cycles each failed to halve rho while it is still above 4 fl
 *      (patience 1 for plain CJM cycles; 2 for the defect-correction loop of R10, whose
 *      residual may jump up once before contracting).
 *   R9 evaluation order of the residual L u - b (any order is exact in real arithmetic):
 *      horizontal pair sums p = u(i-1,.) + u(i+1,.), P = u(i-2,.) + u(i+2,.), vertical
 *      pair sums v1 = u(i,j-1) + u(i,j+1), v2 = u(i,j-2) + u(i,j+2); axis groups
 *      p(j) + v1, P(j) + v2; diagonal groups p(j-1) + p(j+1), P(j-2) + P(j+2); the
 *      coefficients applied by nested fma, innermost fma(centre, u(i,j), -b).
 *   R10 mixed precision (not in the paper; the FP32-inner / FP64-outer form): an outer
 *      FP64 defect-correction loop r = b - L u, rt = (float) r, one FP32 CJM cycle of
 *      length M_in on L e = rt from e = 0 with w32_n = (float)(omega_n / c), then
 *      u <- u + (double) e.  The stop test is the FP64 residual of R8.
 *   R11 double-FP64 outer (not in the paper): as R10, but the solution is the unevaluated
 *      sum u_hi + u_lo of two FP64 arrays and the defect is evaluated to about twice FP64
 *      precision: D (L u_hi - b), D = 1, 6 or 72 the stencil's denominator, is a sum of
 *      terms that are exact in FP64 (power-of-two multiples of u_hi and b), added by the
 *      error-free TwoSum cascade (Ogita, Rump and Oishi's Sum2); D L u_lo is added in plain
 *      FP64.  The correction is added by TwoSum.  This removes the FP64 floor of R8.
 *   R14 FP32 evaluation (not in the paper): the FP32 inner sweep evaluates L e - r from
 *      horizontal and vertical second differences of neighbour differences, an exact
 *      rewriting of Eq. 1 and Eq. 2's stencils (see resid_at32); on a 8192^2 grid the
 *      pair-sum form loses ~40 % of the lowest mode's L e in FP32, the difference forms keep
 *      it to a few FP32 ulps.
 *   R15 non-homogeneous Dirichlet (Sec. 3.3's test problem): the data fill the two-node
 *      ring around the interior and stay fixed (see orc_solve_bc).
 *   R16 real-error stop (Sec. 3.4, Fig. 4 right): the infinity norm of u - u_exact tested
 *      before every cycle and every check_every sweeps (see orc_solve_to_error).
 *   R18 classical Jacobi (the comparison method of Sec. 3.4): omega = 1, residual tested every
 *      M sweeps (see orc_solve_jacobi).
 *   R19 position-dependent coefficient masks (Sec. 3.2): the Jacobi-normalised sweep with the
 *      caller's eigenvalue bounds (see orc_solve_mask).
 *   R20 FP64 inner cycles (not in the paper): R11's double-FP64 outer loop with the inner
 *      cycle run by the plain FP64 sweep of R9 on L e = r, r = -R in FP64 (see
 *      orc_solve_fp64_dd) -- the all-FP64 way to a residual below one array's FP64 floor.
 *
 * Array convention: interior values only, row-major [Ny][Nx], value of node (i, j) at
 * u[(j-1)*Nx + (i-1)].  Compiled with -ffp-contract=off so that every rounding is the
 * one written here.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846

/* ---------------------------------------------------------------- stencils */

/* Stencil radius: 1 for the 5- and 9-point stencils, 2 for the 17-point one. */
int orc_radius(int st) { return st == 17 ? 2 : 1; }

/* c = -(centre coefficient) of L = h^2 * Delta_h (Table 3, Eq. 1, Eq. 2). */
double orc_centre(int st) {
    if (st == 5) return 4.0;
    if (st == 9) return 20.0 / 6.0;
    return 300.0 / 72.0;
}

/* Value of node (i, j), with the homogeneous Dirichlet boundary and the odd
 * reflection for the second ghost layer (reading R6). */
static double at(const double *u, int Nx, int Ny, int i, int j) {
    double s = 1.0;
    if (i == 0 || i == Nx + 1 || j == 0 || j == Ny + 1) return 0.0;
    if (i == -1) { i = 1; s = -s; } else if (i == Nx + 2) { i = Nx; s = -s; }
    if (j == -1) { j = 1; s = -s; } else if (j == Ny + 2) { j = Ny; s = -s; }
    return s * u[(size_t)(j - 1) * Nx + (i - 1)];
}

/* r = (L u)(i, j) - bk in units of 1/h^2, evaluated in the order of reading R9:
 * horizontal pair sums p(j) = u(i-1,j) + u(i+1,j), P(j) = u(i-2,j) + u(i+2,j) and vertical
 * pair sums v1 = u(i,j-1) + u(i,j+1), v2 = u(i,j-2) + u(i,j+2); the centre term and -bk
 * sit in the innermost fma.  With bk = 0 it returns (L u)(i, j) exactly. */
static double resid_at(int st, const double *u, int Nx, int Ny, int i, int j, double bk) {
    double uC = at(u, Nx, Ny, i, j);
    double v1 = at(u, Nx, Ny, i, j - 1) + at(u, Nx, Ny, i, j + 1);
    double p0 = at(u, Nx, Ny, i - 1, j) + at(u, Nx, Ny, i + 1, j);
    if (st == 5) {
        /* Table 3, Cartesian, dx = dy = h: four neighbours with weight 1, centre -4. */
        double a = p0 + v1;
        return a + fma(-4.0, uC, -bk);
    }
    double pm = at(u, Nx, Ny, i - 1, j - 1) + at(u, Nx, Ny, i + 1, j - 1);
    double pp = at(u, Nx, Ny, i - 1, j + 1) + at(u, Nx, Ny, i + 1, j + 1);
    if (st == 9) {
        /* Eq. 1: (1/6)[4 * edges + 1 * corners - 20 * centre]. */
        double a = p0 + v1;
        double d = pm + pp;
        return fma(4.0 / 6.0, a, fma(1.0 / 6.0, d, fma(-20.0 / 6.0, uC, -bk)));
    }
    /* Eq. 2: (1/72)[64 * axis1 - 4 * axis2 + 16 * diag1 - 1 * diag2 - 300 * centre]. */
    double v2 = at(u, Nx, Ny, i, j - 2) + at(u, Nx, Ny, i, j + 2);
    double P0 = at(u, Nx, Ny, i - 2, j) + at(u, Nx, Ny, i + 2, j);
    double Pm = at(u, Nx, Ny, i - 2, j - 2) + at(u, Nx, Ny, i + 2, j - 2);
    double Pp = at(u, Nx, Ny, i - 2, j + 2) + at(u, Nx, Ny, i + 2, j + 2);
    double a1 = p0 + v1;
    double a2 = P0 + v2;
    double d1 = pm + pp;
    double d2 = Pm + Pp;
    return fma(64.0 / 72.0, a1,
               fma(-4.0 / 72.0, a2,
                   fma(16.0 / 72.0, d1, fma(-1.0 / 72.0, d2, fma(-300.0 / 72.0, uC, -bk)))));
}

/* Lu = L u over the whole interior (the residual form with b = 0). */
void orc_apply_L(int st, int Nx, int Ny, const double *u, double *Lu) {
    for (int j = 1; j <= Ny; ++j)
        for (int i = 1; i <= Nx; ++i)
            Lu[(size_t)(j - 1) * Nx + (i - 1)] = resid_at(st, u, Nx, Ny, i, j, 0.0);
}

/* ---------------------------------------------------------------- plan */

static double s2(double x) { double s = sin(x); return s * s; }

/* Eigenvalue bounds of D^-1 A (Sec. 2.1).  Nint_x, Nint_y are the paper's N
 * (number of intervals under reading R4; the paper-literal variant passes Nx). */
void orc_kappa_bounds_n(int st, double Nint_x, double Nint_y, double *kmin, double *kmax) {
    double tx = ORC_PI / (2.0 * Nint_x), ty = ORC_PI / (2.0 * Nint_y);
    if (st == 5) {
        /* reading R5, by the same Fourier analysis the paper applies to Eq. 1 and Eq. 2 */
        *kmin = s2(tx) + s2(ty);
        *kmax = 2.0;
    } else if (st == 9) {
        *kmin = (4.0 / 5.0) * (s2(tx) + s2(ty)) + (1.0 / 5.0) * (s2(tx + ty) + s2(tx - ty));
        *kmax = 8.0 / 5.0;
    } else {
        double Tx = ORC_PI / Nint_x, Ty = ORC_PI / Nint_y;
        *kmin = -(4.0 / 75.0) * (s2(Tx) + s2(Ty)) + (64.0 / 75.0) * (s2(tx) + s2(ty)) -
                (1.0 / 75.0) * (s2(Tx + Ty) + s2(Tx - Ty)) +
                (16.0 / 75.0) * (s2(tx + ty) + s2(tx - ty));
        *kmax = 128.0 / 75.0;
    }
}

void orc_kappa_bounds(int st, int Nx, int Ny, double *kmin, double *kmax) {
    orc_kappa_bounds_n(st, (double)(Nx + 1), (double)(Ny + 1), kmin, kmax);
}

/* Smallest M0 with 1/T_M0(sigma) <= tol (reading R2, before rounding). */
long orc_cycle_length_min(double kmin, double kmax, double tol) {
    double delta = 2.0 * kmin / (kmax - kmin);               /* sigma - 1 */
    double acosh_sigma = log1p(delta + sqrt(delta * (2.0 + delta)));
    double need = log(1.0 / tol + sqrt(1.0 / (tol * tol) - 1.0)); /* acosh(1/tol) */
    double m = ceil(need / acosh_sigma);
    return m < 1.0 ? 1 : (long)m;
}

/* M = smallest power of two >= M0 (reading R2). */
long orc_cycle_length(double kmin, double kmax, double tol) {
    long m0 = orc_cycle_length_min(kmin, kmax, tol), m = 1;
    while (m < m0) m *= 2;
    return m;
}

/* Application order of the Chebyshev zeros for M = 2^p (reading R3): idx[n] in 1..M is
 * the zero used at sweep n of a cycle.  Returns 0, or -1 if M is not a power of two. */
int orc_order(long M, long *idx) {
    if (M < 1 || (M & (M - 1)) != 0) return -1;
    long *tmp = (long *)malloc(sizeof(long) * (size_t)M);
    idx[0] = 1;
    for (long m = 1; m < M; m *= 2) {
        for (long k = 0; k < m; ++k) {
            tmp[2 * k] = idx[k];
            tmp[2 * k + 1] = 2 * m + 1 - idx[k];
        }
        memcpy(idx, tmp, sizeof(long) * (size_t)(2 * m));
    }
    free(tmp);
    return 0;
}

/* Chebyshev-Jacobi weights omega_j for j = 1..M in natural order (reading R1). */
void orc_weights_natural(double kmin, double kmax, long M, double *omega) {
    double hs = 0.5 * (kmax + kmin), hd = 0.5 * (kmax - kmin);
    for (long j = 1; j <= M; ++j) {
        double x = cos((double)(2 * j - 1) * ORC_PI / (double)(2 * M));
        double lam = hs + hd * x;
        omega[j - 1] = 1.0 / lam;
    }
}

/* Per-sweep coefficients w_n = omega_{idx[n]} / c in application order; the sweep
 * is u <- u + w_n (L u - b).  Returns -1 if M is not a power of two. */
int orc_sweep_coeffs(int st, double kmin, double kmax, long M, double *w) {
    long *idx = (long *)malloc(sizeof(long) * (size_t)M);
    if (orc_order(M, idx) != 0) { free(idx); return -1; }
    double c = orc_centre(st);
    double hs = 0.5 * (kmax + kmin), hd = 0.5 * (kmax - kmin);
    for (long n = 0; n < M; ++n) {
        long j = idx[n];
        double x = cos((double)(2 * j - 1) * ORC_PI / (double)(2 * M));
        double lam = hs + hd * x;
        w[n] = 1.0 / (c * lam);
    }
    free(idx);
    return 0;
}

/* ---------------------------------------------------------------- iteration */

/* One weighted Jacobi sweep: u_out = u + w (L u - b)  (Sec. 2.1, with D = -c). */
void orc_sweep(int st, int Nx, int Ny, const double *u, const double *b, double w,
               double *u_out) {
    for (int j = 1; j <= Ny; ++j)
        for (int i = 1; i <= Nx; ++i) {
            size_t k = (size_t)(j - 1) * Nx + (i - 1);
            double r = resid_at(st, u, Nx, Ny, i, j, b[k]);
            u_out[k] = fma(w, r, u[k]);
        }
}

/* Sum of squares and max-abs of the residual L u - b over the interior. */
void orc_residual(int st, int Nx, int Ny, const double *u, const double *b, double *l2sq,
                  double *linf) {
    double s = 0.0, m = 0.0;
    for (int j = 1; j <= Ny; ++j)
        for (int i = 1; i <= Nx; ++i) {
            size_t k = (size_t)(j - 1) * Nx + (i - 1);
            double r = resid_at(st, u, Nx, Ny, i, j, b[k]);
            s += r * r;
            if (fabs(r) > m) m = fabs(r);
        }
    *l2sq = s;
    *linf = m;
}

/* b = h^2 f with h = 1/(Nx+1) (uniform mesh, Sec. 2.1). */
void orc_scale_rhs(int Nx, int Ny, const double *f, double *b) {
    double h = 1.0 / (double)(Nx + 1);
    double h2 = h * h;
    for (size_t k = 0; k < (size_t)Nx * (size_t)Ny; ++k) b[k] = h2 * f[k];
}

/* Sum of |coefficients| of L (S in reading R8). */
double orc_abs_coeff_sum(int st) {
    if (st == 5) return 8.0;
    if (st == 9) return 40.0 / 6.0;
    return 640.0 / 72.0;
}

/* Stop statuses of the solves (reading R8).  "floor" means the residual reached the FP64
 * rounding floor of the solution array (rho <= 4 fl); "stalled" means it stopped falling while
 * still above that floor (a cycle's own rounding, amplified by its partial products, or a goal
 * the iteration cannot reach), so the two are told apart. */
enum { ORC_CONVERGED = 0, ORC_FLOOR = 1, ORC_MAX_SWEEPS = 2, ORC_DIVERGED = 3, ORC_STALLED = 4 };

/* Decide after a residual evaluation whether to stop; returns -1 to continue.  *stall
 * counts consecutive cycles that failed to halve rho. */
static int stop_rule(double rho, double floor_est, double rho_prev, long done_cycles, double tol,
                     int patience, int *stall) {
    if (rho <= tol) return ORC_CONVERGED;
    if (!(rho == rho) || rho > 1e300) return ORC_DIVERGED;
    if (rho <= 4.0 * floor_est) return ORC_FLOOR;
    if (done_cycles > 0) {
        *stall = rho > 0.5 * rho_prev ? *stall + 1 : 0;
        if (*stall >= patience) return ORC_STALLED;
    }
    return -1;
}

/* Full CJM solve (Sec. 2.1 with readings R1-R8).  u holds the initial guess on entry
 * and the result on exit.  The residual is tested before every cycle; a cycle is M
 * sweeps with the weights in the order of R3.  Returns the number of sweeps done, or
 * -1 on a bad argument.  *cycles, *rel_l2, *rel_linf describe the returned u; *status
 * is one of ORC_CONVERGED, ORC_FLOOR, ORC_MAX_SWEEPS, ORC_DIVERGED, ORC_STALLED. */
long orc_solve(int st, int Nx, int Ny, const double *f, double tol, long max_sweeps,
               double *u, double *rel_l2, double *rel_linf, long *cycles, int *status) {
    if (Nx < 1 || Ny < 1 || !(tol > 0.0 && tol < 1.0)) return -1;
    size_t n = (size_t)Nx * (size_t)Ny;
    double kmin, kmax;
    orc_kappa_bounds(st, Nx, Ny, &kmin, &kmax);
    long M = orc_cycle_length(kmin, kmax, tol);
    double *w = (double *)malloc(sizeof(double) * (size_t)M);
    double *b = (double *)malloc(sizeof(double) * n);
    double *v = (double *)malloc(sizeof(double) * n);
    orc_sweep_coeffs(st, kmin, kmax, M, w);
    orc_scale_rhs(Nx, Ny, f, b);
    double bsq = 0.0, bmax = 0.0;
    for (size_t k = 0; k < n; ++k) {
        bsq += b[k] * b[k];
        if (fabs(b[k]) > bmax) bmax = fabs(b[k]);
    }
    double bn = sqrt(bsq), eps = ldexp(1.0, -53), S = orc_abs_coeff_sum(st);
    long sweeps = 0, cyc = 0;
    int stat, stall = 0;
    double rl2 = 0.0, rinf = 0.0, prev = 0.0;
    for (;;) {
        double sq, mx, usq = 0.0;
        orc_residual(st, Nx, Ny, u, b, &sq, &mx);
        for (size_t k = 0; k < n; ++k) usq += u[k] * u[k];
        rl2 = bn > 0.0 ? sqrt(sq) / bn : sqrt(sq);
        rinf = bmax > 0.0 ? mx / bmax : mx;
        double fl = bn > 0.0 ? eps * S * sqrt(usq) / bn : eps * S * sqrt(usq);
        stat = stop_rule(rl2, fl, prev, cyc, tol, 1, &stall);
        if (stat >= 0) break;
        if (sweeps + M > max_sweeps) { stat = ORC_MAX_SWEEPS; break; }
        for (long s = 0; s < M; ++s) {
            orc_sweep(st, Nx, Ny, u, b, w[s], v);
            memcpy(u, v, sizeof(double) * n);
        }
        sweeps += M;
        cyc += 1;
        prev = rl2;
    }
    free(w); free(b); free(v);
    *rel_l2 = rl2;
    *rel_linf = rinf;
    *cycles = cyc;
    *status = stat;
    return sweeps;
}

/* ---------------------------------------------------------------- FP32 inner form */

static float at32(const float *u, int Nx, int Ny, int i, int j) {
    float s = 1.0f;
    if (i == 0 || i == Nx + 1 || j == 0 || j == Ny + 1) return 0.0f;
    if (i == -1) { i = 1; s = -s; } else if (i == Nx + 2) { i = Nx; s = -s; }
    if (j == -1) { j = 1; s = -s; } else if (j == Ny + 2) { j = Ny; s = -s; }
    return s * u[(size_t)(j - 1) * Nx + (i - 1)];
}

/* r = (L e)(i, j) - rk in FP32, in second-difference form (reading R14).  Every value enters
 * through differences of neighbours, which are exact in FP32 whenever the two are within a
 * factor 2 of each other (Sterbenz), as they are for the smooth low modes the solver is
 * slowest on.  With the horizontal and vertical second differences at spacing s,
 *   X_s(dy) = (e(i+s, j+dy) - e(i, j+dy)) - (e(i, j+dy) - e(i-s, j+dy)),
 *   Y_s     = (e(i, j+s) - e(i, j)) - (e(i, j) - e(i, j-s)),
 * the paper's stencils are, exactly:
 *   5-point (Table 3):          h^2 L = X_1(0) + Y_1;
 *   9-point (Eq. 1, alpha 2/3): 6 h^2 L = X_1(-1) + X_1(1) + 4 X_1(0) + 6 Y_1 =: S_1
 *     (the stencil [1 4 1; 4 -20 4; 1 4 1] is the product of [1 4 1] across x and y, less
 *     36 at the centre);
 *   17-point (Eq. 2):          72 h^2 L = 16 S_1 - S_2, S_2 the 9-point form at spacing 2
 *     (X_2(-2) + X_2(2) + 4 X_2(0) + 6 Y_2).
 * Coefficients are the FP32 quotients (e.g. 2.0f/3.0f).  The second differences are formed
 * once per row and node and shared by the rows that use them in the GPU kernels; here they
 * are recomputed per node. */
static float resid_at32(int st, const float *u, int Nx, int Ny, int i, int j, float rk) {
    float uC = at32(u, Nx, Ny, i, j);
#define E32(di, dj) at32(u, Nx, Ny, i + (di), j + (dj))
#define X32(s, dy) ((E32(s, dy) - E32(0, dy)) - (E32(0, dy) - E32(-(s), dy)))
    float Y1 = (E32(0, 1) - uC) - (uC - E32(0, -1));
    float X1c = X32(1, 0);
    if (st == 5) return (X1c + Y1) - rk;
    float X1s = X32(1, -1) + X32(1, 1);
    if (st == 9) return fmaf(1.0f / 6.0f, X1s, fmaf(2.0f / 3.0f, X1c, Y1 - rk));
    float Y2 = (E32(0, 2) - uC) - (uC - E32(0, -2));
    float X2c = X32(2, 0);
    float X2s = X32(2, -2) + X32(2, 2);
#undef X32
#undef E32
    return fmaf(2.0f / 9.0f, X1s,
                fmaf(8.0f / 9.0f, X1c,
                     fmaf(4.0f / 3.0f, Y1,
                          fmaf(-1.0f / 72.0f, X2s, fmaf(-1.0f / 18.0f, X2c, fmaf(-1.0f / 12.0f, Y2, -rk))))));
}

/* One FP32 weighted sweep e_out = e + w (L e - r). */
void orc_sweep_f32(int st, int Nx, int Ny, const float *e, const float *r, float w,
                   float *e_out) {
    for (int j = 1; j <= Ny; ++j)
        for (int i = 1; i <= Nx; ++i) {
            size_t k = (size_t)(j - 1) * Nx + (i - 1);
            float d = resid_at32(st, e, Nx, Ny, i, j, r[k]);
            e_out[k] = fmaf(w, d, e[k]);
        }
}

/* Dirichlet-data node access and residual (reading R15, defined with orc_solve_bc below). */
static double at_bc(const double *u, const double *G, int Nx, int Ny, int i, int j);
static double resid_at_bc(int st, const double *u, const double *G, int Nx, int Ny, int i, int j,
                          double bk);

/* FP64 defect r = b - L u, its square sum and max-abs, and the FP32 copy rt. */
static void defect_g(int st, int Nx, int Ny, const double *u, const double *G, const double *b,
                     float *rt, double *l2sq, double *linf) {
    double s = 0.0, m = 0.0;
    for (int j = 1; j <= Ny; ++j)
        for (int i = 1; i <= Nx; ++i) {
            size_t k = (size_t)(j - 1) * Nx + (i - 1);
            double r = G ? resid_at_bc(st, u, G, Nx, Ny, i, j, b[k]) : resid_at(st, u, Nx, Ny, i, j, b[k]);
            rt[k] = (float)(-r);
            s += r * r;
            if (fabs(r) > m) m = fabs(r);
        }
    *l2sq = s;
    *linf = m;
}

void orc_defect(int st, int Nx, int Ny, const double *u, const double *b, float *rt,
                double *l2sq, double *linf) {
    defect_g(st, Nx, Ny, u, NULL, b, rt, l2sq, linf);
}

/* Mixed-precision CJM (reading R10).  M_in is the inner cycle length (a power of two).
 * u: initial guess in, result out.  Returns the number of FP32 sweeps, or -1 on a bad
 * argument; *outer counts the defect-correction steps; *status as for orc_solve, with
 * an outer step in the role of a cycle. */
/* Real-error stop of a defect-correction solve (R16 with R10/R11): u_hi - u_exact tested at
 * every outer step, after the defect; NULL = the residual stop of R8. */
typedef struct {
    const double *ue;
    double goal;
    double *hist;
    long cap, count;
    double err;
} err_stop;

double orc_real_error(int Nx, int Ny, const double *u, const double *u_exact);

/* The mixed loops' stop test at an outer step: with es, the real error first (recorded in
 * es->hist as (sweeps, E)), then the floor part of R8; else R8 with tol. */
static int mixed_stop(err_stop *es, int Nx, int Ny, const double *u, long sweeps, double rl2, double fl,
                      double prev, long out, double tol, int *stall) {
    if (!es) return stop_rule(rl2, fl, prev, out, tol, 2, stall);
    double E = orc_real_error(Nx, Ny, u, es->ue);
    if (es->count < es->cap) {
        es->hist[2 * es->count] = (double)sweeps;
        es->hist[2 * es->count + 1] = E;
    }
    es->count += 1;
    es->err = E;
    if (!(E == E) || E > 1e300) return ORC_DIVERGED;
    if (E <= es->goal) return ORC_CONVERGED;
    int st = stop_rule(rl2, fl, prev, out, 0.0, 2, stall);
    return st == ORC_CONVERGED ? ORC_FLOOR : st;
}

static long solve_mixed_g(int st, int Nx, int Ny, const double *f, const double *G, double tol,
                          long M_in, long max_outer, double *u, double *rel_l2, double *rel_linf,
                          long *outer, int *status, err_stop *es) {
    if (Nx < 1 || Ny < 1 || !(tol > 0.0 && tol < 1.0) || M_in < 1) return -1;
    size_t n = (size_t)Nx * (size_t)Ny;
    double kmin, kmax;
    orc_kappa_bounds(st, Nx, Ny, &kmin, &kmax);
    double *w = (double *)malloc(sizeof(double) * (size_t)M_in);
    if (orc_sweep_coeffs(st, kmin, kmax, M_in, w) != 0) { free(w); return -1; }
    float *w32 = (float *)malloc(sizeof(float) * (size_t)M_in);
    for (long s = 0; s < M_in; ++s) w32[s] = (float)w[s];
    double *b = (double *)malloc(sizeof(double) * n);
    float *rt = (float *)malloc(sizeof(float) * n);
    float *e = (float *)malloc(sizeof(float) * n);
    float *e2 = (float *)malloc(sizeof(float) * n);
    orc_scale_rhs(Nx, Ny, f, b);
    double bsq = 0.0, bmax = 0.0;
    for (size_t k = 0; k < n; ++k) {
        bsq += b[k] * b[k];
        if (fabs(b[k]) > bmax) bmax = fabs(b[k]);
    }
    double bn = sqrt(bsq), eps = ldexp(1.0, -53), S = orc_abs_coeff_sum(st);
    long sweeps = 0, out = 0;
    int stat, stall = 0;
    double rl2 = 0.0, rinf = 0.0, prev = 0.0;
    for (;;) {
        double sq, mx, usq = 0.0;
        defect_g(st, Nx, Ny, u, G, b, rt, &sq, &mx);
        for (size_t k = 0; k < n; ++k) usq += u[k] * u[k];
        rl2 = bn > 0.0 ? sqrt(sq) / bn : sqrt(sq);
        rinf = bmax > 0.0 ? mx / bmax : mx;
        double fl = bn > 0.0 ? eps * S * sqrt(usq) / bn : eps * S * sqrt(usq);
        stat = mixed_stop(es, Nx, Ny, u, sweeps, rl2, fl, prev, out, tol, &stall);
        if (stat >= 0) break;
        if (out >= max_outer) { stat = ORC_MAX_SWEEPS; break; }
        prev = rl2;
        memset(e, 0, sizeof(float) * n);
        for (long s = 0; s < M_in; ++s) {
            orc_sweep_f32(st, Nx, Ny, e, rt, w32[s], e2);
            memcpy(e, e2, sizeof(float) * n);
        }
        for (size_t k = 0; k < n; ++k) u[k] = u[k] + (double)e[k];
        sweeps += M_in;
        out += 1;
    }
    free(w); free(w32); free(b); free(rt); free(e); free(e2);
    *rel_l2 = rl2;
    *rel_linf = rinf;
    *outer = out;
    *status = stat;
    return sweeps;
}

long orc_solve_mixed(int st, int Nx, int Ny, const double *f, double tol, long M_in,
                     long max_outer, double *u, double *rel_l2, double *rel_linf,
                     long *outer, int *status) {
    return solve_mixed_g(st, Nx, Ny, f, NULL, tol, M_in, max_outer, u, rel_l2, rel_linf, outer, status, NULL);
}

/* Mixed precision with Dirichlet data G (R15 with R10): the FP64 defect takes the data ring,
 * the FP32 inner cycle solves the homogeneous error equation (R6 boundary), and the correction
 * changes the interior only. */
long orc_solve_mixed_bc(int st, int Nx, int Ny, const double *f, const double *G, double tol,
                        long M_in, long max_outer, double *u, double *rel_l2, double *rel_linf,
                        long *outer, int *status) {
    return solve_mixed_g(st, Nx, Ny, f, G, tol, M_in, max_outer, u, rel_l2, rel_linf, outer, status, NULL);
}

/* ---------------------------------------------------------------- double-FP64 outer form */

/* TwoSum (Knuth): s + e = a + b exactly. */
static void two_sum(double a, double b, double *s, double *e) {
    double x = a + b;
    double z = x - a;
    *e = (a - (x - z)) + (b - z);
    *s = x;
}

/* Sum2 accumulation of one term into (S, E). */
static void acc(double t, double *S, double *E) {
    double e;
    two_sum(*S, t, S, &e);
    *E += e;
}

/* R = (L (uh + ul))(i, j) - bk to about twice FP64 precision (reading R11), returned
 * rounded to FP64.  The terms of D (L uh - bk) are added in this fixed order:
 *   5-pt (D = 1) : uW, uE, uS, uN, -4 uC, -bk
 *   9-pt (D = 6) : 4uW, 4uE, 4uS, 4uN, uSW, uSE, uNW, uNE, -16uC, -4uC, -4bk, -2bk
 *   17-pt (D = 72): 64 x (uW, uE, uS, uN), -4 x (uWW, uEE, uSS, uNN),
 *                   16 x (uSW, uSE, uNW, uNE), -(uSSWW, uSSEE, uNNWW, uNNEE),
 *                   -256uC, -32uC, -8uC, -4uC, -64bk, -8bk
 * then R = (S + (E + D * (L ul))) / D with L ul from resid_at. */
/* u_hi at node (i, j): the data ring G when given, else the homogeneous boundary of R6. */
static double nd(const double *uh, const double *G, int Nx, int Ny, int i, int j) {
    return G ? at_bc(uh, G, Nx, Ny, i, j) : at(uh, Nx, Ny, i, j);
}

static double resid_dd_at(int st, const double *uh, const double *ul, const double *G,
                          const double *G0, int Nx, int Ny, int i, int j, double bk) {
    double S = 0.0, E = 0.0, D;
    double uC = nd(uh, G, Nx, Ny, i, j);
    if (st == 5) {
        D = 1.0;
        acc(nd(uh, G, Nx, Ny, i - 1, j), &S, &E);
        acc(nd(uh, G, Nx, Ny, i + 1, j), &S, &E);
        acc(nd(uh, G, Nx, Ny, i, j - 1), &S, &E);
        acc(nd(uh, G, Nx, Ny, i, j + 1), &S, &E);
        acc(-4.0 * uC, &S, &E);
        acc(-bk, &S, &E);
    } else if (st == 9) {
        D = 6.0;
        acc(4.0 * nd(uh, G, Nx, Ny, i - 1, j), &S, &E);
        acc(4.0 * nd(uh, G, Nx, Ny, i + 1, j), &S, &E);
        acc(4.0 * nd(uh, G, Nx, Ny, i, j - 1), &S, &E);
        acc(4.0 * nd(uh, G, Nx, Ny, i, j + 1), &S, &E);
        acc(nd(uh, G, Nx, Ny, i - 1, j - 1), &S, &E);
        acc(nd(uh, G, Nx, Ny, i + 1, j - 1), &S, &E);
        acc(nd(uh, G, Nx, Ny, i - 1, j + 1), &S, &E);
        acc(nd(uh, G, Nx, Ny, i + 1, j + 1), &S, &E);
        acc(-16.0 * uC, &S, &E);
        acc(-4.0 * uC, &S, &E);
        acc(-4.0 * bk, &S, &E);
        acc(-2.0 * bk, &S, &E);
    } else {
        D = 72.0;
        acc(64.0 * nd(uh, G, Nx, Ny, i - 1, j), &S, &E);
        acc(64.0 * nd(uh, G, Nx, Ny, i + 1, j), &S, &E);
        acc(64.0 * nd(uh, G, Nx, Ny, i, j - 1), &S, &E);
        acc(64.0 * nd(uh, G, Nx, Ny, i, j + 1), &S, &E);
        acc(-4.0 * nd(uh, G, Nx, Ny, i - 2, j), &S, &E);
        acc(-4.0 * nd(uh, G, Nx, Ny, i + 2, j), &S, &E);
        acc(-4.0 * nd(uh, G, Nx, Ny, i, j - 2), &S, &E);
        acc(-4.0 * nd(uh, G, Nx, Ny, i, j + 2), &S, &E);
        acc(16.0 * nd(uh, G, Nx, Ny, i - 1, j - 1), &S, &E);
        acc(16.0 * nd(uh, G, Nx, Ny, i + 1, j - 1), &S, &E);
        acc(16.0 * nd(uh, G, Nx, Ny, i - 1, j + 1), &S, &E);
        acc(16.0 * nd(uh, G, Nx, Ny, i + 1, j + 1), &S, &E);
        acc(-nd(uh, G, Nx, Ny, i - 2, j - 2), &S, &E);
        acc(-nd(uh, G, Nx, Ny, i + 2, j - 2), &S, &E);
        acc(-nd(uh, G, Nx, Ny, i - 2, j + 2), &S, &E);
        acc(-nd(uh, G, Nx, Ny, i + 2, j + 2), &S, &E);
        acc(-256.0 * uC, &S, &E);
        acc(-32.0 * uC, &S, &E);
        acc(-8.0 * uC, &S, &E);
        acc(-4.0 * uC, &S, &E);
        acc(-64.0 * bk, &S, &E);
        acc(-8.0 * bk, &S, &E);
    }
    /* u_lo has zero data: the zero ring G0 with data, else the R6 boundary */
    double Llo = G ? resid_at_bc(st, ul, G0, Nx, Ny, i, j, 0.0) : resid_at(st, ul, Nx, Ny, i, j, 0.0);
    return (S + (E + D * Llo)) / D;
}

/* Residual R = L (uh + ul) - b of the double-FP64 form at every node (reading R11). */
static void residual_dd_g(int st, int Nx, int Ny, const double *uh, const double *ul, const double *G,
                          const double *G0, const double *b, double *R) {
    for (int j = 1; j <= Ny; ++j)
        for (int i = 1; i <= Nx; ++i) {
            size_t k = (size_t)(j - 1) * Nx + (i - 1);
            R[k] = resid_dd_at(st, uh, ul, G, G0, Nx, Ny, i, j, b[k]);
        }
}

void orc_residual_dd(int st, int Nx, int Ny, const double *uh, const double *ul,
                     const double *b, double *R) {
    residual_dd_g(st, Nx, Ny, uh, ul, NULL, NULL, b, R);
}

/* Mixed-precision CJM with the double-FP64 outer loop (reading R11).  u: initial guess in
 * (taken as u_hi, u_lo = 0), u_hi + u_lo rounded to FP64 out; u_lo_out (may be NULL)
 * receives u_lo.  Returns the inner sweeps done or -1; *outer, *status as orc_solve_mixed;
 * the floor estimate uses 2^-106 in place of 2^-53.
 * inner64 = 0: the inner cycle runs in FP32 (R10's cycle on rt = (float)(-R)).
 * inner64 = 1 (reading R20): the inner cycle runs in FP64 -- orc_sweep, the plain FP64 sweep
 * of R9 with the homogeneous boundary of R6, on L e = r with r = -R kept in FP64 and the FP64
 * weights of a cycle of length M_in -- so every operation of the solve is FP64 or the
 * error-free double-FP64 defect and correction: the FP64-arithmetic path to a residual below
 * the FP64 floor of one solution array. */
static long solve_mixed_dd_g(int st, int Nx, int Ny, const double *f, const double *G, double tol,
                             long M_in, long max_outer, double *u, double *u_lo_out, double *rel_l2,
                             double *rel_linf, long *outer, int *status, err_stop *es, int inner64) {
    if (Nx < 1 || Ny < 1 || !(tol > 0.0 && tol < 1.0) || M_in < 1) return -1;
    size_t n = (size_t)Nx * (size_t)Ny;
    double *G0 = G ? (double *)calloc((size_t)(Nx + 4) * (size_t)(Ny + 4), sizeof(double)) : NULL;
    double kmin, kmax;
    orc_kappa_bounds(st, Nx, Ny, &kmin, &kmax);
    double *w = (double *)malloc(sizeof(double) * (size_t)M_in);
    if (orc_sweep_coeffs(st, kmin, kmax, M_in, w) != 0) { free(w); free(G0); return -1; }
    float *w32 = (float *)malloc(sizeof(float) * (size_t)M_in);
    for (long s = 0; s < M_in; ++s) w32[s] = (float)w[s];
    double *b = (double *)malloc(sizeof(double) * n);
    double *ul = (double *)calloc(n, sizeof(double));
    double *R = (double *)malloc(sizeof(double) * n);
    float *rt = (float *)malloc(sizeof(float) * n);
    float *e = (float *)malloc(sizeof(float) * n);
    float *e2 = (float *)malloc(sizeof(float) * n);
    double *r64 = inner64 ? (double *)malloc(sizeof(double) * n) : NULL;
    double *e64 = inner64 ? (double *)malloc(sizeof(double) * n) : NULL;
    double *e64b = inner64 ? (double *)malloc(sizeof(double) * n) : NULL;
    orc_scale_rhs(Nx, Ny, f, b);
    double bsq = 0.0, bmax = 0.0;
    for (size_t k = 0; k < n; ++k) {
        bsq += b[k] * b[k];
        if (fabs(b[k]) > bmax) bmax = fabs(b[k]);
    }
    double bn = sqrt(bsq), eps2 = ldexp(1.0, -106), S = orc_abs_coeff_sum(st);
    long sweeps = 0, out = 0;
    int stat, stall = 0;
    double rl2 = 0.0, rinf = 0.0, prev = 0.0;
    for (;;) {
        double sq = 0.0, mx = 0.0, usq = 0.0;
        residual_dd_g(st, Nx, Ny, u, ul, G, G0, b, R);
        for (size_t k = 0; k < n; ++k) {
            sq += R[k] * R[k];
            if (fabs(R[k]) > mx) mx = fabs(R[k]);
            usq += u[k] * u[k];
            rt[k] = (float)(-R[k]);
            if (inner64) r64[k] = -R[k];
        }
        rl2 = bn > 0.0 ? sqrt(sq) / bn : sqrt(sq);
        rinf = bmax > 0.0 ? mx / bmax : mx;
        double fl = bn > 0.0 ? eps2 * S * sqrt(usq) / bn : eps2 * S * sqrt(usq);
        stat = mixed_stop(es, Nx, Ny, u, sweeps, rl2, fl, prev, out, tol, &stall);
        if (stat >= 0) break;
        if (out >= max_outer) { stat = ORC_MAX_SWEEPS; break; }
        prev = rl2;
        if (inner64) {
            memset(e64, 0, sizeof(double) * n);
            for (long s = 0; s < M_in; ++s) {
                orc_sweep(st, Nx, Ny, e64, r64, w[s], e64b);
                memcpy(e64, e64b, sizeof(double) * n);
            }
        } else {
            memset(e, 0, sizeof(float) * n);
            for (long s = 0; s < M_in; ++s) {
                orc_sweep_f32(st, Nx, Ny, e, rt, w32[s], e2);
                memcpy(e, e2, sizeof(float) * n);
            }
        }
        for (size_t k = 0; k < n; ++k) {
            double hi, err;
            two_sum(u[k], inner64 ? e64[k] : (double)e[k], &hi, &err);
            double lo = ul[k] + err;
            two_sum(hi, lo, &u[k], &ul[k]);
        }
        sweeps += M_in;
        out += 1;
    }
    if (u_lo_out) memcpy(u_lo_out, ul, sizeof(double) * n);
    free(w); free(w32); free(b); free(ul); free(R); free(rt); free(e); free(e2); free(G0);
    free(r64); free(e64); free(e64b);
    *rel_l2 = rl2;
    *rel_linf = rinf;
    *outer = out;
    *status = stat;
    return sweeps;
}

long orc_solve_mixed_dd(int st, int Nx, int Ny, const double *f, double tol, long M_in,
                        long max_outer, double *u, double *u_lo_out, double *rel_l2,
                        double *rel_linf, long *outer, int *status) {
    return solve_mixed_dd_g(st, Nx, Ny, f, NULL, tol, M_in, max_outer, u, u_lo_out, rel_l2, rel_linf,
                            outer, status, NULL, 0);
}

/* FP64 inner cycles in the double-FP64 outer loop (reading R20); G: Dirichlet data (R15) or
 * NULL (R6).  Arguments and results as orc_solve_mixed_dd; the count returned is FP64 sweeps. */
long orc_solve_fp64_dd(int st, int Nx, int Ny, const double *f, const double *G, double tol, long M_in,
                       long max_outer, double *u, double *u_lo_out, double *rel_l2, double *rel_linf,
                       long *outer, int *status) {
    return solve_mixed_dd_g(st, Nx, Ny, f, G, tol, M_in, max_outer, u, u_lo_out, rel_l2, rel_linf,
                            outer, status, NULL, 1);
}

/* The double-FP64 form with Dirichlet data G (R15 with R11): u_hi's ghosts are the data, u_lo's
 * are zero; the inner cycle and correction as in orc_solve_mixed_bc. */
long orc_solve_mixed_dd_bc(int st, int Nx, int Ny, const double *f, const double *G, double tol,
                           long M_in, long max_outer, double *u, double *u_lo_out, double *rel_l2,
                           double *rel_linf, long *outer, int *status) {
    return solve_mixed_dd_g(st, Nx, Ny, f, G, tol, M_in, max_outer, u, u_lo_out, rel_l2, rel_linf,
                            outer, status, NULL, 0);
}

/* ---------------------------------------------------------------- non-homogeneous Dirichlet */

/* Reading R15 (the paper's test problem, Sec. 3.3): Dirichlet data given at every node the
 * stencil reaches outside the interior -- the ring of nodes i or j in {-1, 0, N+1, N+2} --
 * in a padded array G of (Ny+4) rows x (Nx+4) columns, node (i, j) at G[(j+1)*(Nx+4) + i+1].
 * Those values are fixed; the interior iterates as before.  The error then iterates with the
 * operator whose ghost values are all zero, whose spectrum lies inside the paper's
 * [kmin, kmax] (pinned by a dense eigenvalue test), so the plan is unchanged. */
static double at_bc(const double *u, const double *G, int Nx, int Ny, int i, int j) {
    if (i < 1 || i > Nx || j < 1 || j > Ny) return G[(size_t)(j + 1) * (Nx + 4) + (i + 1)];
    return u[(size_t)(j - 1) * Nx + (i - 1)];
}

/* resid_at with the ghost values taken from G (same evaluation order, reading R9). */
static double resid_at_bc(int st, const double *u, const double *G, int Nx, int Ny, int i, int j,
                          double bk) {
#define A(di, dj) at_bc(u, G, Nx, Ny, i + (di), j + (dj))
    double uC = A(0, 0);
    double v1 = A(0, -1) + A(0, 1);
    double p0 = A(-1, 0) + A(1, 0);
    if (st == 5) return (p0 + v1) + fma(-4.0, uC, -bk);
    double pm = A(-1, -1) + A(1, -1);
    double pp = A(-1, 1) + A(1, 1);
    if (st == 9) return fma(4.0 / 6.0, p0 + v1, fma(1.0 / 6.0, pm + pp, fma(-20.0 / 6.0, uC, -bk)));
    double v2 = A(0, -2) + A(0, 2);
    double P0 = A(-2, 0) + A(2, 0);
    double Pm = A(-2, -2) + A(2, -2);
    double Pp = A(-2, 2) + A(2, 2);
#undef A
    return fma(64.0 / 72.0, p0 + v1,
               fma(-4.0 / 72.0, P0 + v2,
                   fma(16.0 / 72.0, pm + pp, fma(-1.0 / 72.0, Pm + Pp, fma(-300.0 / 72.0, uC, -bk)))));
}

void orc_sweep_bc(int st, int Nx, int Ny, const double *u, const double *G, const double *b,
                  double w, double *u_out) {
    for (int j = 1; j <= Ny; ++j)
        for (int i = 1; i <= Nx; ++i) {
            size_t k = (size_t)(j - 1) * Nx + (i - 1);
            u_out[k] = fma(w, resid_at_bc(st, u, G, Nx, Ny, i, j, b[k]), u[k]);
        }
}

void orc_residual_bc(int st, int Nx, int Ny, const double *u, const double *G, const double *b,
                     double *l2sq, double *linf) {
    double s = 0.0, m = 0.0;
    for (int j = 1; j <= Ny; ++j)
        for (int i = 1; i <= Nx; ++i) {
            size_t k = (size_t)(j - 1) * Nx + (i - 1);
            double r = resid_at_bc(st, u, G, Nx, Ny, i, j, b[k]);
            s += r * r;
            if (fabs(r) > m) m = fabs(r);
        }
    *l2sq = s;
    *linf = m;
}

/* Plain FP64 CJM with Dirichlet data G (R15); otherwise as orc_solve. */
long orc_solve_bc(int st, int Nx, int Ny, const double *f, const double *G, double tol,
                  long max_sweeps, double *u, double *rel_l2, double *rel_linf, long *cycles,
                  int *status) {
    if (Nx < 1 || Ny < 1 || !(tol > 0.0 && tol < 1.0)) return -1;
    size_t n = (size_t)Nx * (size_t)Ny;
    double kmin, kmax;
    orc_kappa_bounds(st, Nx, Ny, &kmin, &kmax);
    long M = orc_cycle_length(kmin, kmax, tol);
    double *w = (double *)malloc(sizeof(double) * (size_t)M);
    double *b = (double *)malloc(sizeof(double) * n);
    double *v = (double *)malloc(sizeof(double) * n);
    orc_sweep_coeffs(st, kmin, kmax, M, w);
    orc_scale_rhs(Nx, Ny, f, b);
    double bsq = 0.0, bmax = 0.0;
    for (size_t k = 0; k < n; ++k) {
        bsq += b[k] * b[k];
        if (fabs(b[k]) > bmax) bmax = fabs(b[k]);
    }
    double bn = sqrt(bsq), eps = ldexp(1.0, -53), S = orc_abs_coeff_sum(st);
    long sweeps = 0, cyc = 0;
    int stat, stall = 0;
    double rl2 = 0.0, rinf = 0.0, prev = 0.0;
    for (;;) {
        double sq, mx, usq = 0.0;
        orc_residual_bc(st, Nx, Ny, u, G, b, &sq, &mx);
        for (size_t k = 0; k < n; ++k) usq += u[k] * u[k];
        rl2 = bn > 0.0 ? sqrt(sq) / bn : sqrt(sq);
        rinf = bmax > 0.0 ? mx / bmax : mx;
        double fl = bn > 0.0 ? eps * S * sqrt(usq) / bn : eps * S * sqrt(usq);
        stat = stop_rule(rl2, fl, prev, cyc, tol, 1, &stall);
        if (stat >= 0) break;
        if (sweeps + M > max_sweeps) { stat = ORC_MAX_SWEEPS; break; }
        for (long s2 = 0; s2 < M; ++s2) {
            orc_sweep_bc(st, Nx, Ny, u, G, b, w[s2], v);
            memcpy(u, v, sizeof(double) * n);
        }
        sweeps += M;
        cyc += 1;
        prev = rl2;
    }
    free(w); free(b); free(v);
    *rel_l2 = rl2;
    *rel_linf = rinf;
    *cycles = cyc;
    *status = stat;
    return sweeps;
}

/* ---------------------------------------------------------------- real-error stop */

/* Real error of Sec. 3.4 (Fig. 4, right): the infinity norm of u - u_exact over the interior. */
double orc_real_error(int Nx, int Ny, const double *u, const double *u_exact) {
    double m = 0.0;
    size_t n = (size_t)Nx * (size_t)Ny;
    for (size_t k = 0; k < n; ++k) {
        double d = fabs(u[k] - u_exact[k]);
        if (!(d == d)) return d;
        if (d > m) m = d;
    }
    return m;
}

/* Plain FP64 CJM stopped by the real error instead of the residual (Sec. 3.4, reading R16):
 * the cycle length comes from `tol` as in orc_solve; the real error E is tested before every
 * cycle and, when check_every > 0, after every check_every sweeps inside a cycle.  Stops with
 * converged at the first test where E <= err_tol.  The residual of R8 is still evaluated before
 * every cycle, only for the floor and stall parts of the stop rule (a residual at the FP64
 * floor ends the solve with "floor", a cycle that failed to halve it with "stalled": the real
 * error cannot fall further, e.g. when err_tol is below the discretisation error).  E = NaN ends it with
 * "diverged".  G = NULL: homogeneous Dirichlet (R6); else the Dirichlet data of R15.
 * hist[2k], hist[2k+1] = sweeps done and E at the k-th test (up to cap tests; *count = all). */
long orc_solve_to_error(int st, int Nx, int Ny, const double *f, const double *G,
                        const double *u_exact, double tol, double err_tol, long check_every,
                        long max_sweeps, double *u, double *hist, long cap, long *count,
                        double *err, double *rel_l2, long *cycles, int *status) {
    if (Nx < 1 || Ny < 1 || !(tol > 0.0 && tol < 1.0) || !(err_tol >= 0.0) || check_every < 0)
        return -1;
    size_t n = (size_t)Nx * (size_t)Ny;
    double kmin, kmax;
    orc_kappa_bounds(st, Nx, Ny, &kmin, &kmax);
    long M = orc_cycle_length(kmin, kmax, tol);
    double *w = (double *)malloc(sizeof(double) * (size_t)M);
    double *b = (double *)malloc(sizeof(double) * n);
    double *v = (double *)malloc(sizeof(double) * n);
    orc_sweep_coeffs(st, kmin, kmax, M, w);
    orc_scale_rhs(Nx, Ny, f, b);
    double bsq = 0.0;
    for (size_t k = 0; k < n; ++k) bsq += b[k] * b[k];
    double bn = sqrt(bsq), eps = ldexp(1.0, -53), S = orc_abs_coeff_sum(st);
    long sweeps = 0, cyc = 0, tests = 0;
    int stat = -1, stall = 0, mid = 0;
    double rl2 = 0.0, prev = 0.0, E = 0.0, sq, mx;
#define RECORD()                                          \
    do {                                                  \
        if (tests < cap) {                                \
            hist[2 * tests] = (double)sweeps;             \
            hist[2 * tests + 1] = E;                      \
        }                                                 \
        ++tests;                                          \
    } while (0)
    for (;;) {
        double usq = 0.0;
        if (G) orc_residual_bc(st, Nx, Ny, u, G, b, &sq, &mx);
        else orc_residual(st, Nx, Ny, u, b, &sq, &mx);
        for (size_t k = 0; k < n; ++k) usq += u[k] * u[k];
        rl2 = bn > 0.0 ? sqrt(sq) / bn : sqrt(sq);
        double fl = bn > 0.0 ? eps * S * sqrt(usq) / bn : eps * S * sqrt(usq);
        E = orc_real_error(Nx, Ny, u, u_exact);
        RECORD();
        if (!(E == E) || E > 1e300) { stat = ORC_DIVERGED; break; }
        if (E <= err_tol) { stat = ORC_CONVERGED; break; }
        stat = stop_rule(rl2, fl, prev, cyc, 0.0, 1, &stall);
        if (stat == ORC_CONVERGED) stat = ORC_FLOOR; /* rho == 0: u is the discrete solution */
        if (stat >= 0) break;
        if (sweeps + M > max_sweeps) { stat = ORC_MAX_SWEEPS; break; }
        for (long s = 0; s < M; ++s) {
            if (G) orc_sweep_bc(st, Nx, Ny, u, G, b, w[s], v);
            else orc_sweep(st, Nx, Ny, u, b, w[s], v);
            memcpy(u, v, sizeof(double) * n);
            ++sweeps;
            if (check_every > 0 && (s + 1) % check_every == 0 && s + 1 < M) {
                E = orc_real_error(Nx, Ny, u, u_exact);
                RECORD();
                if (!(E == E) || E > 1e300) { stat = ORC_DIVERGED; mid = 1; break; }
                if (E <= err_tol) { stat = ORC_CONVERGED; mid = 1; break; }
            }
        }
        if (mid) break;
        cyc += 1;
        prev = rl2;
    }
#undef RECORD
    if (mid) { /* report the residual where the solve stopped */
        if (G) orc_residual_bc(st, Nx, Ny, u, G, b, &sq, &mx);
        else orc_residual(st, Nx, Ny, u, b, &sq, &mx);
        rl2 = bn > 0.0 ? sqrt(sq) / bn : sqrt(sq);
    }
    free(w); free(b); free(v);
    *count = tests;
    *err = E;
    *rel_l2 = rl2;
    *cycles = cyc;
    *status = stat;
    return sweeps;
}

/* ---------------------------------------------------------------- classical Jacobi */

/* Classical Jacobi (omega = 1, the paper's comparison method, Sec. 3.4 and Table 1), reading
 * R18: every sweep uses w = 1/c; the residual of R8 is tested every M sweeps, M the CJM cycle
 * length of the same tolerance (R2); stops converged at rho <= tol, "floor" at rho <= 4 fl,
 * "stalled" when an interval of M sweeps did not lower rho (Jacobi's residual falls
 * monotonically in exact arithmetic), "diverged" on a non-finite rho.  G = NULL: homogeneous Dirichlet (R6);
 * else the Dirichlet data of R15.  *intervals = the M-sweep intervals done. */
long orc_solve_jacobi(int st, int Nx, int Ny, const double *f, const double *G, double tol,
                      long max_sweeps, double *u, double *rel_l2, double *rel_linf,
                      long *intervals, int *status) {
    if (Nx < 1 || Ny < 1 || !(tol > 0.0 && tol < 1.0)) return -1;
    size_t n = (size_t)Nx * (size_t)Ny;
    double kmin, kmax;
    orc_kappa_bounds(st, Nx, Ny, &kmin, &kmax);
    long M = orc_cycle_length(kmin, kmax, tol);
    double w = 1.0 / orc_centre(st);
    double *b = (double *)malloc(sizeof(double) * n);
    double *v = (double *)malloc(sizeof(double) * n);
    orc_scale_rhs(Nx, Ny, f, b);
    double bsq = 0.0, bmax = 0.0;
    for (size_t k = 0; k < n; ++k) {
        bsq += b[k] * b[k];
        if (fabs(b[k]) > bmax) bmax = fabs(b[k]);
    }
    double bn = sqrt(bsq), eps = ldexp(1.0, -53), S = orc_abs_coeff_sum(st);
    long sweeps = 0, done = 0;
    int stat;
    double rl2 = 0.0, rinf = 0.0, prev = 0.0;
    for (;;) {
        double sq, mx, usq = 0.0;
        if (G) orc_residual_bc(st, Nx, Ny, u, G, b, &sq, &mx);
        else orc_residual(st, Nx, Ny, u, b, &sq, &mx);
        for (size_t k = 0; k < n; ++k) usq += u[k] * u[k];
        rl2 = bn > 0.0 ? sqrt(sq) / bn : sqrt(sq);
        rinf = bmax > 0.0 ? mx / bmax : mx;
        double fl = bn > 0.0 ? eps * S * sqrt(usq) / bn : eps * S * sqrt(usq);
        if (rl2 <= tol) { stat = ORC_CONVERGED; break; }
        if (!(rl2 == rl2) || rl2 > 1e300) { stat = ORC_DIVERGED; break; }
        if (rl2 <= 4.0 * fl) { stat = ORC_FLOOR; break; }
        if (done > 0 && rl2 >= prev) { stat = ORC_STALLED; break; }
        if (sweeps + M > max_sweeps) { stat = ORC_MAX_SWEEPS; break; }
        for (long s = 0; s < M; ++s) {
            if (G) orc_sweep_bc(st, Nx, Ny, u, G, b, w, v);
            else orc_sweep(st, Nx, Ny, u, b, w, v);
            memcpy(u, v, sizeof(double) * n);
        }
        sweeps += M;
        done += 1;
        prev = rl2;
    }
    free(b); free(v);
    *rel_l2 = rl2;
    *rel_linf = rinf;
    *intervals = done;
    *status = stat;
    return sweeps;
}

/* ---------------------------------------------------------------- coefficient masks */

/* Position-dependent coefficient masks (Sec. 3.2, the masks of neighbours at distance one
 * and two, with Cartesian, polar and bipolar examples), reading R19.  The operator is
 *   (A u)(i, j) = sum over the mask's offsets (dx, dy) of c_{dx,dy}(i, j) u(i+dx, j+dy),
 * A u = f.  Patterns: 5 (the cross |dx|+|dy| = 1), 9 (the 3x3 box), 17 (the 17 points of
 * Eq. 2: the 3x3 box, (+-2, 0), (0, +-2) and (+-2, +-2)), 25 (the 5x5 box).  The off-centre
 * offsets are taken in row-major order (dy = -R..R, then dx = -R..R).  Nodes outside the
 * interior take the Dirichlet data of R15 (G) or 0.
 * Coefficients: plane 0 is the centre c_C, planes 1..K the off-centre offsets in that order;
 * value of plane k at (i, j) = coef[k*sp + (j-1)*sy + (i-1)*sx] (a stride of 0 repeats a
 * plane along that axis).  An optional factor s(i, j) = scale[(j-1)*ssy + (i-1)*ssx]
 * multiplies every coefficient.
 * The iteration runs on the Jacobi-normalised system D^-1 A u = D^-1 f, D = diag(s c_C):
 *   chat_k = c_k / c_C (s cancels), bhat = f / (s c_C),
 *   r = (u_C - bhat) + sum_k chat_k u_k   (one subtraction, then fma in offset order),
 *   u' = u_C - w_n r                      (fma(-w_n, r, u_C)),
 * w_n = omega_n = 1/lambda_n of R1 in the order of R3 for the caller's [kmin, kmax] of D^-1 A
 * (the paper gives the bounds only for its uniform Cartesian stencils), or w_n = 1 for
 * classical Jacobi.  Residual test (R8 on the normalised system): rho = ||r||_2 / ||bhat||_2;
 * floor estimate with S = 2 (a bound on 1 + sum |chat_k| for the diagonally dominant masks). */
int orc_mask_offsets(int pat, int *dx, int *dy) {
    int R = (pat == 5 || pat == 9) ? 1 : 2, K = 0;
    for (int y = -R; y <= R; ++y)
        for (int x = -R; x <= R; ++x) {
            int ax = x < 0 ? -x : x, ay = y < 0 ? -y : y, m = ax > ay ? ax : ay, in;
            if (x == 0 && y == 0) continue;
            if (pat == 5) in = ax + ay == 1;
            else if (pat == 9) in = m == 1;
            else if (pat == 17) in = m == 1 || (ax == 2 && ay == 0) || (ax == 0 && ay == 2) || (ax == 2 && ay == 2);
            else in = 1;
            if (!in) continue;
            dx[K] = x;
            dy[K] = y;
            ++K;
        }
    return K;
}

static double mask_at(const double *u, const double *G, int Nx, int Ny, int i, int j) {
    if (i < 1 || i > Nx || j < 1 || j > Ny) return G ? G[(size_t)(j + 1) * (Nx + 4) + (i + 1)] : 0.0;
    return u[(size_t)(j - 1) * Nx + (i - 1)];
}

/* chat: K planes of Nx*Ny (full layout); dC = s c_C (Nx*Ny).  Returns K, or -1 if the pattern
 * is unknown or a centre coefficient is 0. */
int orc_mask_normalize(int pat, int Nx, int Ny, const double *coef, long sx, long sy, long sp,
                       const double *scale, long ssx, long ssy, double *chat, double *dC) {
    int dx[24], dy[24];
    if (pat != 5 && pat != 9 && pat != 17 && pat != 25) return -1;
    int K = orc_mask_offsets(pat, dx, dy);
    size_t n = (size_t)Nx * (size_t)Ny;
    for (int j = 1; j <= Ny; ++j)
        for (int i = 1; i <= Nx; ++i) {
            size_t node = (size_t)(j - 1) * Nx + (i - 1);
            long at = (long)(j - 1) * sy + (long)(i - 1) * sx;
            double cC = coef[at];
            if (cC == 0.0) return -1;
            for (int k = 0; k < K; ++k) chat[(size_t)k * n + node] = coef[(long)(k + 1) * sp + at] / cC;
            dC[node] = scale ? scale[(long)(j - 1) * ssy + (long)(i - 1) * ssx] * cC : cC;
        }
    return K;
}

/* r = (D^-1 A u - bhat)(i, j) in the order above. */
static double mask_resid(int K, const int *dx, const int *dy, const double *u, const double *G,
                         int Nx, int Ny, int i, int j, const double *bhat, const double *chat) {
    size_t n = (size_t)Nx * (size_t)Ny, node = (size_t)(j - 1) * Nx + (i - 1);
    double r = u[node] - bhat[node];
    for (int k = 0; k < K; ++k)
        r = fma(chat[(size_t)k * n + node], mask_at(u, G, Nx, Ny, i + dx[k], j + dy[k]), r);
    return r;
}

void orc_sweep_mask(int pat, int Nx, int Ny, const double *u, const double *G, const double *bhat,
                    const double *chat, double w, double *u_out) {
    int dx[24], dy[24];
    int K = orc_mask_offsets(pat, dx, dy);
    for (int j = 1; j <= Ny; ++j)
        for (int i = 1; i <= Nx; ++i) {
            size_t node = (size_t)(j - 1) * Nx + (i - 1);
            u_out[node] = fma(-w, mask_resid(K, dx, dy, u, G, Nx, Ny, i, j, bhat, chat), u[node]);
        }
}

void orc_residual_mask(int pat, int Nx, int Ny, const double *u, const double *G, const double *bhat,
                       const double *chat, double *l2sq, double *linf) {
    int dx[24], dy[24];
    int K = orc_mask_offsets(pat, dx, dy);
    double s = 0.0, m = 0.0;
    for (int j = 1; j <= Ny; ++j)
        for (int i = 1; i <= Nx; ++i) {
            double r = mask_resid(K, dx, dy, u, G, Nx, Ny, i, j, bhat, chat);
            s += r * r;
            if (fabs(r) > m) m = fabs(r);
        }
    *l2sq = s;
    *linf = m;
}

/* Per-sweep weights omega_n = 1/lambda_n in the order of R3 (the normalised system's c = 1). */
int orc_mask_weights(double kmin, double kmax, long M, double *w) {
    long *idx = (long *)malloc(sizeof(long) * (size_t)M);
    if (orc_order(M, idx) != 0) { free(idx); return -1; }
    double hs = 0.5 * (kmax + kmin), hd = 0.5 * (kmax - kmin);
    for (long n = 0; n < M; ++n) {
        double x = cos((double)(2 * idx[n] - 1) * ORC_PI / (double)(2 * M));
        w[n] = 1.0 / (hs + hd * x);
    }
    free(idx);
    return 0;
}

/* CJM (method 0) or classical Jacobi (method 1, R18) on a masked operator; otherwise as
 * orc_solve / orc_solve_jacobi.  Returns the sweeps done, or -1 on a bad argument. */
long orc_solve_mask(int pat, int Nx, int Ny, const double *f, const double *coef, long sx, long sy,
                    long sp, const double *scale, long ssx, long ssy, double kmin, double kmax,
                    double tol, int method, const double *G, long max_sweeps, double *u,
                    double *rel_l2, double *rel_linf, long *cycles, int *status) {
    if (Nx < 1 || Ny < 1 || !(tol > 0.0 && tol < 1.0) || !(kmin > 0.0 && kmin < kmax)) return -1;
    size_t n = (size_t)Nx * (size_t)Ny;
    double *chat = (double *)malloc(sizeof(double) * n * 24);
    double *dC = (double *)malloc(sizeof(double) * n);
    if (orc_mask_normalize(pat, Nx, Ny, coef, sx, sy, sp, scale, ssx, ssy, chat, dC) < 0) {
        free(chat); free(dC);
        return -1;
    }
    long M = orc_cycle_length(kmin, kmax, tol);
    double *w = (double *)malloc(sizeof(double) * (size_t)M);
    if (method == 1) for (long k = 0; k < M; ++k) w[k] = 1.0;
    else orc_mask_weights(kmin, kmax, M, w);
    double *bh = (double *)malloc(sizeof(double) * n);
    double *v = (double *)malloc(sizeof(double) * n);
    double bsq = 0.0, bmax = 0.0;
    for (size_t k = 0; k < n; ++k) {
        bh[k] = f[k] / dC[k];
        bsq += bh[k] * bh[k];
        if (fabs(bh[k]) > bmax) bmax = fabs(bh[k]);
    }
    double bn = sqrt(bsq), eps = ldexp(1.0, -53), S = 2.0;
    long sweeps = 0, cyc = 0;
    int stat, stall = 0;
    double rl2 = 0.0, rinf = 0.0, prev = 0.0;
    for (;;) {
        double sq, mx, usq = 0.0;
        orc_residual_mask(pat, Nx, Ny, u, G, bh, chat, &sq, &mx);
        for (size_t k = 0; k < n; ++k) usq += u[k] * u[k];
        rl2 = bn > 0.0 ? sqrt(sq) / bn : sqrt(sq);
        rinf = bmax > 0.0 ? mx / bmax : mx;
        double fl = bn > 0.0 ? eps * S * sqrt(usq) / bn : eps * S * sqrt(usq);
        if (method == 1) {
            if (rl2 <= tol) stat = ORC_CONVERGED;
            else if (!(rl2 == rl2) || rl2 > 1e300) stat = ORC_DIVERGED;
            else if (rl2 <= 4.0 * fl) stat = ORC_FLOOR;
            else if (cyc > 0 && rl2 >= prev) stat = ORC_STALLED;
            else stat = -1;
        } else {
            stat = stop_rule(rl2, fl, prev, cyc, tol, 1, &stall);
        }
        if (stat >= 0) break;
        if (sweeps + M > max_sweeps) { stat = ORC_MAX_SWEEPS; break; }
        for (long s = 0; s < M; ++s) {
            orc_sweep_mask(pat, Nx, Ny, u, G, bh, chat, w[s], v);
            memcpy(u, v, sizeof(double) * n);
        }
        sweeps += M;
        cyc += 1;
        prev = rl2;
    }
    free(chat); free(dC); free(w); free(bh); free(v);
    *rel_l2 = rl2;
    *rel_linf = rinf;
    *cycles = cyc;
    *status = stat;
    return sweeps;
}

/* Defect correction (R10; R11 with dd = 1; R20, FP64 inner cycles, with dd = 2) stopped by the
 * real error (R16): u_hi - u_exact in the infinity norm, tested at every outer step after the
 * defect, stops the solve at <= err_goal; the residual's floor and stall parts of R8 still end it
 * ("floor" / "stalled").  G: Dirichlet data (R15) or NULL.  hist[2k], hist[2k+1] = inner sweeps
 * done and E at the k-th test (cap tests; *count = all). */
long orc_solve_mixed_to_error(int st, int Nx, int Ny, const double *f, const double *G,
                              const double *u_exact, double err_goal, long M_in, int dd, long max_outer,
                              double *u, double *u_lo_out, double *hist, long cap, long *count,
                              double *err, double *rel_l2, long *outer, int *status) {
    if (!(err_goal >= 0.0)) return -1;
    err_stop es = {u_exact, err_goal, hist, cap, 0, 0.0};
    double rinf;
    long n = dd ? solve_mixed_dd_g(st, Nx, Ny, f, G, 0.5, M_in, max_outer, u, u_lo_out, rel_l2, &rinf, outer,
                                   status, &es, dd == 2)
                : solve_mixed_g(st, Nx, Ny, f, G, 0.5, M_in, max_outer, u, rel_l2, &rinf, outer, status, &es);
    *count = es.count;
    *err = es.err;
    return n;
}
