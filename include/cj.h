/*
 * cj.h -- C ABI of the GB300 Chebyshev-Jacobi (CJM) solver library (libcj.so).
 *
 * The method (Adsuara et al., arXiv 1705.00103, Sec. 2.1): solve the finite-difference
 * Poisson problem Delta_h u = f on the interior nodes 1 <= i <= Nx, 1 <= j <= Ny of a
 * uniform mesh (h = 1/(Nx+1) in both directions, Sec. 3.2) by weighted Jacobi sweeps
 *     u <- u + w_n (L u - b),   b = h^2 f,   L = h^2 Delta_h,   w_n = omega_n / c,
 * whose weight omega_n changes at every sweep: the M weights are the zeros of the
 * degree-M Chebyshev polynomial mapped onto the eigenvalue interval [kmin, kmax] of the
 * Jacobi iteration matrix, whose ends the paper gives in closed form for each stencil
 * (equations after Eq. 1 and Eq. 2).  Stencils: the classical 5-point Laplacian (Table 3,
 * Cartesian row), the 9-point alpha = 2/3 Laplacian (Eq. 1) and the 17-point alpha = 2/3
 * Laplacian (Eq. 2).  Boundary: homogeneous Dirichlet (u = 0 on nodes 0 and N+1; the
 * 17-point stencil's second ghost layer is the odd reflection u[-1] = -u[1]), or Dirichlet
 * data on both rings (CJ_BC_DIRICHLET, the paper's test problem).  Also: classical Jacobi
 * (CJ_JACOBI), the real-error stop (cj_solve_to_error), position-dependent coefficient
 * masks (cj_plan_create_mask), batched solves and a request server.
 *
 * Conventions for every entry point:
 *   - Grids passed in or out are interior values only, row-major: node (i, j) is element
 *     (j-1)*ld + (i-1), with ld >= Nx the row stride in elements.  "device" pointers are
 *     CUDA device (or managed) memory of the current device; "host" pointers are host
 *     memory (pinned memory gives the fastest copies).
 *   - The library never frees or keeps caller memory.  Objects it creates (plans) own
 *     their device workspace until destroyed.
 *   - Streams are passed as `void *` holding a cudaStream_t (NULL = legacy default stream).
 *   - No C++ exception crosses the ABI; every failure is a cj_status < 0.
 *   - A plan is used by one host thread at a time; its workspace serialises its calls.
 */
#ifndef CJ_H
#define CJ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CJ_OK = 0,                /* solve converged: relative residual <= tol */
    CJ_FLOOR = 1,             /* solve stopped at the FP64 rounding floor: relative residual
                                 <= 4 x cj_result.floor_est */
    CJ_PENDING = 2,           /* reserved for asynchronous requests: not finished yet */
    CJ_STALLED = 3,           /* solve stopped because the residual stopped falling while still
                                 above 4 x floor_est: a cycle failed to halve it (two outer
                                 steps in a row for defect correction; an interval that did not
                                 lower it for CJ_JACOBI).  For plain FP64 cycles on large grids
                                 this is the cycle's own rounding, amplified by the partial
                                 products of its weights; a defect-correction precision reaches
                                 lower residuals */
    CJ_ERR_INVALID_ARG = -1,  /* a size, pointer, stencil, tolerance or option is invalid */
    CJ_ERR_NOMEM = -2,        /* a device or host allocation failed */
    CJ_ERR_NOT_CONVERGED = -3,/* the sweep budget ran out first */
    CJ_ERR_DIVERGED = -4,     /* the residual became non-finite */
    CJ_ERR_TIMEOUT = -5,      /* a bounded device wait gave up */
    CJ_ERR_CUDA = -6,         /* a CUDA runtime call failed (message: cj_last_error) */
    CJ_ERR_BUDGET = -7        /* reserved: a memory budget refused the request */
} cj_status;

typedef enum { CJ_ST5 = 5, CJ_ST9 = 9, CJ_ST17 = 17 } cj_stencil;

typedef enum {
    CJ_BC_DIRICHLET0 = 0,  /* homogeneous Dirichlet; 17-point: odd reflection for the 2nd ring */
    CJ_BC_DIRICHLET = 1    /* Dirichlet data given at both rings around the interior (the paper's
                              test problem, Sec. 3.3), set by cj_set_boundary; in the mixed
                              precisions the FP64 defect reads the data and the FP32 inner
                              cycles solve the homogeneous error equation */
} cj_bc;

typedef enum {
    CJ_FP64 = 0,          /* plain CJM: every sweep in FP64 */
    CJ_FP32_INNER = 1,    /* FP32 inner CJM cycles inside an FP64 defect-correction loop */
    CJ_FP32_INNER_DD = 2, /* FP32 inner CJM cycles inside a double-FP64 defect-correction
                             loop: the solution is u_hi + u_lo and the defect is evaluated
                             to about twice FP64 precision, so the relative residual can go
                             below the FP64 floor (see cj_result.floor_est) */
    CJ_FP64_INNER_DD = 3  /* FP64 inner CJM cycles inside the same double-FP64 loop: every
                             sweep is the plain FP64 sweep (on the error equation L e = r,
                             r = b - L u in FP64), so this is the all-FP64 way to tolerances
                             below one FP64 array's floor, where plain cycles stall; the
                             baseline the FP32-inner precisions are compared with */
} cj_precision;

typedef enum {
    CJ_CJM = 0,     /* Chebyshev-Jacobi: the weights of Sec. 2.1, one cycle of M sweeps between
                       residual tests */
    CJ_JACOBI = 1   /* classical Jacobi (omega = 1 at every sweep), the paper's comparison
                       method (Sec. 3.4, Table 1); the residual is tested every M sweeps, M the
                       CJM cycle length of the same tolerance; it stops (CJ_STALLED) when an
                       interval does not lower the residual.  CJ_FP64 only */
} cj_method;

/* Optional plan settings; pass NULL for the defaults (all fields 0). */
typedef struct {
    int precision;          /* cj_precision (default CJ_FP64) */
    int literal_n;          /* 1: use the paper-literal N = Nx in the kappa formulas instead
                               of the exact N = Nx + 1 (ablation only) */
    int inner_cycle;        /* defect-correction modes: inner cycle length (a power of two);
                               0 = auto (the planner's choice for FP32 or FP64 inner sweeps) */
    int temporal_depth;     /* FP32-inner modes: sweeps fused per HBM round trip (temporal
                               blocking), 1..8; 0 = auto: the depth cj_autotune_depth
                               recorded for this stencil and size class, else 4 for the
                               5-point stencil on grids of 2^16 nodes or more and the
                               9-point one on grids of 2^20 or more, else 1 */
    long long max_sweeps;   /* sweep budget of one solve; 0 = 64 cycles (CJ_JACOBI: the larger
                               of 64 intervals and 4 ln(1/tol) / kmin sweeps) */
    int method;             /* cj_method (default CJ_CJM) */
    int launch;             /* plain FP64 cycles: 0 = auto (a CUDA graph of the cycle's sweeps on
                               grids of up to 2^22 nodes, where one sweep is shorter than a host
                               launch; one launch per sweep above), 1 = one launch per sweep,
                               2 = the graph at any size (needs an even M) */
} cj_options;

/* What one solve did.  The relative residuals are those of the returned u:
 * rel_res_l2 = ||b - L u||_2 / ||b||_2 and rel_res_inf = max|b - L u| / max|b| (absolute
 * when b = 0); floor_est = 2^-53 * S * ||u||_2 / ||b||_2 is the FP64 rounding floor that
 * rel_res_l2 cannot go below (S = sum of the stencil's absolute coefficients). */
typedef struct {
    long long sweeps;       /* weighted sweeps applied (the inner cycles' sweeps for the
                               defect-correction precisions) */
    int cycles;             /* CJM cycles (or outer defect-correction steps) */
    int status;             /* the cj_status the solve returned */
    double rel_res_l2;
    double rel_res_inf;
    double floor_est;
    double seconds;         /* host wall time of the call */
    double sweep_seconds;   /* device time of the sweep phases, by CUDA events recorded on
                               the solve's stream around each cycle's sweeps */
    long long launches;     /* kernels the call launched */
} cj_result;

typedef struct cj_plan cj_plan;

/* Human-readable name of a status code (static storage). */
const char *cj_status_string(int status);

/* Last CUDA error message of the calling thread (static storage, may be ""). */
const char *cj_last_error(void);

/*
 * cj_plan_create -- precompute everything a solve of this problem needs (Sec. 2.1:
 * the weights are "precalculated before starting the iterative algorithm").
 *   1 <= Nx, Ny <= 2^20 interior nodes; st in {5, 9, 17}; bc = CJ_BC_DIRICHLET0 or
 *   CJ_BC_DIRICHLET (data set by cj_set_boundary); 0 < tol < 1 is the relative residual
 *   target; the cycle length may not exceed 2^24 sweeps.
 * Computes kmin, kmax, the cycle length M (smallest power of two whose Chebyshev
 * bound reaches tol), the M weights in mirror-pairing order and the sweep table
 * w_n = omega_n / c; allocates the device workspace on the current device (two padded
 * solution buffers, the padded b, reduction scratch; for CJ_FP32_INNER also the FP32
 * buffers).  On success *out owns all of it.  Errors: CJ_ERR_INVALID_ARG, CJ_ERR_NOMEM,
 * CJ_ERR_CUDA.
 */
cj_status cj_plan_create(int Nx, int Ny, cj_stencil st, cj_bc bc, double tol,
                         const cj_options *opt, cj_plan **out);

/*
 * Position-dependent coefficient masks (Sec. 3.2 and its table of Cartesian, polar and
 * bipolar examples): the operator (A u)(i, j) = sum over the pattern's offsets (dx, dy) of
 * s(i, j) c_{dx,dy}(i, j) u(i+dx, j+dy), A u = f, on nodes 1..Nx x 1..Ny, with the Dirichlet
 * ring of a CJ_BC_DIRICHLET plan (zero until cj_set_boundary sets it).
 *   pattern: 5 (the cross |dx|+|dy| = 1), 9 (the 3 x 3 box), 17 (the points of Eq. 2: the 3 x 3
 *     box, (+-2, 0), (0, +-2), (+-2, +-2)), 25 (the 5 x 5 box).
 *   coef: device, K+1 planes (K = 4, 8, 16, 24): plane 0 the centre c_C, then the off-centre
 *     offsets in row-major order (dy = -R..R, then dx = -R..R); value of plane k at (i, j) =
 *     coef[k*sp + (j-1)*sy + (i-1)*sx] (element strides; 0 repeats along that axis, e.g. a
 *     polar mask that varies with r = x1 only has sy = 0).  Read during cj_plan_create_mask only.
 *   scale: device or NULL (= 1), a node factor s(i, j) = scale[(j-1)*scale_sy + (i-1)*scale_sx]
 *     of every coefficient (e.g. the bipolar (cosh nu - cos mu)/a^2).  Read during the call only.
 *   kmin, kmax: bounds of the spectrum of D^-1 A, D = diag(s c_C), which the paper gives only
 *     for its uniform Cartesian stencils; too small a kmin only lengthens the cycle.
 * The solver iterates the Jacobi-normalised system (chat_k = c_k/c_C, bhat = f/(s c_C)):
 *   r = (u_C - bhat) + sum_k chat_k u_k, u' = u_C - w_n r, w_n = omega_n (or 1 for CJ_JACOBI),
 * and its relative residual is ||r||_2 / ||bhat||_2 (floor_est with S = 2).
 */
typedef enum { CJ_MASK5 = 5, CJ_MASK9 = 9, CJ_MASK17 = 17, CJ_MASK25 = 25 } cj_mask_pattern;

typedef struct {
    int pattern;                 /* cj_mask_pattern */
    const double *coef;          /* device coefficient planes (see above) */
    long long sx, sy, sp;        /* their element strides, >= 0 */
    const double *scale;         /* device node factor or NULL */
    long long scale_sx, scale_sy;
    double kmin, kmax;           /* 0 < kmin < kmax */
} cj_mask;

/*
 * cj_plan_create_mask -- a plan for a masked operator; use it with cj_solve, cj_solve_history,
 * cj_solve_host, cj_solve_to_error, cj_sweeps, cj_residual and cj_set_boundary.  f is the
 * right-hand side of A u = f as given (no h^2 scaling).  Options: CJ_FP64 only (precision),
 * method CJ_CJM or CJ_JACOBI, max_sweeps; sweeps are launched one per kernel.  Returns
 * CJ_ERR_INVALID_ARG for a bad size, pattern, stride, bound or option, or a zero centre
 * coefficient (cj_last_error says which).
 */
cj_status cj_plan_create_mask(int Nx, int Ny, const cj_mask *mask, double tol, const cj_options *opt,
                              cj_plan **out);

/* Frees the plan and its device workspace (NULL is ignored). */
void cj_plan_destroy(cj_plan *plan);

/*
 * cj_plan_weights -- the plan's numbers alone, computed on the host with no device work or
 * allocation (Sec. 2.1: the weights are precalculated before the iteration): kmin, kmax of
 * D^-1 A (equations after Eq. 1 and Eq. 2; the exact N = Nx + 1, or the paper-literal N = Nx when
 * literal_n is 1), the cycle length M and the M sweep coefficients w_n = omega_n / c in
 * application order (mirror pairing), bit-equal to cj_plan_info's.  This is what every rank of a
 * decomposed solve needs of the whole grid's plan.  Arguments as cj_plan_create; w: host array of
 * cap doubles, or NULL to ask for M, kmin, kmax only (any of those may be NULL).
 * CJ_ERR_INVALID_ARG for a bad argument, a cycle longer than 2^24, or cap < M with w given.
 */
cj_status cj_plan_weights(int Nx, int Ny, cj_stencil st, double tol, int literal_n, double *w, long long cap,
                          long long *M, double *kmin, double *kmax);

/*
 * cj_plan_info -- the plan's numbers (any output pointer may be NULL).
 *   *w      host array of M per-sweep coefficients w_n = omega_n / c in application order
 *           (owned by the plan, valid until cj_plan_destroy);
 *   *M      cycle length; *kmin, *kmax eigenvalue bounds of D^-1 A;
 *   *M_inner inner cycle length of the defect-correction precisions (0 for CJ_FP64).
 */
cj_status cj_plan_info(const cj_plan *plan, const double **w, long long *M, double *kmin,
                       double *kmax, long long *M_inner);

/*
 * cj_solve -- full CJM solve on the device (Sec. 2.1 with the plan's readings).
 *   f: device, Ny x ld_f doubles, the unscaled right-hand side f of Delta_h u = f.
 *   u: device, Ny x ld_u doubles; in: initial guess, out: the solution.
 * Runs the cycles on `stream`; the residual is tested on the host before each cycle,
 * so the call blocks until the solve ends.  Stops with CJ_OK when the relative
 * residual <= tol, CJ_FLOOR when it is within 4 x floor_est of the rounding floor of the
 * solution's representation, CJ_STALLED when it stopped falling above that (one plain cycle --
 * two consecutive outer steps of a defect-correction precision -- failed to halve it),
 * CJ_ERR_NOT_CONVERGED when the sweep budget is spent,
 * CJ_ERR_DIVERGED on a non-finite residual.  *res (may be NULL) describes the run.
 */
cj_status cj_solve(cj_plan *plan, const double *f, long long ld_f, double *u, long long ld_u,
                   void *stream, cj_result *res);

/*
 * cj_solve_history -- cj_solve that also records the relative L2 residual found at every
 * residual test (before each cycle / outer step, and the final one) into the host array
 * history[0 .. cap-1]; *count receives the number of tests made (which may exceed cap).
 */
cj_status cj_solve_history(cj_plan *plan, const double *f, long long ld_f, double *u,
                           long long ld_u, void *stream, cj_result *res, double *history,
                           int cap, int *count);

/*
 * cj_solve_to_error -- plain FP64 CJM stopped by the real error instead of the residual
 * (Sec. 3.4 and Fig. 4 right, where the analytic solution of the test problem of Sec. 3.3 is
 * known and the solve runs until the infinity norm of u - u_exact reaches a goal).
 *   f, u: as in cj_solve (device, Ny x ld doubles; u in/out).
 *   u_exact: device, Ny x ld_exact doubles, the analytic solution at the interior nodes.
 *   err_tol: the real-error goal (>= 0).
 *   check_every: the real error is tested before every cycle and, when > 0, after every
 *     check_every sweeps inside a cycle (0: at cycle ends only); the plan's tolerance sets
 *     only the cycle length M.  For the defect-correction precisions the error of u (u_hi)
 *     is tested at every outer step, after its defect; check_every must be 0 and history
 *     counts inner sweeps.
 *   history: host array of 2*cap doubles (may be NULL when cap = 0) receiving (sweeps done,
 *     real error) at every test; *count (may be NULL) = number of tests made (may exceed cap).
 *   *real_error (may be NULL): the real error at the last test.
 * Returns CJ_OK when the goal is met; CJ_FLOOR or CJ_STALLED when the residual, still evaluated
 * before every cycle, reaches its floor or stalls first (a goal below the discretisation error); CJ_ERR_NOT_CONVERGED when the
 * sweep budget is spent; CJ_ERR_DIVERGED on a non-finite error; CJ_ERR_INVALID_ARG for a
 * classical-Jacobi plan, a NULL u_exact, ld_exact < Nx, err_tol < 0, check_every < 0, or a
 * nonzero check_every on a defect-correction plan.
 * Works with either boundary type (cj_set_boundary data for CJ_BC_DIRICHLET plans).
 */
cj_status cj_solve_to_error(cj_plan *plan, const double *f, long long ld_f, double *u,
                            long long ld_u, const double *u_exact, long long ld_exact,
                            double err_tol, long long check_every, void *stream, cj_result *res,
                            double *real_error, double *history, int cap, int *count);

/*
 * cj_solve_host -- cj_solve for host arrays: copies f (Ny x Nx, ld = Nx) and the initial
 * guess u to the device in one transfer each, solves, and copies u back (Sec. 3.2:
 * one transfer in, one out).  u_host is in/out.
 */
cj_status cj_solve_host(cj_plan *plan, const double *f_host, double *u_host, void *stream,
                        cj_result *res);

/*
 * cj_sweeps -- apply `count` weighted FP64 sweeps to u in place, with the plan's weights
 * w_{first mod M}, w_{first+1 mod M}, ... (the sweep of Sec. 2.1 alone, no stop test).
 * f, u: device, as for cj_solve.  Asynchronous on `stream`.
 */
cj_status cj_sweeps(cj_plan *plan, const double *f, long long ld_f, double *u, long long ld_u,
                    long long first, long long count, void *stream);

/*
 * cj_sweeps_ff -- cj_sweeps evaluated in float-float arithmetic on the FP32 pipe: the same weighted
 * sweeps (Sec. 2.1) with the iterate and b held as pairs of floats (48 significant bits) and
 * added and multiplied by error-free transformations (Knuth's TwoSum, the fused-multiply-add
 * TwoProduct), in the FP64 sweep's evaluation order.  Not bit-equal to cj_sweeps: each sweep
 * agrees with the FP64 sweep of the same input to a few units of 2^-47 of the terms it adds (within
 * 1e-12 x (max|u| + |w_n| (9 max|u| + max|b|))); it moves the same bytes with FP32 instructions, where the FP64
 * sweep is bound by GB300's FP64 rate.  Values must lie in the float range.  Plain FP64 plans of the
 * paper's stencils with the homogeneous boundary (CJ_BC_DIRICHLET0) only, else CJ_ERR_INVALID_ARG.
 * Arguments and layout as cj_sweeps; asynchronous on `stream`.
 */
cj_status cj_sweeps_ff(cj_plan *plan, const double *f, long long ld_f, double *u, long long ld_u,
                       long long first, long long count, void *stream);

/*
 * cj_sweeps_f32 -- apply `count` weighted FP32 sweeps e <- e + w32_n (L e - r) in place,
 * w32_n = (float) w_n of the plan's inner cycle (FP32-inner plans only), fused
 * temporal_depth at a time per launch as the solve does (bit-identical to one at a time):
 * depths 2-4 (5 and 9 points) and 2 (17 points) by the register wavefront kernel, 8 (and
 * 17-point 4) by the shared-memory wavefront kernel, 1 by the one-sweep kernel; a remainder
 * shorter than the depth, or a depth no kernel serves, runs at the largest served depth that
 * fits.  r, e: device, Ny x ld floats.  Asynchronous on `stream`.
 */
cj_status cj_sweeps_f32(cj_plan *plan, const float *r, long long ld_r, float *e, long long ld_e,
                        long long first, long long count, void *stream);

/*
 * cj_set_boundary -- Dirichlet data of a CJ_BC_DIRICHLET plan (Sec. 3.3: "the analytic
 * solution ... can be used to compute the boundaries"): g is a device array of Ny+4 rows of
 * ld_g >= Nx+4 doubles with node (i, j), -1 <= i <= Nx+2, -1 <= j <= Ny+2, at
 * g[(j+1)*ld_g + (i+1)]; only the two-node ring around the interior is read (the 5- and
 * 9-point stencils use its inner ring only).  The values stay in the plan and are used by
 * every later cj_solve / cj_sweeps / cj_residual of the plan until set again.  The error of
 * the iteration then sees the operator with zero ghosts, whose spectrum lies inside the
 * paper's [kmin, kmax], so the weights are unchanged.  Asynchronous on `stream`.
 */
cj_status cj_set_boundary(cj_plan *plan, const double *g, long long ld_g, void *stream);

/*
 * cj_autotune_depth -- measure the FP32 sweep at temporal depths 1, 2, 4 and 8 on an Nx x Ny
 * grid (`sweeps` >= 8 sweeps each, CUDA events on `stream`), and record the fastest for the
 * stencil and size class (grids whose node counts are within a factor 4 share a class) in a
 * per-process table; FP32-inner plans created afterwards with temporal_depth = 0 use it.
 * *best_depth (may be NULL) receives the winner, gupd[4] (may be NULL) the measured
 * grid-point updates per second (1e9) at depths 1, 2, 4, 8.  Allocates a temporary plan.
 */
cj_status cj_autotune_depth(int Nx, int Ny, cj_stencil st, int sweeps, void *stream, int *best_depth,
                            double *gupd);

/*
 * cj_solution_lo -- for a CJ_FP32_INNER_DD or CJ_FP64_INNER_DD plan, the low part u_lo of the last solve's
 * double-FP64 solution (cj_solve returned u = u_hi, with |u_lo| <= ulp(u_hi)/2); the
 * relative residual cj_result reported is that of u_hi + u_lo.  u_lo: device, Ny x ld
 * doubles.  Asynchronous on `stream`.  CJ_ERR_INVALID_ARG for other plans.
 */
cj_status cj_solution_lo(cj_plan *plan, double *u_lo, long long ld, void *stream);

/*
 * cj_residual -- relative residual norms of u (the stop test of cj_solve, alone).
 *   f, u: device, as for cj_solve.  Writes *rel_l2, *rel_inf, *floor_est (any may be
 *   NULL) and blocks until they are known.
 */
cj_status cj_residual(cj_plan *plan, const double *f, long long ld_f, const double *u,
                      long long ld_u, void *stream, double *rel_l2, double *rel_inf,
                      double *floor_est);

/* ------------------------------------------------------------------ batched solves */

/* One problem of a batch (device grids, as for cj_solve). */
typedef struct {
    int Nx, Ny;
    cj_stencil st;
    int precision;          /* CJ_FP32_INNER or CJ_FP32_INNER_DD; 0 = CJ_FP32_INNER unless the
                               FP64 floor (about 2^-53 S / (c kmin)) is within 4x of tol */
    double tol;
    int inner_cycle;        /* 0 = the planner's choice */
    int temporal_depth;     /* FP32 sweeps per sweep launch (temporal blocking), 1..8; 0 = the
                               cj_autotune_engine choice for the size class, else 4 for 5- and
                               9-point problems with both sides >= 512, else 1.  Depth 4 of 5 and 9
                               points runs the register wavefront of cj_sweeps_f32 over the
                               problem's (strip, row block) items; other depths > 1 run tiles
                               staged in shared memory */
    long long max_sweeps;   /* 0 = 64 inner cycles */
    const double *f;        /* device, Ny x ld_f, unscaled right-hand side */
    long long ld_f;
    double *u;              /* device, Ny x ld_u: initial guess in, solution out */
    long long ld_u;
} cj_problem;

/*
 * cj_solve_batch -- solve n independent problems (any sizes, stencils, tolerances) together
 * with the mixed-precision CJM: FP32 inner cycles inside FP64 or double-FP64 defect
 * correction, every problem's residual test and stop rule evaluated on the device.  The
 * problems run as slots of one engine whose step (correct, defect, decide, eight sweep
 * launches, export, advance: launches over persistent
 * grids that read a device tile list of 128-column tiles) is captured once in a CUDA graph
 * and replayed until every slot has finished; finished problems leave the tile list; tile
 * rows (16/32/64) and depth come from cj_autotune_engine's table for the size class when it
 * has an entry (depth-4 problems of 5 and 9 points sweep on the register wavefront instead of
 * tiles, one warp per 128-column strip and 128-row block, four sweeps per launch).  A problem's arithmetic does not depend on its batch-mates.  results[k] receives problem k's outcome (status per
 * problem; seconds and launches are those of the whole batch).  Orders itself after the
 * work already on `stream` and makes `stream` wait for it; blocks until done.  Returns
 * CJ_OK, or CJ_ERR_TIMEOUT if a problem did not finish within its sweep budget's steps.
 */
cj_status cj_solve_batch(const cj_problem *problems, int n, void *stream, cj_result *results);

/* ------------------------------------------------------------------ request server */

typedef struct cj_server cj_server;

typedef struct {
    long long queued, active, admitted, completed, steps, peak_active;
    size_t bytes_in_use, peak_bytes, budget_bytes;
} cj_server_stats_t;

/*
 * cj_autotune_engine -- tile rows (16, 32 or 64; 128 columns) and FP32 temporal depth (1, 2 or 4)
 * of the batched / served engine for a stencil and size class (grids within a factor 2 per side),
 * picked by timing the engine loaded with copies of a synthetic problem of Nx x Ny nodes (as
 * many as give the device ~8 tiles per SM, up to 256 and 2^24 nodes) at every combination, and
 * recorded in a per-process table that cj_solve_batch and the server use for problems of that
 * class (the server sweeps one at a time, so it takes the tile rows only; an explicit
 * temporal_depth overrides the depth).  Depth 4 of 5 and 9 points (the register wavefront) is a
 * candidate only when both sides are at least 512: below that its four-sweep launches are
 * latency-bound in a batch, which copies of one problem do not show (its rate is then reported
 * as 0).  Not a method of the paper: a runtime choice of this library.  Synchronous; allocates
 * an Nx x Ny FP64 grid and the engine's slots while it runs.
 *   tile_rows, depth: the choice (may be NULL);
 *   gupd: host array of 9 (may be NULL): measured Gupdates/s, tile rows 16/32/64 (major) x
 *     depth 1/2/4.
 * Returns CJ_ERR_INVALID_ARG for a bad size or stencil.
 */
cj_status cj_autotune_engine(int Nx, int Ny, cj_stencil st, int *tile_rows, int *depth, double *gupd);

/*
 * cj_server_create -- a request loop with continuous batching on the current device.  Requests
 * are sorted into three size lanes (up to 2^20 nodes, up to 2^23, larger); each lane is an engine
 * with up to max_slots slots, its own stream (smaller lanes at higher stream priority) and its
 * own worker thread, which admits the lane's requests, in arrival order, into free slots while
 * their device footprint (FP64 u, b [, u_lo], FP32 e, e', r, weights; 28-36 bytes per node) fits
 * in hbm_budget_bytes (one budget shared by the lanes); admitted problems join the lane's running
 * engine between graph replays and leave it as each one finishes, so requests arriving while
 * others run overlap with them on the device, and a small request's replays sweep only small
 * grids: its latency follows its own work, not that of the largest grids being solved.  The
 * two smaller lanes sweep one sweep per launch; the largest lane sweeps 5- and 9-point requests
 * with both sides of at least 512 on the register wavefront (four sweeps per launch), launched
 * with half a wave of blocks so that the smaller lanes' blocks still find room on every SM.
 * While the smallest lane has requests on the device, the two larger lanes hold their next
 * graph replay (32 sweeps of their slots), within an allowance of 1 s that refills at 0.5 s per
 * second, so a larger lane still runs at least half the time under a sustained stream of small
 * requests.  Results do not depend on the lanes' timing.
 */
cj_status cj_server_create(size_t hbm_budget_bytes, int max_slots, cj_server **out);

/*
 * cj_submit -- queue one solve: f_host (Ny x Nx, copied before return), tolerance tol; the
 * precision follows cj_problem.precision = 0.  *ticket identifies it for cj_poll.
 * CJ_ERR_INVALID_ARG for bad sizes; a problem larger than the whole budget completes with
 * CJ_ERR_BUDGET.
 */
cj_status cj_submit(cj_server *server, int Nx, int Ny, cj_stencil st, double tol, const double *f_host,
                    uint64_t *ticket);

/*
 * cj_poll -- CJ_PENDING while the request is queued or running; otherwise its final status,
 * with the solution copied to u_host (Ny x Nx, may be NULL) and *res filled: res->seconds =
 * latency from submit to result ready, res->sweep_seconds = service time from admission into a
 * slot to result ready (the rest of the latency is the wait in the lane's queue).  A finished
 * ticket can be polled once.
 */
cj_status cj_poll(cj_server *server, uint64_t ticket, double *u_host, cj_result *res);

/* Counters of the server (queue, active slots, admitted, completed, engine steps, memory). */
cj_status cj_server_stats(cj_server *server, cj_server_stats_t *out);

/* Stops the worker (requests still queued or running are dropped) and frees the server. */
void cj_server_destroy(cj_server *server);

/*
 * cj_residual_noalloc -- the relative residual norms of cj_residual for a homogeneous-Dirichlet
 * problem (those of a CJ_BC_DIRICHLET0 plan: zero boundary nodes, odd reflection for the
 * 17-point stencil's second ring; no boundary data is read), for callers that cannot allocate
 * device memory: for example code running under a framework whose caching
 * allocator has already reserved the device (a cudaMalloc of its own would fail or carve
 * up that pool), or a latency-critical loop that must not take the device-wide
 * synchronisation cudaMalloc / cudaFree can cause.  It needs no plan and calls no
 * cudaMalloc, cudaFree or allocating library routine.  (The paper has no counterpart: it
 * is a deployment variant of the stop test's residual.)
 *   1 <= Nx, Ny <= 2^20, st in {5, 9, 17}; f, u: device, Ny x ld_f / Ny x ld_u doubles (f
 *   unscaled, as for cj_solve); out: device, 3 doubles, receives (rel_l2, rel_inf, floor_est)
 *   as in cj_residual (a NaN anywhere in the residual makes both norms NaN).  Asynchronous on
 *   `stream`: out is valid once the stream reaches the call.
 * Scratch: a fixed 640 KiB array in the library's device memory, one slot per block of
 * 128 x 64 nodes, 16384 slots; grids needing more slots (more than 134,217,728 nodes) are
 * rejected with CJ_ERR_INVALID_ARG and a message in cj_last_error().  Every GPU that loads
 * the library holds that array until the process exits.  The first call made on a device
 * looks up the array's device address (cudaGetSymbolAddress) with that device current;
 * make that first call before any stream capture.  All calls share the one array, so
 * calls that may overlap on the GPU (different streams, no ordering between them) race
 * and must not be issued; calls on one stream are ordered and safe.  Each call writes
 * every slot it later reads, so nothing needs clearing between calls.
 */
cj_status cj_residual_noalloc(int Nx, int Ny, cj_stencil st, const double *f, long long ld_f,
                              const double *u, long long ld_u, double *out, void *stream);

/* ------------------------------------------------------------------ subdomains */

/*
 * Kernels for a rank of a 2-D domain decomposition of one grid (the partition, the halo exchange
 * and the stop test across ranks are host logic; the Python module dd.py drives them).  The grid
 * is split into blocks; each rank keeps its block in an extended array whose margin holds the
 * neighbours' halo (or, on the sides that are the grid's boundary, the homogeneous ghosts: 0 at
 * distance 1 and, for the 17-point stencil, the odd reflection at distance 2).  Both kernels work
 * on a box of nx x ny nodes of such an array: u, b and out point at the box's first node, rows
 * ld apart, and the stencil reads up to 2 nodes outside the box from the array itself, which the
 * caller guarantees exist.  The arithmetic and its order are those of the plan kernels, so a
 * decomposed solve gives the undecomposed solve's bits at every node.
 *
 * cj_box_sweep -- out = u + w (L u - b) on the box (Sec. 2.1's sweep with the weight w);
 *   out != u, ldo == ldu.  edges: bit 0 the box's first column is the grid's column 1, bit 1 its
 *   last is column Nx, bit 2 its first row is row 1, bit 3 its last is row Ny; for the 17-point
 *   stencil the odd-reflection ghosts beyond those sides are written with the nodes.
 * cj_box_residual -- (sum r^2, max |r|, sum u^2, sum b^2, max |b|) of r = L u - b over the box
 *   into out[0..4] (device), reduced in a fixed order (maxima keep a NaN); scratch: device, at
 *   least cj_box_residual_slots(nx, ny) doubles.
 * cj_box_scale -- dst = alpha * src on nx x ny nodes (b = h^2 f of a block).
 * All asynchronous on `stream`.  Errors: CJ_ERR_INVALID_ARG, CJ_ERR_CUDA.
 */
cj_status cj_box_sweep(int nx, int ny, cj_stencil st, double w, const double *u, long long ldu, const double *b,
                       long long ldb, double *out, long long ldo, int edges, void *stream);
cj_status cj_box_residual(int nx, int ny, cj_stencil st, const double *u, long long ldu, const double *b,
                          long long ldb, double *scratch, long long scratch_len, double *out, void *stream);
long long cj_box_residual_slots(int nx, int ny);
cj_status cj_box_scale(int nx, int ny, double alpha, const double *src, long long lds, double *dst, long long ldd,
                       void *stream);

/*
 * cj_issue_peaks -- measured FP64 and FP32 fused multiply-add issue rates of the current device,
 * in 10^12 FMA instructions per second: the denominators of the instruction-issue rooflines of
 * the FP64 sweep (on GB300 every FP64 operation of its tree is issued as an FMA, and the FP64
 * pipe, not HBM, bounds it) and of the temporally blocked FP32 sweep.  Not part of the paper's
 * method: a measurement of this library.  Each thread of 4 blocks of 256 per SM runs 8
 * independent dependent FMA chains; the rate is the FMAs of one launch over its CUDA-event time
 * on `stream`, after a warm-up launch (each stream about 50 ms).  Either output may be NULL (not
 * measured), not both.  Synchronous.  Errors: CJ_ERR_INVALID_ARG, CJ_ERR_CUDA.
 */
cj_status cj_issue_peaks(void *stream, double *fp64_tfma, double *fp32_tfma);

#ifdef __cplusplus
}
#endif

#endif /* CJ_H */
