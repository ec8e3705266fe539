// C ABI of libcj: plan lifetime, the CJM solve drivers (Sec. 2.1: "a set of weights ...
// precalculated before starting the iterative algorithm", then M weighted sweeps per
// cycle), the sweep and residual entry points.  Host C++; the device work is in
// kernels.cu.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <utility>

#include "cj_internal.h"

int stencil_slot(int st) { return st == 5 ? 0 : st == 9 ? 1 : 2; }

int size_class(int Nx, int Ny) {
    long long n = (long long)Nx * Ny;
    int c = 0;
    while (n > 3) {
        n >>= 2;
        ++c;
    }
    return c < 32 ? c : 31;
}

namespace {

thread_local char g_err[256] = "";

// Autotuned FP32 temporal depth per (stencil, size class); size class = floor(log2(Nx*Ny)/2),
// i.e. grids within a factor 2 of each other per side share a class.  0 = not tuned.
std::mutex g_tune_mu;
int g_tuned_depth[3][32] = {};


int tuned_depth(int st, int Nx, int Ny) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    return g_tuned_depth[stencil_slot(st)][size_class(Nx, Ny)];
}

const double kEps = 1.1102230246251565e-16;  // 2^-53

bool is_pow2(long long m) { return m >= 1 && (m & (m - 1)) == 0; }

void free_plan(cj_plan *p) {
    if (!p) return;
    cudaFree(p->u0);
    cudaFree(p->u1);
    cudaFree(p->b);
    cudaFree(p->e0);
    cudaFree(p->e1);
    cudaFree(p->rt);
    cudaFree(p->d0);
    cudaFree(p->d1);
    cudaFree(p->r64);
    cudaFree(p->partials);
    cudaFree(p->red);
    if (p->h_red) cudaFreeHost(p->h_red);
    if (p->ev0) cudaEventDestroy(p->ev0);
    if (p->ev1) cudaEventDestroy(p->ev1);
    if (p->graph) cudaGraphExecDestroy(p->graph);
    cudaFree(p->w_dev);
    cudaFree(p->pos);
    cudaFree(p->chat);
    cudaFree(p->dC);
    delete p;
}

template <typename T>
cudaError_t dev_alloc(T **ptr, size_t count) {
    cudaError_t e = cudaMalloc((void **)ptr, count * sizeof(T));
    if (e != cudaSuccess) return e;
    return cudaMemset(*ptr, 0, count * sizeof(T));
}

// Stop rule applied after each residual evaluation; -1 = go on.  Converged at tol; at
// the rounding floor when rho <= 4 fl; stalled when `patience` consecutive cycles each
// failed to halve rho above that (*stall counts them): 1 for plain cycles, 2 for
// defect-correction steps, whose residual may jump up once (rounding noise of the inner
// cycle, high-frequency) before it contracts.
int stop_rule(double rho, double fl, double prev, long long cycles, double tol, int patience,
              int *stall) {
    if (rho <= tol) return CJ_OK;
    if (!(rho == rho) || rho > 1e300) return CJ_ERR_DIVERGED;
    if (rho <= 4.0 * fl) return CJ_FLOOR;
    if (cycles > 0) {
        *stall = rho > 0.5 * prev ? *stall + 1 : 0;
        if (*stall >= patience) return CJ_STALLED;
    }
    return -1;
}

// Stop rule of classical Jacobi, tested every M sweeps: its residual falls monotonically in
// exact arithmetic, so an interval that did not lower it has stalled on rounding.
int jacobi_stop_rule(double rho, double fl, double prev, long long intervals, double tol) {
    if (rho <= tol) return CJ_OK;
    if (!(rho == rho) || rho > 1e300) return CJ_ERR_DIVERGED;
    if (rho <= 4.0 * fl) return CJ_FLOOR;
    if (intervals > 0 && rho >= prev) return CJ_STALLED;
    return -1;
}

// Optional convergence history of the call in progress (rho at every residual test).
struct History {
    double *buf = nullptr;
    int cap = 0, n = 0;
    void add(double v) {
        if (n < cap) buf[n] = v;
        ++n;
    }
};

struct Norms {
    double l2, inf, fl;
    double err, err_sq;  // real error: max |u - u_exact| and sum (u - u_exact)^2 (red[5..6])
};

// Reads red[] (filled by the residual and import reductions) after a stream sync.  The
// floor estimate uses unit roundoff `eps` of the solution's representation.
cj_status fetch_norms(cj_plan *p, cudaStream_t s, Norms *n, double eps = kEps) {
    cudaError_t e = cudaMemcpyAsync(p->h_red, p->red, 8 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        set_cuda_error(e, "residual readback");
        return CJ_ERR_CUDA;
    }
    const double *r = p->h_red;
    double bn = std::sqrt(r[3]), bmax = r[4];
    double rn = std::sqrt(r[0]), un = std::sqrt(r[2]);
    n->l2 = bn > 0.0 ? rn / bn : rn;
    n->inf = bmax > 0.0 ? r[1] / bmax : r[1];
    n->fl = bn > 0.0 ? eps * p->S * un / bn : eps * p->S * un;
    n->err_sq = r[5];
    n->err = r[6];
    return CJ_OK;
}

// Device time between the plan's two events (both already completed).
double elapsed_ms(cj_plan *p) {
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, p->ev0, p->ev1) != cudaSuccess) return 0.0;
    return ms;
}

#define CJ_TRY(call, where)                 \
    do {                                    \
        cudaError_t e_ = (call);            \
        if (e_ != cudaSuccess) {            \
            set_cuda_error(e_, where);      \
            return CJ_ERR_CUDA;             \
        }                                   \
    } while (0)

cj_status check_grid_args(const cj_plan *p, const void *f, long long ldf, const void *u,
                          long long ldu) {
    if (!p || !f || !u || ldf < p->Nx || ldu < p->Nx) return CJ_ERR_INVALID_ARG;
    return CJ_OK;
}

// FP64 launchers for either operator: the paper's stencils or a coefficient mask.
cudaError_t sweep64(const cj_plan *p, const double *u, double *out, double w, cudaStream_t s) {
    return p->pattern ? launch_mask_sweep(p, u, out, w, s) : launch_sweep64(p, u, out, w, s);
}

cudaError_t residual64(const cj_plan *p, const double *u, cudaStream_t s) {
    return p->pattern ? launch_mask_residual(p, u, s) : launch_residual(p, u, nullptr, nullptr, s);
}

cudaError_t import64(const cj_plan *p, const double *f, long long ldf, const double *u, long long ldu,
                     cudaStream_t s) {
    return p->pattern ? launch_mask_import(p, f, ldf, u, ldu, s)
                      : launch_import(p, f, ldf, u, ldu, p->b, p->u0, s);
}

// A whole plain FP64 solve in one cluster launch (small grids): the stop test runs on the
// device, so its outcome is read back behind the solution's export, and the host synchronises
// once per solve.
cj_status solve_fp64_cluster(cj_plan *p, double *u, long long ldu, cudaStream_t s, cj_result *res) {
    CJ_TRY(cudaEventRecord(p->ev0, s), "event");
    CJ_TRY(launch_cluster_solve(p, p->red, s), "cluster solve");
    CJ_TRY(cudaEventRecord(p->ev1, s), "event");
    CJ_TRY(cudaMemcpyAsync(p->h_red, p->red, 6 * sizeof(double), cudaMemcpyDeviceToHost, s), "cluster readback");
    CJ_TRY(launch_export(p, p->u0, u, ldu, s), "export");
    res->launches += 2;
    CJ_TRY(cudaStreamSynchronize(s), "solve sync");
    const double *r = p->h_red;
    res->sweep_seconds = 1e-3 * elapsed_ms(p);
    res->status = (int)r[0];
    res->sweeps = (long long)r[1];
    res->cycles = (int)r[2];
    res->rel_res_l2 = r[3];
    res->rel_res_inf = r[4];
    res->floor_est = r[5];
    return (cj_status)res->status;
}

// The solve proper, once f and u have been imported into the plan's padded buffers.
cj_status run_fp64(cj_plan *p, cudaStream_t s, double **cur_out, cj_result *res, History *h) {
    double *cur = p->u0, *nxt = p->u1;
    long long sweeps = 0, cycles = 0;
    double prev = 0.0, sweep_ms = 0.0;
    bool timed = false;
    Norms n{};
    int stat, stall = 0;
    for (;;) {
        CJ_TRY(residual64(p, cur, s), "residual");
        res->launches += 2;
        cj_status st = fetch_norms(p, s, &n);
        if (st != CJ_OK) return st;
        if (timed) sweep_ms += elapsed_ms(p);
        h->add(n.l2);
        stat = p->method == CJ_JACOBI ? jacobi_stop_rule(n.l2, n.fl, prev, cycles, p->tol)
                                      : stop_rule(n.l2, n.fl, prev, cycles, p->tol, 1, &stall);
        if (stat != -1) break;
        if (sweeps + p->M > p->max_sweeps) {
            stat = CJ_ERR_NOT_CONVERGED;
            break;
        }
        CJ_TRY(cudaEventRecord(p->ev0, s), "event");
        if (p->graph) {
            // a cycle from u0 ends in u0 (M even)
            CJ_TRY(launch_sweep_cycle_graph(p, s), "sweep graph");
            res->launches += p->M / p->graph_G;  // the position advances
        } else {
            for (long long k = 0; k < p->M; ++k) {
                CJ_TRY(sweep64(p, cur, nxt, p->w[k], s), "sweep");
                double *t = cur;
                cur = nxt;
                nxt = t;
            }
        }
        CJ_TRY(cudaEventRecord(p->ev1, s), "event");
        timed = true;
        res->launches += p->M;
        sweeps += p->M;
        cycles += 1;
        prev = n.l2;
    }
    res->sweep_seconds = 1e-3 * sweep_ms;
    *cur_out = cur;
    res->sweeps = sweeps;
    res->cycles = (int)cycles;
    res->status = stat;
    res->rel_res_l2 = n.l2;
    res->rel_res_inf = n.inf;
    res->floor_est = n.fl;
    return (cj_status)stat;
}

// Real-error stop (Sec. 3.4, Fig. 4 right): plain FP64 cycles of the plan's length; the real
// error E = max |u - u_exact| is tested before every cycle and every `every` sweeps inside one
// (every = 0: at cycle ends only) and the solve stops at the first test with E <= err_tol.  The
// residual is still evaluated before every cycle, for the floor and stall parts of the stop rule
// only (a goal below the discretisation error ends with CJ_FLOOR or CJ_STALLED).  hist
// receives (sweeps, E) pairs.
struct ErrorStop {
    const double *ue;
    long long lde;
    double tol;
    long long every;
    double *hist;
    int cap, n;
    void add(long long sweeps, double e) {
        if (n < cap) {
            hist[2 * n] = (double)sweeps;
            hist[2 * n + 1] = e;
        }
        ++n;
    }
};

cj_status run_fp64_to_error(cj_plan *p, cudaStream_t s, ErrorStop *es, double **cur_out,
                            cj_result *res) {
    double *cur = p->u0, *nxt = p->u1;
    long long sweeps = 0, cycles = 0;
    double prev = 0.0, sweep_ms = 0.0;
    Norms n{};
    int stat = -1, stall = 0;
    bool mid = false;
    for (;;) {
        CJ_TRY(residual64(p, cur, s), "residual");
        CJ_TRY(launch_real_error(p, cur, es->ue, es->lde, s), "real error");
        res->launches += 4;
        cj_status st = fetch_norms(p, s, &n);
        if (st != CJ_OK) return st;
        es->add(sweeps, n.err);
        if (!(n.err_sq == n.err_sq) || n.err > 1e300) {
            stat = CJ_ERR_DIVERGED;
            break;
        }
        if (n.err <= es->tol) {
            stat = CJ_OK;
            break;
        }
        stat = stop_rule(n.l2, n.fl, prev, cycles, 0.0, 1, &stall);
        if (stat == CJ_OK) stat = CJ_FLOOR;  // zero residual: u is the discrete solution
        if (stat != -1) break;
        if (sweeps + p->M > p->max_sweeps) {
            stat = CJ_ERR_NOT_CONVERGED;
            break;
        }
        for (long long k = 0; k < p->M;) {
            const long long chunk = es->every > 0 ? std::min(es->every, p->M - k) : p->M - k;
            CJ_TRY(cudaEventRecord(p->ev0, s), "event");
            for (long long q = 0; q < chunk; ++q) {
                CJ_TRY(sweep64(p, cur, nxt, p->w[k + q], s), "sweep");
                std::swap(cur, nxt);
            }
            CJ_TRY(cudaEventRecord(p->ev1, s), "event");
            res->launches += chunk;
            k += chunk;
            sweeps += chunk;
            if (k < p->M) {
                CJ_TRY(launch_real_error(p, cur, es->ue, es->lde, s), "real error");
                res->launches += 2;
                st = fetch_norms(p, s, &n);
                if (st != CJ_OK) return st;
                sweep_ms += elapsed_ms(p);
                es->add(sweeps, n.err);
                if (!(n.err_sq == n.err_sq) || n.err > 1e300) {
                    stat = CJ_ERR_DIVERGED;
                    mid = true;
                    break;
                }
                if (n.err <= es->tol) {
                    stat = CJ_OK;
                    mid = true;
                    break;
                }
            } else {
                CJ_TRY(cudaStreamSynchronize(s), "cycle sync");
                sweep_ms += elapsed_ms(p);
            }
        }
        if (mid) break;
        cycles += 1;
        prev = n.l2;
    }
    if (mid) {  // the residual where the solve stopped
        CJ_TRY(residual64(p, cur, s), "residual");
        res->launches += 2;
        cj_status st = fetch_norms(p, s, &n);
        if (st != CJ_OK) return st;
    }
    res->sweep_seconds = 1e-3 * sweep_ms;
    *cur_out = cur;
    res->sweeps = sweeps;
    res->cycles = (int)cycles;
    res->status = stat;
    res->rel_res_l2 = n.l2;
    res->rel_res_inf = n.inf;
    res->floor_est = n.fl;
    return (cj_status)stat;
}

// The real-error stop at an outer step of a defect-correction solve (after the defect and the
// real-error launches have been read): the error first, then the floor and stall parts of the
// stop rule.
int mixed_error_stop(ErrorStop *es, long long sweeps, const Norms &n, double prev, long long outer,
                     int *stall) {
    es->add(sweeps, n.err);
    if (!(n.err_sq == n.err_sq) || n.err > 1e300) return CJ_ERR_DIVERGED;
    if (n.err <= es->tol) return CJ_OK;
    const int st = stop_rule(n.l2, n.fl, prev, outer, 0.0, 2, stall);
    return st == CJ_OK ? CJ_FLOOR : st;
}

// One inner cycle of FP32 sweeps with weights w32[first .. first+count-1], `depth` per
// launch; *cur holds the input on entry and the result on exit (ping-pong with *nxt).
cudaError_t fp32_sweeps(cj_plan *p, float **cur, float **nxt, const float *r, long long first,
                        long long count, cudaStream_t s, long long *launches) {
    long long n = 0;
    while (n < count) {
        long long k = p->depth < count - n ? p->depth : count - n;
        // the temporal-blocking kernels exist for depths 2, 3 and 4 (register wavefront; 17
        // points: 2) and 2, 4 and 8 (wavefront strips): use the largest that fits
        while (k > 1 && !wave_reg_supported(p->st, (int)k) && !wave_depth_supported((int)k)) --k;
        cudaError_t e;
        if (k == 1) {
            e = launch_sweep32(p, *cur, r, *nxt, p->w32[(first + n) % p->M_in], s);
        } else {
            float w[kTbMaxDepth];
            for (long long q = 0; q < k; ++q) w[q] = p->w32[(first + n + q) % p->M_in];
            e = wave_reg_supported(p->st, (int)k) ? launch_sweep32_wave_reg(p, *cur, r, *nxt, w, (int)k, s)
                                                   : launch_sweep32_wave(p, *cur, r, *nxt, w, (int)k, s);
        }
        if (e != cudaSuccess) return e;
        float *t = *cur;
        *cur = *nxt;
        *nxt = t;
        n += k;
        ++*launches;
    }
    return cudaSuccess;
}

// Mixed precision: FP64 defect r = b - L u -> FP32 rt; one FP32 CJM cycle of length M_in
// on L e = rt from e = 0; u += e in FP64; repeat until the FP64 stop rule ends it.
cj_status run_mixed(cj_plan *p, cudaStream_t s, double **cur_out, cj_result *res, History *h,
                    ErrorStop *es = nullptr) {
    long long sweeps = 0, outer = 0;
    const long long max_outer = p->max_sweeps / p->M_in;
    double prev = 0.0, sweep_ms = 0.0;
    bool timed = false;
    Norms n{};
    int stat, stall = 0;
    for (;;) {
        CJ_TRY(launch_residual(p, p->u0, p->rt, p->e0, s), "defect");
        res->launches += 2;
        if (es) {
            CJ_TRY(launch_real_error(p, p->u0, es->ue, es->lde, s), "real error");
            res->launches += 2;
        }
        cj_status st = fetch_norms(p, s, &n);
        if (st != CJ_OK) return st;
        if (timed) sweep_ms += elapsed_ms(p);
        h->add(n.l2);
        stat = es ? mixed_error_stop(es, sweeps, n, prev, outer, &stall)
                  : stop_rule(n.l2, n.fl, prev, outer, p->tol, 2, &stall);
        if (stat != -1) break;
        if (outer >= max_outer) {
            stat = CJ_ERR_NOT_CONVERGED;
            break;
        }
        float *cur = p->e0, *nxt = p->e1;
        CJ_TRY(cudaEventRecord(p->ev0, s), "event");
        CJ_TRY(fp32_sweeps(p, &cur, &nxt, p->rt, 0, p->M_in, s, &res->launches), "sweep32");
        CJ_TRY(cudaEventRecord(p->ev1, s), "event");
        timed = true;
        CJ_TRY(launch_correct(p, p->u0, cur, s), "correct");
        res->launches += 1;
        sweeps += p->M_in;
        outer += 1;
        prev = n.l2;
    }
    res->sweep_seconds = 1e-3 * sweep_ms;
    *cur_out = p->u0;
    res->sweeps = sweeps;
    res->cycles = (int)outer;
    res->status = stat;
    res->rel_res_l2 = n.l2;
    res->rel_res_inf = n.inf;
    res->floor_est = n.fl;
    return (cj_status)stat;
}

// Mixed precision with the double-FP64 outer loop: the solution is u0 + u1 (hi + lo), the
// defect is evaluated to about twice FP64 precision and the correction added by TwoSum.
cj_status run_mixed_dd(cj_plan *p, cudaStream_t s, double **cur_out, cj_result *res, History *h,
                       ErrorStop *es = nullptr) {
    long long sweeps = 0, outer = 0;
    const long long max_outer = p->max_sweeps / p->M_in;
    const double eps2 = 1.2325951644078309e-32;  // 2^-106
    double prev = 0.0, sweep_ms = 0.0;
    bool timed = false;
    Norms n{};
    int stat, stall = 0;
    CJ_TRY(cudaMemsetAsync(p->u1, 0, (size_t)p->g64.elems() * sizeof(double), s), "zero u_lo");
    for (;;) {
        CJ_TRY(launch_defect_dd(p, p->u0, p->u1, p->rt, p->e0, s), "defect dd");
        res->launches += 2;
        if (es) {  // the real error of u_hi
            CJ_TRY(launch_real_error(p, p->u0, es->ue, es->lde, s), "real error");
            res->launches += 2;
        }
        cj_status st = fetch_norms(p, s, &n, eps2);
        if (st != CJ_OK) return st;
        if (timed) sweep_ms += elapsed_ms(p);
        h->add(n.l2);
        stat = es ? mixed_error_stop(es, sweeps, n, prev, outer, &stall)
                  : stop_rule(n.l2, n.fl, prev, outer, p->tol, 2, &stall);
        if (stat != -1) break;
        if (outer >= max_outer) {
            stat = CJ_ERR_NOT_CONVERGED;
            break;
        }
        float *cur = p->e0, *nxt = p->e1;
        CJ_TRY(cudaEventRecord(p->ev0, s), "event");
        CJ_TRY(fp32_sweeps(p, &cur, &nxt, p->rt, 0, p->M_in, s, &res->launches), "sweep32");
        CJ_TRY(cudaEventRecord(p->ev1, s), "event");
        timed = true;
        CJ_TRY(launch_correct_dd(p, p->u0, p->u1, cur, s), "correct dd");
        res->launches += 1;
        sweeps += p->M_in;
        outer += 1;
        prev = n.l2;
    }
    res->sweep_seconds = 1e-3 * sweep_ms;
    *cur_out = p->u0;
    res->sweeps = sweeps;
    res->cycles = (int)outer;
    res->status = stat;
    res->rel_res_l2 = n.l2;
    res->rel_res_inf = n.inf;
    res->floor_est = n.fl;
    return (cj_status)stat;
}

// FP64 inner cycles in the double-FP64 outer loop: as run_mixed_dd, with the defect -R kept in
// FP64 (r64) and the inner cycle of M_in FP64 sweeps of L e = r64 (the plain FP64 sweep kernel
// with the homogeneous boundary, weights w_in), so every operation is FP64 or error-free.
cj_status run_fp64_dd(cj_plan *p, cudaStream_t s, double **cur_out, cj_result *res, History *h,
                      ErrorStop *es = nullptr) {
    long long sweeps = 0, outer = 0;
    const long long max_outer = p->max_sweeps / p->M_in;
    const double eps2 = 1.2325951644078309e-32;  // 2^-106
    double prev = 0.0, sweep_ms = 0.0;
    bool timed = false;
    Norms n{};
    int stat, stall = 0;
    CJ_TRY(cudaMemsetAsync(p->u1, 0, (size_t)p->g64.elems() * sizeof(double), s), "zero u_lo");
    for (;;) {
        CJ_TRY(launch_defect_dd64(p, p->u0, p->u1, p->r64, p->d0, s), "defect dd");
        res->launches += 2;
        if (es) {  // the real error of u_hi
            CJ_TRY(launch_real_error(p, p->u0, es->ue, es->lde, s), "real error");
            res->launches += 2;
        }
        cj_status st = fetch_norms(p, s, &n, eps2);
        if (st != CJ_OK) return st;
        if (timed) sweep_ms += elapsed_ms(p);
        h->add(n.l2);
        stat = es ? mixed_error_stop(es, sweeps, n, prev, outer, &stall)
                  : stop_rule(n.l2, n.fl, prev, outer, p->tol, 2, &stall);
        if (stat != -1) break;
        if (outer >= max_outer) {
            stat = CJ_ERR_NOT_CONVERGED;
            break;
        }
        double *cur = p->d0, *nxt = p->d1;
        CJ_TRY(cudaEventRecord(p->ev0, s), "event");
        for (long long k = 0; k < p->M_in; ++k) {
            CJ_TRY(launch_sweep64_err(p, cur, p->r64, nxt, p->w_in[k], s), "sweep");
            std::swap(cur, nxt);
        }
        CJ_TRY(cudaEventRecord(p->ev1, s), "event");
        timed = true;
        res->launches += p->M_in;
        CJ_TRY(launch_correct_dd64(p, p->u0, p->u1, cur, s), "correct dd");
        res->launches += 1;
        sweeps += p->M_in;
        outer += 1;
        prev = n.l2;
    }
    res->sweep_seconds = 1e-3 * sweep_ms;
    *cur_out = p->u0;
    res->sweeps = sweeps;
    res->cycles = (int)outer;
    res->status = stat;
    res->rel_res_l2 = n.l2;
    res->rel_res_inf = n.inf;
    res->floor_est = n.fl;
    return (cj_status)stat;
}

cj_status solve_core(cj_plan *p, const double *f, long long ldf, double *u, long long ldu,
                     cudaStream_t s, cj_result *res, History *h) {
    auto t0 = std::chrono::steady_clock::now();
    cj_result r{};
    CJ_TRY(import64(p, f, ldf, u, ldu, s), "import");
    r.launches = 2;
    if (p->precision == CJ_FP64 && p->cluster_C > 0 && h->cap == 0) {
        cj_status st = solve_fp64_cluster(p, u, ldu, s, &r);
        if (st == CJ_ERR_CUDA) return st;
        r.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (res) *res = r;
        return st;
    }
    double *cur = nullptr;
    cj_status st = p->precision == CJ_FP32_INNER      ? run_mixed(p, s, &cur, &r, h)
                   : p->precision == CJ_FP32_INNER_DD ? run_mixed_dd(p, s, &cur, &r, h)
                   : p->precision == CJ_FP64_INNER_DD ? run_fp64_dd(p, s, &cur, &r, h)
                                                      : run_fp64(p, s, &cur, &r, h);
    if (st < 0 && st != CJ_ERR_NOT_CONVERGED && st != CJ_ERR_DIVERGED) return st;
    CJ_TRY(launch_export(p, cur, u, ldu, s), "export");
    r.launches += 1;
    CJ_TRY(cudaStreamSynchronize(s), "solve sync");
    r.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (res) *res = r;
    return st;
}

}  // namespace

void set_cuda_error(cudaError_t e, const char *where) {
    std::snprintf(g_err, sizeof(g_err), "%s: %s", where, cudaGetErrorString(e));
}

void set_error_text(const char *msg) { std::snprintf(g_err, sizeof(g_err), "%s", msg); }

extern "C" {

const char *cj_status_string(int status) {
    switch (status) {
        case CJ_OK: return "converged";
        case CJ_FLOOR: return "stopped at the rounding floor";
        case CJ_PENDING: return "pending";
        case CJ_STALLED: return "stalled above the rounding floor";
        case CJ_ERR_INVALID_ARG: return "invalid argument";
        case CJ_ERR_NOMEM: return "out of memory";
        case CJ_ERR_NOT_CONVERGED: return "sweep budget exhausted";
        case CJ_ERR_DIVERGED: return "residual not finite";
        case CJ_ERR_TIMEOUT: return "device wait timed out";
        case CJ_ERR_CUDA: return "CUDA error";
        case CJ_ERR_BUDGET: return "memory budget exceeded";
        default: return "unknown status";
    }
}

const char *cj_last_error(void) { return g_err; }

cj_status cj_plan_create(int Nx, int Ny, cj_stencil st, cj_bc bc, double tol,
                         const cj_options *opt, cj_plan **out) {
    if (!out) return CJ_ERR_INVALID_ARG;
    *out = nullptr;
    cj_options o{};
    if (opt) o = *opt;
    if (Nx < 1 || Ny < 1 || Nx > (1 << 20) || Ny > (1 << 20)) return CJ_ERR_INVALID_ARG;
    if (st != CJ_ST5 && st != CJ_ST9 && st != CJ_ST17) return CJ_ERR_INVALID_ARG;
    if (bc != CJ_BC_DIRICHLET0 && bc != CJ_BC_DIRICHLET) return CJ_ERR_INVALID_ARG;
    if (!(tol > 0.0 && tol < 1.0)) return CJ_ERR_INVALID_ARG;
    if (o.precision != CJ_FP64 && o.precision != CJ_FP32_INNER && o.precision != CJ_FP32_INNER_DD &&
        o.precision != CJ_FP64_INNER_DD)
        return CJ_ERR_INVALID_ARG;
    if (o.inner_cycle != 0 && !is_pow2(o.inner_cycle)) return CJ_ERR_INVALID_ARG;
    if (o.max_sweeps < 0) return CJ_ERR_INVALID_ARG;
    if (o.temporal_depth < 0 || o.temporal_depth > kTbMaxDepth) return CJ_ERR_INVALID_ARG;
    if (o.method != CJ_CJM && o.method != CJ_JACOBI) return CJ_ERR_INVALID_ARG;
    if (o.method == CJ_JACOBI && o.precision != CJ_FP64) return CJ_ERR_INVALID_ARG;
    if (o.launch < 0 || o.launch > 3) return CJ_ERR_INVALID_ARG;

    cj_plan *p = new (std::nothrow) cj_plan();
    if (!p) return CJ_ERR_NOMEM;
    try {
        p->Nx = Nx;
        p->Ny = Ny;
        p->st = st;
        p->r = st == CJ_ST17 ? 2 : 1;
        p->precision = o.precision;
        p->literal_n = o.literal_n ? 1 : 0;
        p->bc = bc;
        p->tol = tol;
        plan_kappa_bounds(st, p->literal_n ? (double)Nx : (double)(Nx + 1),
                          p->literal_n ? (double)Ny : (double)(Ny + 1), &p->kmin, &p->kmax);
        if (!(p->kmin > 0.0 && p->kmin < p->kmax)) {
            free_plan(p);
            return CJ_ERR_INVALID_ARG;
        }
        p->c = plan_centre(st);
        p->S = plan_abs_coeff_sum(st);
        double h = 1.0 / (double)(Nx + 1);
        p->h2 = h * h;
        p->M = plan_cycle_length(p->kmin, p->kmax, tol);
        if (p->M > (1LL << 24)) {
            free_plan(p);
            return CJ_ERR_INVALID_ARG;
        }
        p->method = o.method;
        if (p->method == CJ_JACOBI)
            p->w.assign((size_t)p->M, 1.0 / p->c);  // omega = 1: w = 1/c at every sweep
        else
            plan_sweep_coeffs(st, p->kmin, p->kmax, p->M, p->w);
        p->M_in = 0;
        if (p->precision == CJ_FP64_INNER_DD) {
            p->M_in = o.inner_cycle ? o.inner_cycle : plan_inner_cycle_fp64(p->kmin, p->kmax, p->M, tol);
            plan_sweep_coeffs(st, p->kmin, p->kmax, p->M_in, p->w_in);
        } else if (p->precision != CJ_FP64) {
            p->M_in = o.inner_cycle ? o.inner_cycle : plan_inner_cycle(p->kmin, p->kmax, p->M);
            std::vector<double> wi;
            plan_sweep_coeffs(st, p->kmin, p->kmax, p->M_in, wi);
            p->w32.resize(p->M_in);
            for (long long k = 0; k < p->M_in; ++k) p->w32[k] = (float)wi[k];
        }
        // default FP32 temporal depth, from measurements (cj_sweeps_f32, Gupd/s at depth 1 / 4):
        // 9-point 63 / 57 at 512^2, 179 / 226 at 1024^2, 510 / 545 at 2048^2, 480 / 1211 at
        // 4096^2, 539 / 1493 at 8192^2; 5-point 16 / 18 at 256^2, 63 / 72 at 512^2 and 481 / 1413
        // at 4096^2; 17-point depth 1 / 2: 382 / 356 at 4096^2, 422 / 408 at 8192^2.
        // cj_autotune_depth records a measured choice per size class, which takes precedence.
        const int tuned = tuned_depth(st, Nx, Ny);
        const long long nodes = (long long)Nx * Ny;
        const int dflt = (st == 5 && nodes >= (1LL << 16)) || (st == 9 && nodes >= (1LL << 20)) ? 4 : 1;
        p->depth = o.temporal_depth ? o.temporal_depth : tuned ? tuned : dflt;
        long long unit = p->precision != CJ_FP64 ? p->M_in : p->M;
        p->max_sweeps = o.max_sweeps ? o.max_sweeps : 64 * unit;
        if (p->method == CJ_JACOBI && !o.max_sweeps) {
            // Jacobi's lowest mode falls by 1 - kmin per sweep: ln(1/tol)/kmin sweeps, x 4
            const double need = 4.0 * std::log(1.0 / tol) / p->kmin;
            if (need > (double)p->max_sweeps)
                p->max_sweeps = need < 9e15 ? (long long)need : (1LL << 53);
        }
    } catch (...) {
        free_plan(p);
        return CJ_ERR_NOMEM;
    }
    cudaError_t e = cudaGetDevice(&p->device);
    if (e != cudaSuccess) {
        set_cuda_error(e, "cudaGetDevice");
        free_plan(p);
        return CJ_ERR_CUDA;
    }
    p->g64 = make_grid(Nx, Ny, 8);
    p->g32 = make_grid(Nx, Ny, 4);
    p->m64 = plan_march(Nx, Ny, st, true);
    p->m32 = plan_march(Nx, Ny, st, false);
    long long copy_parts = (long long)((Nx + kBX - 1) / kBX) * (Ny < 1024 ? Ny : 1024);
    long long parts = p->m64.blocks();
    if (copy_parts > parts) parts = copy_parts;
    p->max_parts = (int)parts;
    const size_t n64 = (size_t)p->g64.elems(), n32 = (size_t)p->g32.elems();
    e = dev_alloc(&p->u0, n64);
    if (e == cudaSuccess) e = dev_alloc(&p->b, n64);
    if (e == cudaSuccess && p->precision != CJ_FP32_INNER) e = dev_alloc(&p->u1, n64);
    if (e == cudaSuccess && p->precision == CJ_FP64_INNER_DD) {
        e = dev_alloc(&p->d0, n64);
        if (e == cudaSuccess) e = dev_alloc(&p->d1, n64);
        if (e == cudaSuccess) e = dev_alloc(&p->r64, n64);
    } else if (e == cudaSuccess && p->precision != CJ_FP64) {
        e = dev_alloc(&p->e0, n32);
        if (e == cudaSuccess) e = dev_alloc(&p->e1, n32);
        if (e == cudaSuccess) e = dev_alloc(&p->rt, n32);
    }
    if (e == cudaSuccess) e = dev_alloc(&p->partials, (size_t)3 * parts);
    if (e == cudaSuccess) e = dev_alloc(&p->red, 8);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&p->h_red, 8 * sizeof(double));
    if (e == cudaSuccess) e = cudaEventCreate(&p->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&p->ev1);
    const bool graph = p->precision == CJ_FP64 && p->M % 2 == 0 &&
                       (o.launch == 2 || (o.launch == 0 && sweep_graph_wanted(p)));
    if (e == cudaSuccess && graph) e = make_sweep_graph(p);
    if (e == cudaSuccess && (o.launch == 0 || o.launch == 3)) {
        p->cluster_C = cluster_solve_size(p);
        if (p->cluster_C > 0 && !p->w_dev) {
            e = cudaMalloc((void **)&p->w_dev, sizeof(double) * (size_t)p->M);
            if (e == cudaSuccess)
                e = cudaMemcpy(p->w_dev, p->w.data(), sizeof(double) * (size_t)p->M, cudaMemcpyHostToDevice);
        }
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        set_cuda_error(e, "plan allocation");
        free_plan(p);
        return e == cudaErrorMemoryAllocation ? CJ_ERR_NOMEM : CJ_ERR_CUDA;
    }
    if (o.launch == 3 && p->cluster_C == 0) {  // the cluster solve was asked for and does not fit
        set_error_text("cj_plan_create: launch 3 needs a plain FP64 plan of at most 2^14 nodes");
        free_plan(p);
        return CJ_ERR_INVALID_ARG;
    }
    *out = p;
    return CJ_OK;
}

cj_status cj_plan_create_mask(int Nx, int Ny, const cj_mask *m, double tol, const cj_options *opt,
                              cj_plan **out) {
    if (!out) return CJ_ERR_INVALID_ARG;
    *out = nullptr;
    if (!m || !m->coef) return CJ_ERR_INVALID_ARG;
    const int pat = m->pattern;
    if (pat != 5 && pat != 9 && pat != 17 && pat != 25) return CJ_ERR_INVALID_ARG;
    if (m->sx < 0 || m->sy < 0 || m->sp < 0 || m->scale_sx < 0 || m->scale_sy < 0) return CJ_ERR_INVALID_ARG;
    if (!(m->kmin > 0.0 && m->kmin < m->kmax) || !(m->kmax < 1e300)) return CJ_ERR_INVALID_ARG;
    cj_options o{};
    if (opt) o = *opt;
    if (o.precision != CJ_FP64 || o.literal_n != 0 || o.launch == 2) return CJ_ERR_INVALID_ARG;
    if (!(tol > 0.0 && tol < 1.0)) return CJ_ERR_INVALID_ARG;
    const long long M = plan_cycle_length(m->kmin, m->kmax, tol);
    if (M > (1LL << 24)) return CJ_ERR_INVALID_ARG;
    // the padded buffers, reductions and ring of a Dirichlet-data FP64 plan of the same size
    // (its stencil only picks the launch shape), with one launch per sweep
    cj_options base = o;
    base.launch = 1;
    const cj_stencil shape = pat == 5 ? CJ_ST5 : pat == 9 ? CJ_ST9 : CJ_ST17;
    cj_plan *p = nullptr;
    cj_status st = cj_plan_create(Nx, Ny, shape, CJ_BC_DIRICHLET, tol, &base, &p);
    if (st != CJ_OK) return st;
    try {
        p->pattern = pat;
        p->kmin = m->kmin;
        p->kmax = m->kmax;
        p->c = 1.0;
        p->S = 2.0;
        p->M = M;
        if (p->method == CJ_JACOBI)
            p->w.assign((size_t)M, 1.0);
        else
            plan_sweep_coeffs_c(1.0, m->kmin, m->kmax, M, p->w);
        p->max_sweeps = o.max_sweeps ? o.max_sweeps : 64 * M;
        if (p->method == CJ_JACOBI && !o.max_sweeps) {
            const double need = 4.0 * std::log(1.0 / tol) / m->kmin;
            if (need > (double)p->max_sweeps) p->max_sweeps = need < 9e15 ? (long long)need : (1LL << 53);
        }
    } catch (...) {
        free_plan(p);
        return CJ_ERR_NOMEM;
    }
    int zero_centres = 0;
    cudaError_t e = mask_prepare(p, m->coef, m->sx, m->sy, m->sp, m->scale, m->scale_sx, m->scale_sy,
                                 &zero_centres);
    if (e != cudaSuccess) {
        set_cuda_error(e, "mask coefficients");
        free_plan(p);
        return e == cudaErrorMemoryAllocation ? CJ_ERR_NOMEM : CJ_ERR_CUDA;
    }
    if (zero_centres) {
        set_error_text("cj_plan_create_mask: a centre coefficient is 0");
        free_plan(p);
        return CJ_ERR_INVALID_ARG;
    }
    *out = p;
    return CJ_OK;
}

void cj_plan_destroy(cj_plan *plan) { free_plan(plan); }

cj_status cj_plan_weights(int Nx, int Ny, cj_stencil st, double tol, int literal_n, double *w, long long cap,
                          long long *M, double *kmin, double *kmax) {
    if (Nx < 1 || Ny < 1 || Nx > (1 << 20) || Ny > (1 << 20)) return CJ_ERR_INVALID_ARG;
    if (st != CJ_ST5 && st != CJ_ST9 && st != CJ_ST17) return CJ_ERR_INVALID_ARG;
    if (!(tol > 0.0 && tol < 1.0) || cap < 0) return CJ_ERR_INVALID_ARG;
    double a = 0.0, b = 0.0;
    plan_kappa_bounds(st, literal_n ? (double)Nx : (double)(Nx + 1), literal_n ? (double)Ny : (double)(Ny + 1), &a,
                      &b);
    if (!(a > 0.0 && a < b)) return CJ_ERR_INVALID_ARG;
    const long long m = plan_cycle_length(a, b, tol);
    if (m > (1LL << 24)) return CJ_ERR_INVALID_ARG;
    if (M) *M = m;
    if (kmin) *kmin = a;
    if (kmax) *kmax = b;
    if (!w) return CJ_OK;
    if (cap < m) return CJ_ERR_INVALID_ARG;
    try {
        std::vector<double> v;
        plan_sweep_coeffs(st, a, b, m, v);
        std::memcpy(w, v.data(), (size_t)m * sizeof(double));
    } catch (...) {
        return CJ_ERR_NOMEM;
    }
    return CJ_OK;
}

cj_status cj_plan_info(const cj_plan *p, const double **w, long long *M, double *kmin,
                       double *kmax, long long *M_inner) {
    if (!p) return CJ_ERR_INVALID_ARG;
    if (w) *w = p->w.data();
    if (M) *M = p->M;
    if (kmin) *kmin = p->kmin;
    if (kmax) *kmax = p->kmax;
    if (M_inner) *M_inner = p->M_in;
    return CJ_OK;
}

cj_status cj_solve(cj_plan *p, const double *f, long long ldf, double *u, long long ldu,
                   void *stream, cj_result *res) {
    cj_status a = check_grid_args(p, f, ldf, u, ldu);
    if (a != CJ_OK) return a;
    History h;
    return solve_core(p, f, ldf, u, ldu, (cudaStream_t)stream, res, &h);
}

cj_status cj_solve_history(cj_plan *p, const double *f, long long ldf, double *u, long long ldu,
                           void *stream, cj_result *res, double *history, int cap, int *count) {
    cj_status a = check_grid_args(p, f, ldf, u, ldu);
    if (a != CJ_OK) return a;
    if (cap < 0 || (cap > 0 && !history)) return CJ_ERR_INVALID_ARG;
    History h;
    h.buf = history;
    h.cap = cap;
    cj_status st = solve_core(p, f, ldf, u, ldu, (cudaStream_t)stream, res, &h);
    if (count) *count = h.n;
    return st;
}

cj_status cj_solve_to_error(cj_plan *p, const double *f, long long ldf, double *u, long long ldu,
                            const double *u_exact, long long ld_exact, double err_tol,
                            long long check_every, void *stream, cj_result *res, double *real_error,
                            double *history, int cap, int *count) {
    cj_status a = check_grid_args(p, f, ldf, u, ldu);
    if (a != CJ_OK) return a;
    if (!u_exact || ld_exact < p->Nx || !(err_tol >= 0.0) || check_every < 0 || cap < 0 ||
        (cap > 0 && !history) || p->method != CJ_CJM)
        return CJ_ERR_INVALID_ARG;
    // defect-correction plans test the real error at their outer steps
    if (p->precision != CJ_FP64 && check_every != 0) return CJ_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    auto t0 = std::chrono::steady_clock::now();
    cj_result r{};
    ErrorStop es{u_exact, ld_exact, err_tol, check_every, history, cap, 0};
    CJ_TRY(import64(p, f, ldf, u, ldu, s), "import");
    r.launches = 2;
    double *cur = nullptr;
    History h;
    cj_status st = p->precision == CJ_FP32_INNER      ? run_mixed(p, s, &cur, &r, &h, &es)
                   : p->precision == CJ_FP32_INNER_DD ? run_mixed_dd(p, s, &cur, &r, &h, &es)
                   : p->precision == CJ_FP64_INNER_DD ? run_fp64_dd(p, s, &cur, &r, &h, &es)
                                                      : run_fp64_to_error(p, s, &es, &cur, &r);
    if (count) *count = es.n;
    if (st < 0 && st != CJ_ERR_NOT_CONVERGED && st != CJ_ERR_DIVERGED) return st;
    CJ_TRY(launch_export(p, cur, u, ldu, s), "export");
    r.launches += 1;
    CJ_TRY(cudaStreamSynchronize(s), "solve sync");
    r.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (res) *res = r;
    if (real_error) *real_error = p->h_red[6];
    return st;
}

cj_status cj_solve_host(cj_plan *p, const double *f_host, double *u_host, void *stream,
                        cj_result *res) {
    if (!p || !f_host || !u_host) return CJ_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    auto t0 = std::chrono::steady_clock::now();
    const Grid &g = p->g64;
    double *b_in = p->b + g.idx(1, 1), *u_in = p->u0 + g.idx(1, 1);
    const size_t row = (size_t)p->Nx * sizeof(double), dpitch = (size_t)g.pitch * sizeof(double);
    CJ_TRY(cudaMemcpy2DAsync(b_in, dpitch, f_host, row, row, p->Ny, cudaMemcpyHostToDevice, s), "H2D f");
    CJ_TRY(cudaMemcpy2DAsync(u_in, dpitch, u_host, row, row, p->Ny, cudaMemcpyHostToDevice, s), "H2D u");
    cj_result r{};
    History h;
    // f and u now sit in the interiors of the plan's own buffers; the import runs in place.
    cj_status st = solve_core(p, b_in, g.pitch, u_in, g.pitch, s, &r, &h);
    if (st < 0 && st != CJ_ERR_NOT_CONVERGED && st != CJ_ERR_DIVERGED) return st;
    CJ_TRY(cudaMemcpy2DAsync(u_host, row, u_in, dpitch, row, p->Ny, cudaMemcpyDeviceToHost, s), "D2H u");
    CJ_TRY(cudaStreamSynchronize(s), "D2H sync");
    r.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (res) *res = r;
    return st;
}

cj_status cj_sweeps(cj_plan *p, const double *f, long long ldf, double *u, long long ldu,
                    long long first, long long count, void *stream) {
    cj_status a = check_grid_args(p, f, ldf, u, ldu);
    if (a != CJ_OK) return a;
    if (first < 0 || count < 0 || !p->u1) return CJ_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    CJ_TRY(import64(p, f, ldf, u, ldu, s), "import");
    double *cur = p->u0, *nxt = p->u1;
    for (long long k = 0; k < count; ++k) {
        CJ_TRY(sweep64(p, cur, nxt, p->w[(first + k) % p->M], s), "sweep");
        double *t = cur;
        cur = nxt;
        nxt = t;
    }
    CJ_TRY(launch_export(p, cur, u, ldu, s), "export");
    return CJ_OK;
}

cj_status cj_sweeps_ff(cj_plan *p, const double *f, long long ldf, double *u, long long ldu, long long first,
                       long long count, void *stream) {
    cj_status a = check_grid_args(p, f, ldf, u, ldu);
    if (a != CJ_OK) return a;
    if (first < 0 || count < 0 || !ff_sweeps_supported(p)) return CJ_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    CJ_TRY(import64(p, f, ldf, u, ldu, s), "import");
    const double *bufs[3] = {p->u0, p->u1, p->b};
    int cur = 0;
    CJ_TRY(launch_sweeps_ff(p, bufs, first, count, &cur, s), "sweep ff");
    CJ_TRY(launch_export(p, cur ? p->u1 : p->u0, u, ldu, s), "export");
    return CJ_OK;
}

cj_status cj_sweeps_f32(cj_plan *p, const float *r, long long ldr, float *e, long long lde,
                        long long first, long long count, void *stream) {
    cj_status a = check_grid_args(p, r, ldr, e, lde);
    if (a != CJ_OK) return a;
    if (first < 0 || count < 0 || !p->e0) return CJ_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    CJ_TRY(launch_import32(p, r, ldr, p->rt, s), "import32 r");
    CJ_TRY(launch_import32(p, e, lde, p->e0, s), "import32 e");
    float *cur = p->e0, *nxt = p->e1;
    long long launches = 0;
    CJ_TRY(fp32_sweeps(p, &cur, &nxt, p->rt, first, count, s, &launches), "sweep32");
    CJ_TRY(launch_export32(p, cur, e, lde, s), "export32");
    return CJ_OK;
}

cj_status cj_autotune_depth(int Nx, int Ny, cj_stencil st, int sweeps, void *stream,
                            int *best_depth, double *gupd) {
    if (Nx < 1 || Ny < 1 || sweeps < 8) return CJ_ERR_INVALID_ARG;
    if (st != CJ_ST5 && st != CJ_ST9 && st != CJ_ST17) return CJ_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int depths[4] = {1, 2, 4, 8};
    double rate[4] = {0, 0, 0, 0};
    int best = 1;
    cudaEvent_t e0, e1;
    CJ_TRY(cudaEventCreate(&e0), "autotune event");
    CJ_TRY(cudaEventCreate(&e1), "autotune event");
    for (int k = 0; k < 4; ++k) {
        cj_options o{};
        o.precision = CJ_FP32_INNER;
        o.inner_cycle = 64;
        o.temporal_depth = depths[k];
        cj_plan *p = nullptr;
        cj_status st2 = cj_plan_create(Nx, Ny, st, CJ_BC_DIRICHLET0, 1e-6, &o, &p);
        if (st2 != CJ_OK) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return st2;
        }
        float *cur = p->e0, *nxt = p->e1;
        long long launches = 0;
        cudaError_t err = fp32_sweeps(p, &cur, &nxt, p->rt, 0, 8, s, &launches);  // warm-up
        if (err == cudaSuccess) err = cudaEventRecord(e0, s);
        if (err == cudaSuccess) err = fp32_sweeps(p, &cur, &nxt, p->rt, 0, sweeps, s, &launches);
        if (err == cudaSuccess) err = cudaEventRecord(e1, s);
        if (err == cudaSuccess) err = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
        cj_plan_destroy(p);
        if (err != cudaSuccess) {
            set_cuda_error(err, "autotune");
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return CJ_ERR_CUDA;
        }
        rate[k] = (double)Nx * Ny * sweeps / (ms * 1e-3) / 1e9;
    }
    int kbest = 0;  // the fastest depth; the shallower one on a tie
    for (int k = 1; k < 4; ++k)
        if (rate[k] > rate[kbest]) kbest = k;
    best = depths[kbest];
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tuned_depth[stencil_slot(st)][size_class(Nx, Ny)] = best;
    }
    if (best_depth) *best_depth = best;
    if (gupd)
        for (int k = 0; k < 4; ++k) gupd[k] = rate[k];
    return CJ_OK;
}

cj_status cj_set_boundary(cj_plan *p, const double *g, long long ldg, void *stream) {
    if (!p || !g || p->bc != CJ_BC_DIRICHLET || ldg < p->Nx + 4) return CJ_ERR_INVALID_ARG;
    CJ_TRY(launch_set_ring(p, g, ldg, (cudaStream_t)stream), "boundary ring");
    return CJ_OK;
}

cj_status cj_solution_lo(cj_plan *p, double *u_lo, long long ld, void *stream) {
    if (!p || !u_lo || ld < p->Nx || (p->precision != CJ_FP32_INNER_DD && p->precision != CJ_FP64_INNER_DD))
        return CJ_ERR_INVALID_ARG;
    CJ_TRY(launch_export(p, p->u1, u_lo, ld, (cudaStream_t)stream), "export lo");
    return CJ_OK;
}

cj_status cj_residual(cj_plan *p, const double *f, long long ldf, const double *u,
                      long long ldu, void *stream, double *rel_l2, double *rel_inf,
                      double *floor_est) {
    cj_status a = check_grid_args(p, f, ldf, u, ldu);
    if (a != CJ_OK) return a;
    cudaStream_t s = (cudaStream_t)stream;
    CJ_TRY(import64(p, f, ldf, u, ldu, s), "import");
    CJ_TRY(residual64(p, p->u0, s), "residual");
    Norms n{};
    cj_status st = fetch_norms(p, s, &n);
    if (st != CJ_OK) return st;
    if (rel_l2) *rel_l2 = n.l2;
    if (rel_inf) *rel_inf = n.inf;
    if (floor_est) *floor_est = n.fl;
    return CJ_OK;
}

}  // extern "C"
