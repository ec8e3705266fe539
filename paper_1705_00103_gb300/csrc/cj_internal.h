// Internal declarations of libcj: plan object, padded grid layout, kernel launchers.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "cj.h"

// Padded device layout of one grid (FP64 or FP32).  Rows j = -1 .. Ny+2 (two ghost rows
// each side), columns i = -1 .. Nx+2.  The interior column i = 1 starts `padl` elements
// into the row, with padl * sizeof(T) = 128 bytes, and the row pitch is a multiple of
// 128 bytes, so every interior row starts on a 128-byte boundary.  Nodes 0 and N+1 hold
// the Dirichlet value 0 for the whole life of the buffer; the outer ghost layer (-1, N+2)
// holds the odd reflection of the interior, rewritten by every kernel that writes the
// interior (needed by the 17-point stencil only).
struct Grid {
    int Nx, Ny;
    int padl;        // elements before column i = 1
    long long pitch; // elements per row
    __host__ __device__ long long idx(int i, int j) const {
        return (long long)(j + 1) * pitch + (padl - 1) + i;
    }
    __host__ __device__ long long elems() const { return pitch * (long long)(Ny + 4); }
};

Grid make_grid(int Nx, int Ny, int elem_bytes);

// Launch shape of the y-marching kernels: blocks of kBX threads, one column each, every
// block walks `ty` consecutive rows.
constexpr int kBX = 128;
// Deepest temporal blocking of the FP32 inner sweep (sweeps per HBM round trip).
constexpr int kTbMaxDepth = 8;
struct March {
    int nbx, nby, ty;
    int blocks() const { return nbx * nby; }
};

struct cj_plan {
    int Nx, Ny, st, r, precision, literal_n, bc;
    int method = 0;           // cj_method: CJ_CJM or CJ_JACOBI (every w_n = 1/c)
    double tol, kmin, kmax, c, S, h2;
    long long M, M_in, max_sweeps;
    int depth = 1;            // FP32 sweeps per launch (temporal blocking depth)
    std::vector<double> w;    // sweep coefficients w_n = omega_n / c, application order
    std::vector<float> w32;   // FP32 inner cycle coefficients
    std::vector<double> w_in; // FP64 inner cycle coefficients (CJ_FP64_INNER_DD)
    int device;
    Grid g64, g32;
    March m64, m32;
    double *u0 = nullptr, *u1 = nullptr, *b = nullptr;    // padded FP64
    float *e0 = nullptr, *e1 = nullptr, *rt = nullptr;    // padded FP32 (mixed only)
    double *d0 = nullptr, *d1 = nullptr, *r64 = nullptr;  // padded FP64 correction ping-pong and
                                                          // defect (CJ_FP64_INNER_DD only)
    double *partials = nullptr;                           // 3 doubles per block
    double *red = nullptr;                                // 8 reduced doubles
    double *h_red = nullptr;                              // pinned copy of red
    int max_parts = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;             // brackets of a cycle's sweeps
    // FP64 cycle as a CUDA graph (small grids, graph.cu): device weight table, table position,
    // the instantiated graph of graph_G sweeps + position advance
    double *w_dev = nullptr;
    long long *pos = nullptr;
    cudaGraphExec_t graph = nullptr;
    int graph_G = 0;
    // whole solves in one thread-block cluster (cluster.cu): CTAs per cluster (0 = not used)
    int cluster_C = 0;
    // coefficient-mask plans (mask.cu): pattern 5/9/17/25 (0 = one of the paper's stencils),
    // normalised off-centre planes with their element strides, and dC = s c_C (full)
    int pattern = 0;
    double *chat = nullptr;
    long long chat_sx = 0, chat_sy = 0, chat_sp = 0;
    double *dC = nullptr;
};

// ---- plan math (plan.cpp)
double plan_centre(int st);
double plan_abs_coeff_sum(int st);
void plan_kappa_bounds(int st, double nint_x, double nint_y, double *kmin, double *kmax);
long long plan_cycle_length(double kmin, double kmax, double tol);
long long plan_inner_cycle(double kmin, double kmax, long long M);
long long plan_inner_cycle_fp64(double kmin, double kmax, long long M, double tol);
void plan_sweep_coeffs(int st, double kmin, double kmax, long long M, std::vector<double> &w);
// the same with the centre c given (c = 1: the weights omega_n of a Jacobi-normalised operator)
void plan_sweep_coeffs_c(double c, double kmin, double kmax, long long M, std::vector<double> &w);

// ---- autotuning tables (solve.cpp): stencil index 0/1/2 and size class floor(log4(Nx Ny))
int stencil_slot(int st);
int size_class(int Nx, int Ny);

// ---- error reporting (solve.cpp)
void set_cuda_error(cudaError_t e, const char *where);
void set_error_text(const char *msg);

// ---- coefficient masks (mask.cu)
int mask_points(int pattern);  // off-centre points K of a pattern
// normalised planes and dC from the caller's coefficients (synchronous); *zero_centres
// receives the number of nodes whose centre coefficient is 0
cudaError_t mask_prepare(cj_plan *p, const double *coef, long long sx, long long sy, long long sp,
                         const double *scale, long long ssx, long long ssy, int *zero_centres);
cudaError_t launch_mask_sweep(const cj_plan *p, const double *u, double *out, double w, cudaStream_t s);
// red[0..2] = (sum r^2, max |r|, sum u^2) of the normalised residual
cudaError_t launch_mask_residual(const cj_plan *p, const double *u, cudaStream_t s);
// bhat = f / dC and u into the plan's buffers; red[3..4] = (sum bhat^2, max |bhat|)
cudaError_t launch_mask_import(const cj_plan *p, const double *f, long long ldf, const double *u,
                               long long ldu, cudaStream_t s);

// ---- FP64 cycles as CUDA graphs (graph.cu)
// true when the plan's grid is small enough for its sweeps to be bound by host launches
bool sweep_graph_wanted(const cj_plan *p);
// builds p->w_dev, p->pos and p->graph (call once, on the plan's device)
cudaError_t make_sweep_graph(cj_plan *p);
// one full cycle (p->M sweeps from u0, ending in u0) on stream s
cudaError_t launch_sweep_cycle_graph(const cj_plan *p, cudaStream_t s);

// ---- FP64-accuracy sweeps in float-float on the FP32 pipe (ff.cu)
// plain FP64 plans of the paper's stencils with the homogeneous boundary
bool ff_sweeps_supported(const cj_plan *p);
// bufs = {u0, u1, b} of the plan (imported); count sweeps from u0 with weights w[(first + k) mod M];
// the buffers are converted to float-float for the sweeps and back; *cur_out: 0 if the result is
// in u0, 1 if in u1
cudaError_t launch_sweeps_ff(const cj_plan *p, const double *const *bufs, long long first, long long count,
                             int *cur_out, cudaStream_t s);

// ---- whole small FP64 solves in one cluster (cluster.cu)
// CTAs of the cluster the plan's solve fits in (0: not eligible: not plain FP64 on the paper's
// stencils, more than 2^14 nodes, or no cluster launch on this device)
int cluster_solve_size(const cj_plan *p);
// the solve of p->u0 against p->b (imported, red[3..4] set) with the plan's weights table w_dev;
// res_dev[0..5] = status, sweeps, cycles, rho, rinf, fl
cudaError_t launch_cluster_solve(const cj_plan *p, double *res_dev, cudaStream_t s);

// ---- kernel launchers (kernels.cu); every launcher returns the launch error
March plan_march(int Nx, int Ny, int st, bool fp64);
// caller grids -> padded b = h^2 f and u; red[3..4] = (sum b^2, max |b|)
cudaError_t launch_import(const cj_plan *p, const double *f, long long ldf, const double *u,
                          long long ldu, double *b_out, double *u_out, cudaStream_t s);
// Dirichlet data into the ghost ring of both FP64 solution buffers (CJ_BC_DIRICHLET plans)
cudaError_t launch_set_ring(const cj_plan *p, const double *gdat, long long ldg, cudaStream_t s);
// real error of u_pad against the caller's u_exact: red[5..6] = (sum d^2, max |d|)
cudaError_t launch_real_error(const cj_plan *p, const double *u_pad, const double *ue, long long lde,
                              cudaStream_t s);
cudaError_t launch_export(const cj_plan *p, const double *u_pad, double *u, long long ldu,
                          cudaStream_t s);
cudaError_t launch_sweep64(const cj_plan *p, const double *u, double *out, double w,
                           cudaStream_t s);
// FP64 sweep of the error equation L e = rhs with the homogeneous boundary of the plan's stencil
// (odd reflection for 17 points whatever the plan's bc): the inner cycle of CJ_FP64_INNER_DD
cudaError_t launch_sweep64_err(const cj_plan *p, const double *e, const double *rhs, double *out,
                               double w, cudaStream_t s);
cudaError_t launch_sweep32(const cj_plan *p, const float *e, const float *r, float *out, float w,
                           cudaStream_t s);
// residual of u_pad against p->b: red[0..2] = (sum r^2, max|r|, sum u^2); with rt != NULL
// also writes rt = (float)(b - L u) and zeroes e_zero (the defect step of the mixed solve)
cudaError_t launch_residual(const cj_plan *p, const double *u_pad, float *rt, float *e_zero,
                            cudaStream_t s);
// fixed-order reduction of nparts (sum, max, sum) triples into out[0..2]
cudaError_t launch_reduce(const double *partials, int nparts, double *out, cudaStream_t s);
cudaError_t launch_correct(const cj_plan *p, double *u_pad, const float *e, cudaStream_t s);
// double-FP64 outer form (dd.cu): defect R = L (uh + ul) - b to about twice FP64
// precision -> rt = (float)(-R), e_zero = 0, red[0..2] = (sum R^2, max |R|, sum uh^2);
// and the correction (uh, ul) += e by TwoSum
cudaError_t launch_defect_dd(const cj_plan *p, const double *uh, const double *ul, float *rt,
                             float *e_zero, cudaStream_t s);
cudaError_t launch_correct_dd(const cj_plan *p, double *uh, double *ul, const float *e,
                              cudaStream_t s);
// the same two steps with an FP64 inner cycle: r64 = -R in FP64, e_zero (FP64) = 0; (uh, ul) += e
cudaError_t launch_defect_dd64(const cj_plan *p, const double *uh, const double *ul, double *r64,
                               double *e_zero, cudaStream_t s);
cudaError_t launch_correct_dd64(const cj_plan *p, double *uh, double *ul, const double *e,
                                cudaStream_t s);
// register wavefront temporal-blocked FP32 sweeps (wave_reg.cu): k = 2 sweeps per launch, or
// 3 or 4 for the 5- and 9-point stencils
int wave_reg_supported(int st, int k);
cudaError_t launch_sweep32_wave_reg(const cj_plan *p, const float *e, const float *r, float *out,
                                    const float *w, int k, cudaStream_t s);
// wavefront temporal-blocked FP32 sweeps (wave.cu): k in {2, 4, 8} sweeps per launch
int wave_depth_supported(int k);
cudaError_t launch_sweep32_wave(const cj_plan *p, const float *e, const float *r, float *out,
                                const float *w, int k, cudaStream_t s);
cudaError_t launch_import32(const cj_plan *p, const float *src, long long ld, float *dst_pad,
                            cudaStream_t s);
cudaError_t launch_export32(const cj_plan *p, const float *src_pad, float *dst, long long ld,
                            cudaStream_t s);
