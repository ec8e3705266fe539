// Double-FP64 outer step of the mixed-precision Chebyshev-Jacobi solve (sm_103a).
//
// The solution is kept as the unevaluated sum u_hi + u_lo of two FP64 grids, and the
// defect R = L (u_hi + u_lo) - b is evaluated to about twice FP64 precision: multiplied by
// the stencil's denominator D (1, 6 or 72; Table 3, Eq. 1, Eq. 2), L u_hi - b becomes a sum
// of terms that are exact in FP64 (power-of-two multiples of u_hi and b), which are added
// by the error-free TwoSum cascade (Sum2 of Ogita, Rump and Oishi); D L u_lo is added in
// plain FP64.  This lifts the FP64 rounding floor of the relative residual (about
// 2^-53 S ||u|| / ||b||, 5e-10 for the 9-point stencil on 4096^2), so the FP32 inner
// cycles can drive the residual to 1e-10 and below.  Runs once per outer step, so it is a
// plain one-thread-per-node kernel; the term order is fixed and equals the reference's.
// The inner cycle's type T is float (FP32 inner cycles) or double (FP64 inner cycles, whose
// defect -R and correction e stay in FP64).
#include "cj_internal.h"
#include "grid_dev.cuh"
#include "stencil_dev.cuh"

namespace {

template <int ST, typename T>
__global__ void __launch_bounds__(kBX) defect_dd_kernel(const double *__restrict__ uh,
                                                        const double *__restrict__ ul,
                                                        const double *__restrict__ b, Grid g,
                                                        T *rt, T *ez, Grid gt,
                                                        double *partials) {
    const int i = blockIdx.x * kBX + threadIdx.x + 1;
    double s2 = 0.0, mx = 0.0, u2 = 0.0;
    if (i <= g.Nx) {
        for (int j = blockIdx.y + 1; j <= g.Ny; j += gridDim.y) {
            const double R = resid_dd<ST>(uh, ul, g, i, j, b[g.idx(i, j)]);
            const double uc = uh[g.idx(i, j)];
            s2 = fma(R, R, s2);
            mx = fmax(mx, fabs(R));
            u2 = fma(uc, uc, u2);
            rt[gt.idx(i, j)] = (T)(-R);
            store_node<(ST == 17 ? 2 : 1), T>(ez, gt, i, j, (T)0);
        }
    }
    block_reduce3(s2, mx, u2, partials);
}

template <int R, typename T>
__global__ void __launch_bounds__(kBX) correct_dd_kernel(double *uh, double *ul,
                                                         const T *__restrict__ e, Grid g,
                                                         Grid gt) {
    const int i = blockIdx.x * kBX + threadIdx.x + 1;
    if (i > g.Nx) return;
    for (int j = blockIdx.y + 1; j <= g.Ny; j += gridDim.y) {
        const long long k = g.idx(i, j);
        double hi, err, h2, l2;
        two_sum(uh[k], (double)e[gt.idx(i, j)], hi, err);
        const double lo = ul[k] + err;
        two_sum(hi, lo, h2, l2);
        store_node<R, double>(uh, g, i, j, h2);
        store_node<R, double>(ul, g, i, j, l2);
    }
}

inline dim3 node_grid(const Grid &g) {
    return dim3((g.Nx + kBX - 1) / kBX, g.Ny < 1024 ? g.Ny : 1024);
}

template <typename T>
cudaError_t defect_dd_any(const cj_plan *p, const double *uh, const double *ul, T *rt, T *e_zero,
                          const Grid &gt, cudaStream_t s) {
    const dim3 grid = node_grid(p->g64);
    switch (p->st) {
        case 5: defect_dd_kernel<5, T><<<grid, kBX, 0, s>>>(uh, ul, p->b, p->g64, rt, e_zero, gt, p->partials); break;
        case 9: defect_dd_kernel<9, T><<<grid, kBX, 0, s>>>(uh, ul, p->b, p->g64, rt, e_zero, gt, p->partials); break;
        default: defect_dd_kernel<17, T><<<grid, kBX, 0, s>>>(uh, ul, p->b, p->g64, rt, e_zero, gt, p->partials); break;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_reduce(p->partials, (int)(grid.x * grid.y), p->red, s);
}

template <typename T>
cudaError_t correct_dd_any(const cj_plan *p, double *uh, double *ul, const T *e, const Grid &gt,
                           cudaStream_t s) {
    if (p->r == 2 && p->bc == CJ_BC_DIRICHLET0)  // with Dirichlet data the ring stays as set
        correct_dd_kernel<2, T><<<node_grid(p->g64), kBX, 0, s>>>(uh, ul, e, p->g64, gt);
    else
        correct_dd_kernel<1, T><<<node_grid(p->g64), kBX, 0, s>>>(uh, ul, e, p->g64, gt);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_defect_dd(const cj_plan *p, const double *uh, const double *ul, float *rt,
                             float *e_zero, cudaStream_t s) {
    return defect_dd_any<float>(p, uh, ul, rt, e_zero, p->g32, s);
}

cudaError_t launch_correct_dd(const cj_plan *p, double *uh, double *ul, const float *e,
                              cudaStream_t s) {
    return correct_dd_any<float>(p, uh, ul, e, p->g32, s);
}

cudaError_t launch_defect_dd64(const cj_plan *p, const double *uh, const double *ul, double *r64,
                               double *e_zero, cudaStream_t s) {
    return defect_dd_any<double>(p, uh, ul, r64, e_zero, p->g64, s);
}

cudaError_t launch_correct_dd64(const cj_plan *p, double *uh, double *ul, const double *e,
                                cudaStream_t s) {
    return correct_dd_any<double>(p, uh, ul, e, p->g64, s);
}
