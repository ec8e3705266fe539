// Real error of Sec. 3.4 (Fig. 4 right): the distance of the iterate from the analytic solution
// of the test problem, max |u - u_exact| over the interior, for the real-error stop.
#include "cj_internal.h"
#include "grid_dev.cuh"

namespace {

// Per block: (sum d^2, max |d|, 0) of d = u - u_exact over its columns and a stride of rows;
// a NaN d makes the sum NaN, which the host reads as divergence.
__global__ void __launch_bounds__(kBX) error_kernel(const double *__restrict__ up, Grid g,
                                                    const double *__restrict__ ue, long long lde,
                                                    double *partials) {
    const int i = blockIdx.x * kBX + threadIdx.x + 1;
    double s = 0.0, m = 0.0;
    if (i <= g.Nx) {
        for (int j = blockIdx.y + 1; j <= g.Ny; j += gridDim.y) {
            const double d = up[g.idx(i, j)] - ue[(long long)(j - 1) * lde + (i - 1)];
            s = fma(d, d, s);
            m = fmax(m, fabs(d));
        }
    }
    block_reduce3(s, m, 0.0, partials);
}

}  // namespace

cudaError_t launch_real_error(const cj_plan *p, const double *u_pad, const double *ue, long long lde,
                              cudaStream_t s) {
    // the import's launch shape, for which p->partials is sized
    const dim3 grid((p->Nx + kBX - 1) / kBX, p->Ny < 1024 ? p->Ny : 1024);
    error_kernel<<<grid, kBX, 0, s>>>(u_pad, p->g64, ue, lde, p->partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_reduce(p->partials, (int)(grid.x * grid.y), p->red + 5, s);
}
