// Subdomain kernels of the 2-D domain decomposition (one grid split into blocks across
// ranks).  The paper runs one grid on one GPU (Sec. 3.2); these two kernels are what a rank
// needs to take part in a decomposed CJM solve: the weighted sweep of Sec. 2.1 and the
// residual statistics, both on a box of nodes inside the caller's extended array, whose
// neighbours (the halo the ranks exchange, or the physical boundary) are read from the array
// itself.  The evaluation order is the sweep kernels' (resid_direct), so a decomposed solve
// gives the same bits at every node as the undecomposed one.
//
// One thread per node: a subdomain solve is bound by its halo exchanges, not by these loops.
#include <cstdio>

#include "cj_internal.h"
#include "grid_dev.cuh"
#include "stencil_dev.cuh"

namespace {

constexpr int kBoxTX = 32, kBoxTY = 8;

// edges: bit 0 the box's first column is the global column 1, bit 1 its last is the global
// column Nx, bit 2 its first row is the global row 1, bit 3 its last is the global row Ny; for
// a radius-2 stencil the odd-reflection ghosts beyond those sides are written with each node.
template <int ST>
__global__ void __launch_bounds__(kBoxTX *kBoxTY)
    box_sweep_kernel(const double *__restrict__ u, long long ldu, const double *__restrict__ b,
                     long long ldb, double *__restrict__ out, long long ldo, int nx, int ny, double w,
                     int edges) {
    const int i = blockIdx.x * kBoxTX + threadIdx.x;
    const int j = blockIdx.y * kBoxTY + threadIdx.y;
    if (i >= nx || j >= ny) return;
    auto U = [&](int di, int dj) { return u[(long long)(j + dj) * ldu + (i + di)]; };
    const double v = fma(w, resid_direct<ST, double>(U, b[(long long)j * ldb + i]), U(0, 0));
    out[(long long)j * ldo + i] = v;
    if (ST == 17) {  // as store_node: a one-node-wide box may touch both sides
        const bool L = (edges & 1) && i == 0, Rt = (edges & 2) && i == nx - 1;
        const bool B = (edges & 4) && j == 0, T = (edges & 8) && j == ny - 1;
        if (L) out[(long long)j * ldo - 2] = -v;
        if (Rt) out[(long long)j * ldo + i + 2] = -v;
        if (B) {
            out[-2 * ldo + i] = -v;
            if (L) out[-2 * ldo - 2] = v;
            if (Rt) out[-2 * ldo + i + 2] = v;
        }
        if (T) {
            out[(long long)(j + 2) * ldo + i] = -v;
            if (L) out[(long long)(j + 2) * ldo - 2] = v;
            if (Rt) out[(long long)(j + 2) * ldo + i + 2] = v;
        }
    }
}

template <int ST>
__global__ void __launch_bounds__(kBoxTX *kBoxTY)
    box_residual_kernel(const double *__restrict__ u, long long ldu, const double *__restrict__ b,
                        long long ldb, int nx, int ny, double *partials) {
    __shared__ double sh[kBoxTX * kBoxTY][5];
    const int i = blockIdx.x * kBoxTX + threadIdx.x;
    const int j = blockIdx.y * kBoxTY + threadIdx.y;
    const int t = threadIdx.y * kBoxTX + threadIdx.x;
    double s[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    if (i < nx && j < ny) {
        auto U = [&](int di, int dj) { return u[(long long)(j + dj) * ldu + (i + di)]; };
        const double bk = b[(long long)j * ldb + i];
        const double r = resid_direct<ST, double>(U, bk);
        const double uc = U(0, 0);
        s[0] = r * r;
        s[1] = fabs(r);
        s[2] = uc * uc;
        s[3] = bk * bk;
        s[4] = fabs(bk);
    }
#pragma unroll
    for (int k = 0; k < 5; ++k) sh[t][k] = s[k];
    __syncthreads();
    for (int h = kBoxTX * kBoxTY / 2; h > 0; h >>= 1) {
        if (t < h)
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                const double a = sh[t][k], c = sh[t + h][k];
                // the maxima keep a NaN (a non-finite residual must not vanish from the L-inf norm)
                sh[t][k] = (k == 1 || k == 4) ? ((a != a || a > c) ? a : c) : a + c;
            }
        __syncthreads();
    }
    if (t < 5) partials[((long long)blockIdx.y * gridDim.x + blockIdx.x) * 5 + t] = sh[0][t];
}

// One block: fixed-order reduction of nblk slots of 5 into out[0..4].
__global__ void __launch_bounds__(256) box_finish_kernel(const double *__restrict__ partials, long long nblk,
                                                         double *out) {
    __shared__ double sh[256][5];
    double v[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (long long k = threadIdx.x; k < nblk; k += 256)
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            const double x = partials[k * 5 + q];
            v[q] = (q == 1 || q == 4) ? ((v[q] != v[q] || v[q] > x) ? v[q] : x) : v[q] + x;
        }
#pragma unroll
    for (int q = 0; q < 5; ++q) sh[threadIdx.x][q] = v[q];
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h)
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                const double a = sh[threadIdx.x][q], c = sh[threadIdx.x + h][q];
                sh[threadIdx.x][q] = (q == 1 || q == 4) ? ((a != a || a > c) ? a : c) : a + c;
            }
        __syncthreads();
    }
    if (threadIdx.x < 5) out[threadIdx.x] = sh[0][threadIdx.x];
}

__global__ void __launch_bounds__(kBoxTX *kBoxTY)
    box_scale_kernel(const double *__restrict__ src, long long lds, double *__restrict__ dst, long long ldd, int nx,
                     int ny, double alpha) {
    const int i = blockIdx.x * kBoxTX + threadIdx.x;
    const int j = blockIdx.y * kBoxTY + threadIdx.y;
    if (i < nx && j < ny) dst[(long long)j * ldd + i] = alpha * src[(long long)j * lds + i];
}

dim3 box_grid(int nx, int ny) { return dim3((nx + kBoxTX - 1) / kBoxTX, (ny + kBoxTY - 1) / kBoxTY); }

bool box_args_ok(int nx, int ny, int st, const void *u, long long ldu, const void *b, long long ldb) {
    return nx >= 1 && ny >= 1 && nx <= (1 << 20) && ny <= (1 << 20) && u && b && ldu >= nx && ldb >= nx &&
           (st == 5 || st == 9 || st == 17);
}

}  // namespace

extern "C" long long cj_box_residual_slots(int nx, int ny) {
    if (nx < 1 || ny < 1) return 0;
    const dim3 g = box_grid(nx, ny);
    return (long long)g.x * g.y * 5;
}

extern "C" cj_status cj_box_sweep(int nx, int ny, cj_stencil st, double w, const double *u, long long ldu,
                                  const double *b, long long ldb, double *out, long long ldo, int edges,
                                  void *stream) {
    if (!box_args_ok(nx, ny, st, u, ldu, b, ldb) || !out || ldo != ldu || out == u || edges < 0 ||
        edges > 15)
        return CJ_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const dim3 grid = box_grid(nx, ny), block(kBoxTX, kBoxTY);
    switch (st) {
        case CJ_ST5: box_sweep_kernel<5><<<grid, block, 0, s>>>(u, ldu, b, ldb, out, ldo, nx, ny, w, edges); break;
        case CJ_ST9: box_sweep_kernel<9><<<grid, block, 0, s>>>(u, ldu, b, ldb, out, ldo, nx, ny, w, edges); break;
        default: box_sweep_kernel<17><<<grid, block, 0, s>>>(u, ldu, b, ldb, out, ldo, nx, ny, w, edges); break;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_cuda_error(e, "cj_box_sweep");
        return CJ_ERR_CUDA;
    }
    return CJ_OK;
}

extern "C" cj_status cj_box_residual(int nx, int ny, cj_stencil st, const double *u, long long ldu,
                                     const double *b, long long ldb, double *scratch, long long scratch_len,
                                     double *out, void *stream) {
    if (!box_args_ok(nx, ny, st, u, ldu, b, ldb) || !scratch || !out ||
        scratch_len < cj_box_residual_slots(nx, ny))
        return CJ_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const dim3 grid = box_grid(nx, ny), block(kBoxTX, kBoxTY);
    switch (st) {
        case CJ_ST5: box_residual_kernel<5><<<grid, block, 0, s>>>(u, ldu, b, ldb, nx, ny, scratch); break;
        case CJ_ST9: box_residual_kernel<9><<<grid, block, 0, s>>>(u, ldu, b, ldb, nx, ny, scratch); break;
        default: box_residual_kernel<17><<<grid, block, 0, s>>>(u, ldu, b, ldb, nx, ny, scratch); break;
    }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        box_finish_kernel<<<1, 256, 0, s>>>(scratch, (long long)grid.x * grid.y, out);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        set_cuda_error(e, "cj_box_residual");
        return CJ_ERR_CUDA;
    }
    return CJ_OK;
}

extern "C" cj_status cj_box_scale(int nx, int ny, double alpha, const double *src, long long lds, double *dst,
                                  long long ldd, void *stream) {
    if (nx < 1 || ny < 1 || nx > (1 << 20) || ny > (1 << 20) || !src || !dst || lds < nx || ldd < nx)
        return CJ_ERR_INVALID_ARG;
    box_scale_kernel<<<box_grid(nx, ny), dim3(kBoxTX, kBoxTY), 0, (cudaStream_t)stream>>>(src, lds, dst, ldd, nx, ny,
                                                                                          alpha);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_cuda_error(e, "cj_box_scale");
        return CJ_ERR_CUDA;
    }
    return CJ_OK;
}
