// Position-dependent coefficient masks (Sec. 3.2): the generic stencil operator
//   (A u)(i, j) = sum over the pattern's offsets (dx, dy) of c_{dx,dy}(i, j) u(i+dx, j+dy)
// of up to 5 x 5 points, iterated in Jacobi-normalised form:
//   chat_k = c_k / c_C, bhat = f / (s c_C),
//   r = (u_C - bhat) + sum_k chat_k u_k   (off-centre offsets in row-major order, one fma each),
//   u' = u_C - w_n r.
// Patterns: 5 (cross), 9 (3 x 3 box), 17 (the points of Eq. 2), 25 (5 x 5 box).  The
// normalised planes keep the caller's broadcast layout (a plane that does not vary along an
// axis is stored once along it), so a polar mask (varying with r only) or a bipolar one
// (constant after normalisation) adds almost no HBM traffic to the sweep.  Nodes outside the
// interior are the plan's Dirichlet ring (zero, or set by cj_set_boundary).
//
// Bound: FP64 issue, K + 2 FP64 instructions per node for K off-centre points, plus the
// coefficient planes' bytes when they vary in both directions (8 K bytes per node).
#include "cj_internal.h"
#include "grid_dev.cuh"

namespace {

__host__ __device__ constexpr int mask_radius(int pat) { return pat == 5 || pat == 9 ? 1 : 2; }

// Whether offset (x, y) != (0, 0) belongs to the pattern.
__host__ __device__ constexpr bool in_mask(int pat, int x, int y) {
    const int ax = x < 0 ? -x : x, ay = y < 0 ? -y : y, m = ax > ay ? ax : ay;
    if (x == 0 && y == 0) return false;
    if (pat == 5) return ax + ay == 1;
    if (pat == 9) return m == 1;
    if (pat == 17) return m == 1 || (ax == 2 && ay == 0) || (ax == 0 && ay == 2) || (ax == 2 && ay == 2);
    return m <= 2;
}

struct Planes {
    const double *c;           // normalised off-centre planes
    long long sx, sy, sp;      // element strides (0 = repeated along that axis)
    __device__ __forceinline__ double at(int k, int i, int j) const {
        return __ldg(c + (long long)k * sp + (long long)(j - 1) * sy + (long long)(i - 1) * sx);
    }
};

// r = (D^-1 A u - bhat)(i, j) in the fixed order.
template <int PAT>
__device__ __forceinline__ double mask_resid(const double *__restrict__ u, const Grid &g, const Planes &pl,
                                             int i, int j, double bh, double uc, double one) {
    constexpr int R = mask_radius(PAT);
    double r = fma(uc, one, -bh);
    int k = 0;
#pragma unroll
    for (int y = -R; y <= R; ++y) {
#pragma unroll
        for (int x = -R; x <= R; ++x) {
            if (in_mask(PAT, x, y)) {
                r = fma(pl.at(k, i, j), __ldg(u + g.idx(i + x, j + y)), r);
                ++k;
            }
        }
    }
    return r;
}

template <int PAT>
__global__ void __launch_bounds__(kBX) mask_sweep_kernel(const double *__restrict__ u,
                                                         const double *__restrict__ bh,
                                                         double *__restrict__ out, Grid g, int ty,
                                                         Planes pl, double w, double one) {
    const int i = blockIdx.x * kBX + threadIdx.x + 1;
    const int j0 = blockIdx.y * ty + 1;
    const int j1 = min(j0 + ty - 1, g.Ny);
    if (i > g.Nx) return;
    for (int j = j0; j <= j1; ++j) {
        const long long c = g.idx(i, j);
        const double uc = __ldg(u + c);
        const double r = mask_resid<PAT>(u, g, pl, i, j, __ldg(bh + c), uc, one);
        out[c] = fma(-w, r, uc);
    }
}

// Per block (sum r^2, max |r|, sum u^2) of the normalised residual.
template <int PAT>
__global__ void __launch_bounds__(kBX) mask_resid_kernel(const double *__restrict__ u,
                                                         const double *__restrict__ bh, Grid g, int ty,
                                                         Planes pl, double *partials, double one) {
    const int i = blockIdx.x * kBX + threadIdx.x + 1;
    const int j0 = blockIdx.y * ty + 1;
    const int j1 = min(j0 + ty - 1, g.Ny);
    double s2 = 0.0, mx = 0.0, u2 = 0.0;
    if (i <= g.Nx) {
        for (int j = j0; j <= j1; ++j) {
            const long long c = g.idx(i, j);
            const double uc = __ldg(u + c);
            const double r = mask_resid<PAT>(u, g, pl, i, j, __ldg(bh + c), uc, one);
            s2 = fma(r, r, s2);
            mx = fmax(mx, fabs(r));
            u2 = fma(uc, uc, u2);
        }
    }
    block_reduce3(s2, mx, u2, partials);
}

// Caller grids -> padded bhat = f / dC and u; per block (sum bhat^2, max |bhat|, 0).
__global__ void __launch_bounds__(kBX) mask_import_kernel(const double *f, long long ldf,
                                                          const double *uin, long long ldu,
                                                          const double *__restrict__ dC, double *bh,
                                                          double *u, Grid g, double *partials) {
    const int i = blockIdx.x * kBX + threadIdx.x + 1;
    double s = 0.0, m = 0.0;
    if (i <= g.Nx) {
        for (int j = blockIdx.y + 1; j <= g.Ny; j += gridDim.y) {
            const double v = f[(long long)(j - 1) * ldf + (i - 1)] / dC[(long long)(j - 1) * g.Nx + (i - 1)];
            bh[g.idx(i, j)] = v;
            s = fma(v, v, s);
            m = fmax(m, fabs(v));
            u[g.idx(i, j)] = uin[(long long)(j - 1) * ldu + (i - 1)];
        }
    }
    block_reduce3(s, m, 0.0, partials);
}

// Normalised planes (in the caller's broadcast layout) and dC = s c_C (full); *bad counts
// zero centre coefficients.
__global__ void mask_normalize_kernel(const double *coef, long long sx, long long sy, long long sp,
                                      const double *scale, long long ssx, long long ssy, int K, int Nx,
                                      int Ny, int nx, int ny, double *chat, double *dC, int *bad) {
    const long long n = (long long)Nx * Ny, nst = (long long)nx * ny;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t % Nx) + 1, j = (int)(t / Nx) + 1;
        const long long at = (long long)(j - 1) * sy + (long long)(i - 1) * sx;
        const double cC = coef[at];
        if (cC == 0.0) atomicAdd(bad, 1);
        dC[t] = scale ? scale[(long long)(j - 1) * ssy + (long long)(i - 1) * ssx] * cC : cC;
        // the stored element of this node in the normalised layout, written by its first node
        const int si = nx == 1 ? 1 : i, sj = ny == 1 ? 1 : j;
        if (si == i && sj == j) {
            const long long e = (long long)(sj - 1) * nx + (si - 1);
            for (int k = 0; k < K; ++k) chat[(long long)k * nst + e] = coef[(long long)(k + 1) * sp + at] / cC;
        }
    }
}

inline dim3 mask_copy_grid(const Grid &g) {
    return dim3((g.Nx + kBX - 1) / kBX, g.Ny < 1024 ? g.Ny : 1024);
}

Planes planes_of(const cj_plan *p) {
    return Planes{p->chat, p->chat_sx, p->chat_sy, p->chat_sp};
}

}  // namespace

int mask_points(int pat) {
    int K = 0;
    const int R = mask_radius(pat);
    for (int y = -R; y <= R; ++y)
        for (int x = -R; x <= R; ++x) K += in_mask(pat, x, y) ? 1 : 0;
    return K;
}

cudaError_t mask_prepare(cj_plan *p, const double *coef, long long sx, long long sy, long long sp,
                         const double *scale, long long ssx, long long ssy, int *zero_centres) {
    const int K = mask_points(p->pattern);
    const int nx = sx ? p->Nx : 1, ny = sy ? p->Ny : 1;
    const long long nst = (long long)nx * ny;
    cudaError_t e = cudaMalloc((void **)&p->chat, sizeof(double) * (size_t)(K * nst));
    if (e == cudaSuccess) e = cudaMalloc((void **)&p->dC, sizeof(double) * (size_t)p->Nx * p->Ny);
    int *bad = nullptr;
    if (e == cudaSuccess) e = cudaMalloc((void **)&bad, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(bad, 0, sizeof(int));
    if (e != cudaSuccess) {
        cudaFree(bad);
        return e;
    }
    p->chat_sx = nx == 1 ? 0 : 1;
    p->chat_sy = ny == 1 ? 0 : nx;
    p->chat_sp = nst;
    const long long n = (long long)p->Nx * p->Ny;
    const int blocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
    mask_normalize_kernel<<<blocks, 256>>>(coef, sx, sy, sp, scale, ssx, ssy, K, p->Nx, p->Ny, nx, ny,
                                           p->chat, p->dC, bad);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpy(zero_centres, bad, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(bad);
    return e;
}

cudaError_t launch_mask_sweep(const cj_plan *p, const double *u, double *out, double w, cudaStream_t s) {
    const dim3 grid(p->m64.nbx, p->m64.nby);
    const Planes pl = planes_of(p);
    switch (p->pattern) {
        case 5: mask_sweep_kernel<5><<<grid, kBX, 0, s>>>(u, p->b, out, p->g64, p->m64.ty, pl, w, 1.0); break;
        case 9: mask_sweep_kernel<9><<<grid, kBX, 0, s>>>(u, p->b, out, p->g64, p->m64.ty, pl, w, 1.0); break;
        case 17: mask_sweep_kernel<17><<<grid, kBX, 0, s>>>(u, p->b, out, p->g64, p->m64.ty, pl, w, 1.0); break;
        default: mask_sweep_kernel<25><<<grid, kBX, 0, s>>>(u, p->b, out, p->g64, p->m64.ty, pl, w, 1.0); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_mask_residual(const cj_plan *p, const double *u, cudaStream_t s) {
    const dim3 grid(p->m64.nbx, p->m64.nby);
    const Planes pl = planes_of(p);
    switch (p->pattern) {
        case 5: mask_resid_kernel<5><<<grid, kBX, 0, s>>>(u, p->b, p->g64, p->m64.ty, pl, p->partials, 1.0); break;
        case 9: mask_resid_kernel<9><<<grid, kBX, 0, s>>>(u, p->b, p->g64, p->m64.ty, pl, p->partials, 1.0); break;
        case 17: mask_resid_kernel<17><<<grid, kBX, 0, s>>>(u, p->b, p->g64, p->m64.ty, pl, p->partials, 1.0); break;
        default: mask_resid_kernel<25><<<grid, kBX, 0, s>>>(u, p->b, p->g64, p->m64.ty, pl, p->partials, 1.0); break;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_reduce(p->partials, grid.x * grid.y, p->red, s);
}

cudaError_t launch_mask_import(const cj_plan *p, const double *f, long long ldf, const double *u,
                               long long ldu, cudaStream_t s) {
    const dim3 grid = mask_copy_grid(p->g64);
    mask_import_kernel<<<grid, kBX, 0, s>>>(f, ldf, u, ldu, p->dC, p->b, p->u0, p->g64, p->partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_reduce(p->partials, (int)(grid.x * grid.y), p->red + 3, s);
}
