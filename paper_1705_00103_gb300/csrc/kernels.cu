// Device kernels of the Chebyshev-Jacobi solver for sm_103a.
//
// Hot kernel: the weighted sweep u' = u + w_n (L u - b) of Sec. 2.1 for the 5-point
// (Table 3), 9-point (Eq. 1) and 17-point (Eq. 2) Laplacians.  A stencil is not a dense
// contraction, so there are no tensor cores here.  On GB300 the FP64 pipe issues about
// two FMAs per SM clock (~0.6 T instructions/s; FP32 issues ~60x more), so the FP64 sweep
// is bound by FP64 instruction issue, not by HBM: the kernels below evaluate L u - b in
// the fewest FP64 instructions, and every FP64 addition is issued as fma(a, one, b)
// (bit-identical to a + b; the FMA path has the higher issue rate on this part).
//
// Evaluation order of L u - b (fixed, shared by design with the FP64 reference):
//   horizontal pair sums p(k) = u(i-1,k) + u(i+1,k), P(k) = u(i-2,k) + u(i+2,k);
//   vertical pairs v1 = u(i,j-1) + u(i,j+1), v2 = u(i,j-2) + u(i,j+2);
//   5-pt : (p(j) + v1) + fma(-4, u, -b)
//   9-pt : fma(4/6, p(j) + v1, fma(1/6, p(j-1) + p(j+1), fma(-20/6, u, -b)))
//   17-pt: fma(64/72, p(j)+v1, fma(-4/72, P(j)+v2, fma(16/72, p(j-1)+p(j+1),
//              fma(-1/72, P(j-2)+P(j+2), fma(-300/72, u, -b)))))
// Each thread owns one column i and walks down `ty` rows, keeping u(i, .), p and P of the
// rows around j in registers, so every p and P is formed once and reused by the three
// (five) rows that need it.
//
// Compiled with --fmad=false: no multiply-add is contracted behind the code's back.
#include <cstdint>

#include "cj_internal.h"
#include "grid_dev.cuh"
#include "stencil_dev.cuh"

namespace {

// Stores the updated node; for the 17-point stencil with MIRROR also its reflection ghosts
// (without MIRROR the ghost ring holds fixed Dirichlet data).
template <int ST, typename T, bool MIRROR = true>
struct SweepOp {
    T *out;
    const Grid *g;
    int i;
    T w;
    __device__ __forceinline__ void operator()(int j, T r, T uc) {
        store_node<((ST == 17 && MIRROR) ? 2 : 1)>(out, *g, i, j, Ar<T>::fm(w, r, uc));
    }
};

// One FP64 weighted sweep: out = u + w (L u - b) in the pair-sum order above (the FP32 inner
// sweep, in difference form, is sweep32.cu's).
// MIRROR: rewrite the odd-reflection ghosts of the 17-point stencil (homogeneous boundary);
// without it the ghost ring holds fixed Dirichlet data and is left alone.
template <int ST, typename T, bool MIRROR = true>
__global__ void __launch_bounds__(kBX) sweep_kernel(const T *__restrict__ u,
                                                    const T *__restrict__ b, T *__restrict__ out,
                                                    Grid g, int ty, T w, T one) {
    const int i = blockIdx.x * kBX + threadIdx.x + 1;
    const int j0 = blockIdx.y * ty + 1;
    const int j1 = min(j0 + ty - 1, g.Ny);
    if (i > g.Nx) return;
    SweepOp<ST, T, MIRROR> op{out, &g, i, w};
    march<ST, T>(u, b, g, i, j0, j1, one, op);
}

struct ResidOp {
    double s2 = 0.0, mx = 0.0, u2 = 0.0;
    float *rt = nullptr, *ez = nullptr;
    const Grid *g32 = nullptr;
    int i = 0;
    int r2 = 0;
    __device__ __forceinline__ void operator()(int j, double r, double uc) {
        s2 = fma(r, r, s2);
        mx = fmax(mx, fabs(r));
        u2 = fma(uc, uc, u2);
        if (rt) {
            rt[g32->idx(i, j)] = (float)(-r);
            if (r2)
                store_node<2, float>(ez, *g32, i, j, 0.0f);
            else
                ez[g32->idx(i, j)] = 0.0f;
        }
    }
};

// Residual of u against b; with rt != nullptr also the defect rt = (float)(b - L u) and
// zeroes the FP32 correction buffer ez (the defect step of the mixed-precision solve).
template <int ST>
__global__ void __launch_bounds__(kBX) resid_kernel(const double *__restrict__ u,
                                                    const double *__restrict__ b, Grid g, int ty,
                                                    double *partials, float *rt, float *ez,
                                                    Grid g32, double one) {
    const int i = blockIdx.x * kBX + threadIdx.x + 1;
    const int j0 = blockIdx.y * ty + 1;
    const int j1 = min(j0 + ty - 1, g.Ny);
    ResidOp op;
    op.rt = rt;
    op.ez = ez;
    op.g32 = &g32;
    op.i = i;
    op.r2 = (ST == 17);
    if (i <= g.Nx) march<ST, double>(u, b, g, i, j0, j1, one, op);
    block_reduce3(op.s2, op.mx, op.u2, partials);
}

// Fixed-order reduction of nparts partial triples into out[0..2] (deterministic).
__global__ void __launch_bounds__(256) reduce_kernel(const double *__restrict__ partials,
                                                     int nparts, double *out) {
    __shared__ double sa[256], sm[256], sc[256];
    double a = 0.0, m = 0.0, c = 0.0;
    for (int k = threadIdx.x; k < nparts; k += 256) {
        a += partials[3 * k + 0];
        m = fmax(m, partials[3 * k + 1]);
        c += partials[3 * k + 2];
    }
    sa[threadIdx.x] = a;
    sm[threadIdx.x] = m;
    sc[threadIdx.x] = c;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            sa[threadIdx.x] += sa[threadIdx.x + s];
            sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + s]);
            sc[threadIdx.x] += sc[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = sa[0];
        out[1] = sm[0];
        out[2] = sc[0];
    }
}

// Caller grids (interior, row stride ld) -> padded b = h^2 f and padded u with its
// reflection ghosts; partial (sum b^2, max |b|, 0) per block.
template <int R>
__global__ void __launch_bounds__(kBX) import_kernel(const double *f, long long ldf,
                                                     const double *uin, long long ldu,
                                                     double *b, double *u, Grid g, double h2,
                                                     double *partials) {
    const int i = blockIdx.x * kBX + threadIdx.x + 1;
    double s = 0.0, m = 0.0;
    if (i <= g.Nx) {
        for (int j = blockIdx.y + 1; j <= g.Ny; j += gridDim.y) {
            double fk = f[(long long)(j - 1) * ldf + (i - 1)];
            double bk = h2 * fk;
            b[g.idx(i, j)] = bk;
            s = fma(bk, bk, s);
            m = fmax(m, fabs(bk));
            store_node<R, double>(u, g, i, j, uin[(long long)(j - 1) * ldu + (i - 1)]);
        }
    }
    block_reduce3(s, m, 0.0, partials);
}

__global__ void __launch_bounds__(kBX) export_kernel(const double *__restrict__ up, Grid g,
                                                     double *u, long long ldu) {
    const int i = blockIdx.x * kBX + threadIdx.x + 1;
    if (i > g.Nx) return;
    for (int j = blockIdx.y + 1; j <= g.Ny; j += gridDim.y)
        u[(long long)(j - 1) * ldu + (i - 1)] = up[g.idx(i, j)];
}

template <int R>
__global__ void __launch_bounds__(kBX) correct_kernel(double *u, const float *__restrict__ e,
                                                      Grid g, Grid g32, double one) {
    const int i = blockIdx.x * kBX + threadIdx.x + 1;
    if (i > g.Nx) return;
    for (int j = blockIdx.y + 1; j <= g.Ny; j += gridDim.y) {
        double v = fma(u[g.idx(i, j)], one, (double)e[g32.idx(i, j)]);
        store_node<R, double>(u, g, i, j, v);
    }
}

template <int R>
__global__ void __launch_bounds__(kBX) import32_kernel(const float *src, long long ld, float *dst,
                                                       Grid g) {
    const int i = blockIdx.x * kBX + threadIdx.x + 1;
    if (i > g.Nx) return;
    for (int j = blockIdx.y + 1; j <= g.Ny; j += gridDim.y)
        store_node<R, float>(dst, g, i, j, src[(long long)(j - 1) * ld + (i - 1)]);
}

__global__ void __launch_bounds__(kBX) export32_kernel(const float *__restrict__ src, Grid g,
                                                       float *dst, long long ld) {
    const int i = blockIdx.x * kBX + threadIdx.x + 1;
    if (i > g.Nx) return;
    for (int j = blockIdx.y + 1; j <= g.Ny; j += gridDim.y)
        dst[(long long)(j - 1) * ld + (i - 1)] = src[g.idx(i, j)];
}

}  // namespace

cudaError_t launch_reduce(const double *partials, int nparts, double *out, cudaStream_t s) {
    reduce_kernel<<<1, 256, 0, s>>>(partials, nparts, out);
    return cudaGetLastError();
}

namespace {

inline dim3 copy_grid(const Grid &g) {
    int nbx = (g.Nx + kBX - 1) / kBX;
    int nby = g.Ny < 1024 ? g.Ny : 1024;
    return dim3(nbx, nby);
}

// SMs of the current device, looked up once (thread-safe initialisation)
int num_sms() {
    static const int n = [] {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
            sms = 152;
        return sms;
    }();
    return n;
}

}  // namespace

Grid make_grid(int Nx, int Ny, int elem_bytes) {
    Grid g;
    g.Nx = Nx;
    g.Ny = Ny;
    g.padl = 128 / elem_bytes;
    long long per = 128 / elem_bytes;
    long long need = g.padl + Nx + 2;
    g.pitch = (need + per - 1) / per * per;
    return g;
}

March plan_march(int Nx, int Ny, int st, bool fp64) {
    // one wave of blocks: SMs x resident blocks, each block a 128-column strip of ty rows
    const int per_sm = fp64 ? 8 : 12;
    March m;
    m.nbx = (Nx + kBX - 1) / kBX;
    long long target = (long long)num_sms() * per_sm;
    long long nby = target / m.nbx;
    if (nby < 1) nby = 1;
    if (nby > Ny) nby = Ny;
    int min_ty = st == 17 ? 8 : 4;
    m.ty = (int)((Ny + nby - 1) / nby);
    if (m.ty < min_ty) m.ty = min_ty < Ny ? min_ty : Ny;
    m.nby = (Ny + m.ty - 1) / m.ty;
    (void)st;
    return m;
}

cudaError_t launch_sweep64(const cj_plan *p, const double *u, double *out, double w,
                           cudaStream_t s) {
    dim3 grid(p->m64.nbx, p->m64.nby);
    switch (p->st) {
        case 5: sweep_kernel<5, double><<<grid, kBX, 0, s>>>(u, p->b, out, p->g64, p->m64.ty, w, 1.0); break;
        case 9: sweep_kernel<9, double><<<grid, kBX, 0, s>>>(u, p->b, out, p->g64, p->m64.ty, w, 1.0); break;
        default:
            if (p->bc == CJ_BC_DIRICHLET)
                sweep_kernel<17, double, false><<<grid, kBX, 0, s>>>(u, p->b, out, p->g64, p->m64.ty, w, 1.0);
            else
                sweep_kernel<17, double><<<grid, kBX, 0, s>>>(u, p->b, out, p->g64, p->m64.ty, w, 1.0);
            break;
    }
    return cudaGetLastError();
}

cudaError_t launch_sweep64_err(const cj_plan *p, const double *e, const double *rhs, double *out,
                               double w, cudaStream_t s) {
    dim3 grid(p->m64.nbx, p->m64.nby);
    switch (p->st) {
        case 5: sweep_kernel<5, double><<<grid, kBX, 0, s>>>(e, rhs, out, p->g64, p->m64.ty, w, 1.0); break;
        case 9: sweep_kernel<9, double><<<grid, kBX, 0, s>>>(e, rhs, out, p->g64, p->m64.ty, w, 1.0); break;
        default: sweep_kernel<17, double><<<grid, kBX, 0, s>>>(e, rhs, out, p->g64, p->m64.ty, w, 1.0); break;
    }
    return cudaGetLastError();
}

// Dirichlet data g (node (i, j) at g[(j+1) ldg + i+1], i, j in -1..N+2) into the ghost ring of
// both FP64 solution buffers.
__global__ void __launch_bounds__(256) ring_kernel(const double *__restrict__ gdat, long long ldg,
                                                  double *u0, double *u1, Grid g) {
    const long long W = g.Nx + 4, H = g.Ny + 4;
    for (long long k = blockIdx.x * 256LL + threadIdx.x; k < W * H; k += (long long)gridDim.x * 256) {
        const int i = (int)(k % W) - 1, j = (int)(k / W) - 1;
        if (i >= 1 && i <= g.Nx && j >= 1 && j <= g.Ny) continue;
        const double v = gdat[(long long)(j + 1) * ldg + (i + 1)];
        u0[g.idx(i, j)] = v;
        if (u1) u1[g.idx(i, j)] = v;
    }
}

cudaError_t launch_set_ring(const cj_plan *p, const double *gdat, long long ldg, cudaStream_t s) {
    const long long cells = (long long)(p->Nx + 4) * (p->Ny + 4);
    const int blocks = (int)((cells + 255) / 256 < 4096 ? (cells + 255) / 256 : 4096);
    ring_kernel<<<blocks, 256, 0, s>>>(gdat, ldg, p->u0, p->u1, p->g64);
    return cudaGetLastError();
}


cudaError_t launch_residual(const cj_plan *p, const double *u_pad, float *rt, float *e_zero,
                            cudaStream_t s) {
    dim3 grid(p->m64.nbx, p->m64.nby);
    switch (p->st) {
        case 5: resid_kernel<5><<<grid, kBX, 0, s>>>(u_pad, p->b, p->g64, p->m64.ty, p->partials, rt, e_zero, p->g32, 1.0); break;
        case 9: resid_kernel<9><<<grid, kBX, 0, s>>>(u_pad, p->b, p->g64, p->m64.ty, p->partials, rt, e_zero, p->g32, 1.0); break;
        default: resid_kernel<17><<<grid, kBX, 0, s>>>(u_pad, p->b, p->g64, p->m64.ty, p->partials, rt, e_zero, p->g32, 1.0); break;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    reduce_kernel<<<1, 256, 0, s>>>(p->partials, p->m64.blocks(), p->red);
    return cudaGetLastError();
}

cudaError_t launch_import(const cj_plan *p, const double *f, long long ldf, const double *u,
                          long long ldu, double *b_out, double *u_out, cudaStream_t s) {
    dim3 grid = copy_grid(p->g64);
    if (p->r == 2 && p->bc == CJ_BC_DIRICHLET0)
        import_kernel<2><<<grid, kBX, 0, s>>>(f, ldf, u, ldu, b_out, u_out, p->g64, p->h2, p->partials);
    else
        import_kernel<1><<<grid, kBX, 0, s>>>(f, ldf, u, ldu, b_out, u_out, p->g64, p->h2, p->partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    reduce_kernel<<<1, 256, 0, s>>>(p->partials, (int)(grid.x * grid.y), p->red + 3);
    return cudaGetLastError();
}

cudaError_t launch_export(const cj_plan *p, const double *u_pad, double *u, long long ldu,
                          cudaStream_t s) {
    export_kernel<<<copy_grid(p->g64), kBX, 0, s>>>(u_pad, p->g64, u, ldu);
    return cudaGetLastError();
}

cudaError_t launch_correct(const cj_plan *p, double *u_pad, const float *e, cudaStream_t s) {
    if (p->r == 2 && p->bc == CJ_BC_DIRICHLET0)  // with Dirichlet data the ring stays as set
        correct_kernel<2><<<copy_grid(p->g64), kBX, 0, s>>>(u_pad, e, p->g64, p->g32, 1.0);
    else
        correct_kernel<1><<<copy_grid(p->g64), kBX, 0, s>>>(u_pad, e, p->g64, p->g32, 1.0);
    return cudaGetLastError();
}

cudaError_t launch_import32(const cj_plan *p, const float *src, long long ld, float *dst_pad,
                            cudaStream_t s) {
    if (p->r == 2)
        import32_kernel<2><<<copy_grid(p->g32), kBX, 0, s>>>(src, ld, dst_pad, p->g32);
    else
        import32_kernel<1><<<copy_grid(p->g32), kBX, 0, s>>>(src, ld, dst_pad, p->g32);
    return cudaGetLastError();
}

cudaError_t launch_export32(const cj_plan *p, const float *src_pad, float *dst, long long ld,
                            cudaStream_t s) {
    export32_kernel<<<copy_grid(p->g32), kBX, 0, s>>>(src_pad, p->g32, dst, ld);
    return cudaGetLastError();
}
