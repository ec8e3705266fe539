// Residual norms without any allocation: a variant of the plan-based residual (which keeps
// its block partial sums in device memory the plan allocated) for callers that cannot call
// cudaMalloc.  Typical such callers: code that runs inside a framework whose caching
// allocator has already reserved the device's memory, so a cudaMalloc of its own fails or
// fragments that pool; and latency-critical loops that cannot afford the implicit device
// synchronisation cudaMalloc and cudaFree may cause.
//
// The scratch is a file-scope device array of fixed size; every GPU that loads this library
// holds it until the process exits.  Host code cannot pass the array's name to a kernel
// (in host code the name is a host-side stand-in, not a device address), so the device
// address is looked up with cudaGetSymbolAddress, once per device, by the first call made
// with that device current, and reused afterwards.
#include <cmath>
#include <cstdio>
#include <mutex>

#include "cj_internal.h"
#include "grid_dev.cuh"

namespace {

constexpr int kNaRows = 64;           // rows per block (each block: 128 columns x 64 rows)
constexpr int kNaMaxBlocks = 16384;   // scratch capacity: one slot of 5 doubles per block
constexpr int kNaSlot = 5;            // sum r^2, max |r|, sum u^2, sum b^2, max |b|
constexpr int kNaMaxDevices = 64;

// 16384 x 5 doubles = 640 KiB per device.
static __device__ __align__(256) double g_na_scratch[kNaMaxBlocks * kNaSlot];

std::mutex g_na_mu;
double *g_na_addr[kNaMaxDevices] = {};

// Node (i, j) of a caller grid (interior only, row stride ld) with the homogeneous
// Dirichlet boundary and the odd reflection of the second ghost layer.
__device__ __forceinline__ double node(const double *u, long long ld, int Nx, int Ny, int i,
                                       int j) {
    if (i == 0 || i == Nx + 1 || j == 0 || j == Ny + 1) return 0.0;
    double s = 1.0;
    if (i == -1) { i = 1; s = -s; } else if (i == Nx + 2) { i = Nx; s = -s; }
    if (j == -1) { j = 1; s = -s; } else if (j == Ny + 2) { j = Ny; s = -s; }
    return s * u[(long long)(j - 1) * ld + (i - 1)];
}

// (L u - b)(i, j) in the evaluation order of the sweep kernels.
template <int ST>
__device__ __forceinline__ double resid_node(const double *u, long long ld, int Nx, int Ny,
                                             int i, int j, double bk) {
    auto U = [&](int di, int dj) { return node(u, ld, Nx, Ny, i + di, j + dj); };
    const double uC = U(0, 0);
    const double v1 = U(0, -1) + U(0, 1);
    const double p0 = U(-1, 0) + U(1, 0);
    if (ST == 5) return (p0 + v1) + fma(-4.0, uC, -bk);
    const double pm = U(-1, -1) + U(1, -1);
    const double pp = U(-1, 1) + U(1, 1);
    if (ST == 9) return fma(4.0 / 6.0, p0 + v1, fma(1.0 / 6.0, pm + pp, fma(-20.0 / 6.0, uC, -bk)));
    const double v2 = U(0, -2) + U(0, 2);
    const double P0 = U(-2, 0) + U(2, 0);
    const double Pm = U(-2, -2) + U(2, -2);
    const double Pp = U(-2, 2) + U(2, 2);
    return fma(64.0 / 72.0, p0 + v1,
               fma(-4.0 / 72.0, P0 + v2,
                   fma(16.0 / 72.0, pm + pp, fma(-1.0 / 72.0, Pm + Pp, fma(-300.0 / 72.0, uC, -bk)))));
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// max that keeps a NaN (fmax would drop it), so a non-finite residual shows in the L-inf norm too
__device__ __forceinline__ double max_nan(double a, double b) { return (a != a || a > b) ? a : b; }

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max_nan(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

// Block (bx, by) covers columns bx*128+1 .. and rows by*64+1 ..; its five statistics go to
// slot bx + by * gridDim.x of the scratch.
template <int ST>
__global__ void __launch_bounds__(kBX) na_partials(const double *__restrict__ f, long long ldf,
                                                   const double *__restrict__ u, long long ldu,
                                                   int Nx, int Ny, double h2, double *scratch) {
    const int i = blockIdx.x * kBX + threadIdx.x + 1;
    const int j0 = blockIdx.y * kNaRows + 1;
    const int j1 = min(j0 + kNaRows - 1, Ny);
    double v[kNaSlot] = {0.0, 0.0, 0.0, 0.0, 0.0};
    if (i <= Nx) {
        for (int j = j0; j <= j1; ++j) {
            const double bk = h2 * f[(long long)(j - 1) * ldf + (i - 1)];
            const double r = resid_node<ST>(u, ldu, Nx, Ny, i, j, bk);
            const double uc = u[(long long)(j - 1) * ldu + (i - 1)];
            v[0] = fma(r, r, v[0]);
            v[1] = max_nan(v[1], fabs(r));
            v[2] = fma(uc, uc, v[2]);
            v[3] = fma(bk, bk, v[3]);
            v[4] = max_nan(v[4], fabs(bk));
        }
    }
    __shared__ double sh[kBX / 32][kNaSlot];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < kNaSlot; ++k) {
        const double w = (k == 1 || k == 4) ? warp_max(v[k]) : warp_sum(v[k]);
        if (lane == 0) sh[wid][k] = w;
    }
    __syncthreads();
    if (threadIdx.x < kNaSlot) {
        const int k = threadIdx.x;
        double a = 0.0;
        for (int w = 0; w < kBX / 32; ++w) a = (k == 1 || k == 4) ? max_nan(a, sh[w][k]) : a + sh[w][k];
        scratch[(long long)(blockIdx.y * gridDim.x + blockIdx.x) * kNaSlot + k] = a;
    }
}

// One block: fixed-order reduction of nblk slots, then the relative norms into out[0..2].
__global__ void __launch_bounds__(256) na_finish(const double *__restrict__ scratch, int nblk,
                                                 double S, double *out) {
    __shared__ double sh[kNaSlot][256];
    double v[kNaSlot] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nblk; b += 256)
#pragma unroll
        for (int k = 0; k < kNaSlot; ++k) {
            const double x = scratch[(long long)b * kNaSlot + k];
            v[k] = (k == 1 || k == 4) ? max_nan(v[k], x) : v[k] + x;
        }
#pragma unroll
    for (int k = 0; k < kNaSlot; ++k) sh[k][threadIdx.x] = v[k];
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s)
#pragma unroll
            for (int k = 0; k < kNaSlot; ++k)
                sh[k][threadIdx.x] = (k == 1 || k == 4) ? max_nan(sh[k][threadIdx.x], sh[k][threadIdx.x + s])
                                                        : sh[k][threadIdx.x] + sh[k][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double rn = sqrt(sh[0][0]), un = sqrt(sh[2][0]), bn = sqrt(sh[3][0]), bmax = sh[4][0];
        const double eps = 1.1102230246251565e-16;
        out[0] = bn > 0.0 ? rn / bn : rn;
        out[1] = bmax > 0.0 ? sh[1][0] / bmax : sh[1][0];
        out[2] = bn > 0.0 ? eps * S * un / bn : eps * S * un;
    }
}

// Device address of the scratch array for the current device (looked up once per device).
cudaError_t scratch_address(double **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kNaMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_na_mu);
    if (!g_na_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_na_scratch);
        if (e != cudaSuccess) return e;
        g_na_addr[dev] = static_cast<double *>(p);
    }
    *out = g_na_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" cj_status cj_residual_noalloc(int Nx, int Ny, cj_stencil st, const double *f,
                                         long long ld_f, const double *u, long long ld_u,
                                         double *out, void *stream) {
    // sides up to 2^20 nodes, as for cj_plan_create; the block counts are formed in 64 bits
    if (Nx < 1 || Ny < 1 || Nx > (1 << 20) || Ny > (1 << 20) || !f || !u || !out || ld_f < Nx ||
        ld_u < Nx)
        return CJ_ERR_INVALID_ARG;
    if (st != CJ_ST5 && st != CJ_ST9 && st != CJ_ST17) return CJ_ERR_INVALID_ARG;
    const long long bx = ((long long)Nx + kBX - 1) / kBX, by = ((long long)Ny + kNaRows - 1) / kNaRows;
    if (bx * by > kNaMaxBlocks) {
        char msg[256];
        std::snprintf(msg, sizeof(msg),
                      "cj_residual_noalloc: a %d x %d grid needs %lld scratch slots, the limit is %d "
                      "(at most %d nodes)", Nx, Ny, bx * by, kNaMaxBlocks, kNaMaxBlocks * kBX * kNaRows);
        set_error_text(msg);
        return CJ_ERR_INVALID_ARG;
    }
    double *scratch = nullptr;
    cudaError_t e = scratch_address(&scratch);
    if (e != cudaSuccess) {
        set_cuda_error(e, "cj_residual_noalloc: scratch address");
        return CJ_ERR_CUDA;
    }
    const double h = 1.0 / ((double)Nx + 1.0);
    const double h2 = h * h;
    cudaStream_t s = (cudaStream_t)stream;
    const dim3 grid((unsigned)bx, (unsigned)by);
    switch (st) {
        case CJ_ST5: na_partials<5><<<grid, kBX, 0, s>>>(f, ld_f, u, ld_u, Nx, Ny, h2, scratch); break;
        case CJ_ST9: na_partials<9><<<grid, kBX, 0, s>>>(f, ld_f, u, ld_u, Nx, Ny, h2, scratch); break;
        default: na_partials<17><<<grid, kBX, 0, s>>>(f, ld_f, u, ld_u, Nx, Ny, h2, scratch); break;
    }
    e = cudaGetLastError();
    if (e == cudaSuccess) {
        na_finish<<<1, 256, 0, s>>>(scratch, (int)(bx * by), plan_abs_coeff_sum(st), out);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        set_cuda_error(e, "cj_residual_noalloc: launch");
        return CJ_ERR_CUDA;
    }
    return CJ_OK;
}
