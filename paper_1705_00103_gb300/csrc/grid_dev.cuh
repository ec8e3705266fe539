// Device helpers shared by the kernel translation units: writing an interior node
// together with the odd-reflection ghost values that mirror it, and the block reduction
// of the residual statistics.
#pragma once

#include "cj_internal.h"

// Writes v at interior node (i, j) and, for a radius-2 stencil, the odd-reflection ghost
// values that mirror it (u[-1] = -u[1], u[N+2] = -u[N], corners +u).
template <int R, typename T>
__device__ __forceinline__ void store_node(T *out, const Grid &g, int i, int j, T v) {
    out[g.idx(i, j)] = v;
    if (R == 2) {
        const T nv = -v;
        if (i == 1) out[g.idx(-1, j)] = nv;
        if (i == g.Nx) out[g.idx(g.Nx + 2, j)] = nv;
        if (j == 1) {
            out[g.idx(i, -1)] = nv;
            if (i == 1) out[g.idx(-1, -1)] = v;
            if (i == g.Nx) out[g.idx(g.Nx + 2, -1)] = v;
        }
        if (j == g.Ny) {
            out[g.idx(i, g.Ny + 2)] = nv;
            if (i == 1) out[g.idx(-1, g.Ny + 2)] = v;
            if (i == g.Nx) out[g.idx(g.Nx + 2, g.Ny + 2)] = v;
        }
    }
}


// Block reduction of (sum, max, sum) into partials[3 * block].
__device__ __forceinline__ void block_reduce3(double a, double m, double c, double *partials) {
    __shared__ double sh[kBX / 32][3];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
        c += __shfl_down_sync(0xffffffffu, c, o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        sh[wid][0] = a;
        sh[wid][1] = m;
        sh[wid][2] = c;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double A = 0.0, Mx = 0.0, Cc = 0.0;
        for (int k = 0; k < kBX / 32; ++k) {
            A += sh[k][0];
            Mx = fmax(Mx, sh[k][1]);
            Cc += sh[k][2];
        }
        const long long blk = (long long)blockIdx.y * gridDim.x + blockIdx.x;
        partials[3 * blk + 0] = A;
        partials[3 * blk + 1] = Mx;
        partials[3 * blk + 2] = Cc;
    }
}

