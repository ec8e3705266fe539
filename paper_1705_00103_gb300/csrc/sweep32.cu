// One FP32 weighted sweep e' = e + w (L e - r) of the inner CJM cycles, in the difference form
// of the FP32 evaluation (resid_diff32): four adjacent columns per thread.
//
// The sweep moves 12 bytes per update (read e and r, write e') and does ~20 FP32 operations,
// so it is bound by HBM; what limits a one-column-per-thread march is the number of bytes in
// flight.  Here each thread loads the four columns of a row as one 16-byte vector (plus R
// scalar side columns on either side, which the neighbouring threads' vectors have just brought
// into L1), stores its four results as one vector, and issues the next row's loads before it
// computes the current row; a thread keeps the 2R+1 rows of its 4 + 2R columns in registers
// and walks down `ty` rows.  The grid is exactly one wave of resident blocks.
//
// Boundaries are those of the padded FP32 grids: nodes 0 and N+1 hold 0 and, for the 17-point
// stencil, the outer ghost layer holds the odd reflection, which store_node rewrites whenever a
// boundary-adjacent node changes.  Results equal the one-column march's bit for bit (same
// formula per node).
#include "cj_internal.h"
#include "grid_dev.cuh"
#include "stencil_dev.cuh"

namespace {

// Row y at columns c0-R .. c0+3+R into v[0 .. 3+2R]; columns past the padded row read as 0.
template <int R>
__device__ __forceinline__ void load_row4(const float *__restrict__ a, const Grid &g, int c0, int y, float *v) {
    const float *row = a + g.idx(c0, y);
    if (c0 + 3 <= g.Nx + 2) {
        const float4 q = __ldg(reinterpret_cast<const float4 *>(row));
        v[R] = q.x;
        v[R + 1] = q.y;
        v[R + 2] = q.z;
        v[R + 3] = q.w;
    } else {
#pragma unroll
        for (int m = 0; m < 4; ++m) v[R + m] = c0 + m <= g.Nx + 2 ? __ldg(row + m) : 0.0f;
    }
#pragma unroll
    for (int q = 1; q <= R; ++q) {
        v[R - q] = __ldg(row - q);  // column c0 - q >= -1
        v[R + 3 + q] = c0 + 3 + q <= g.Nx + 2 ? __ldg(row + 3 + q) : 0.0f;
    }
}

// r of row y at columns c0 .. c0+3.
__device__ __forceinline__ void load_r4(const float *__restrict__ a, const Grid &g, int c0, int y, float *v) {
    const float *row = a + g.idx(c0, y);
    if (c0 + 3 <= g.Nx + 2) {
        const float4 q = __ldg(reinterpret_cast<const float4 *>(row));
        v[0] = q.x;
        v[1] = q.y;
        v[2] = q.z;
        v[3] = q.w;
    } else {
#pragma unroll
        for (int m = 0; m < 4; ++m) v[m] = c0 + m <= g.Nx + 2 ? __ldg(row + m) : 0.0f;
    }
}

template <int ST>
__global__ void __launch_bounds__(kBX) sweep32_vec_kernel(const float *__restrict__ e, const float *__restrict__ r,
                                                          float *__restrict__ out, Grid g, int ty, float w) {
    constexpr int R = ST == 17 ? 2 : 1, W = 2 * R + 1, WC = 4 + 2 * R;
    const int c0 = ((int)blockIdx.x * kBX + (int)threadIdx.x) * 4 + 1;  // first of this thread's columns
    const int j0 = (int)blockIdx.y * ty + 1;
    const int j1 = min(j0 + ty - 1, g.Ny);
    if (c0 > g.Nx) return;
    // win[dy + R][dx + R]: row j + dy, column c0 + dx
    float win[W][WC];
#pragma unroll
    for (int dy = -R; dy < R; ++dy) load_row4<R>(e, g, c0, j0 + dy, win[dy + R + 1]);
    float nxt[WC], nb[4];
    load_row4<R>(e, g, c0, j0 + R, nxt);
    load_r4(r, g, c0, j0, nb);
    const bool full = c0 + 3 <= g.Nx;
#pragma unroll 1
    for (int j = j0; j <= j1; ++j) {
#pragma unroll
        for (int q = 0; q < W - 1; ++q)
#pragma unroll
            for (int c = 0; c < WC; ++c) win[q][c] = win[q + 1][c];
#pragma unroll
        for (int c = 0; c < WC; ++c) win[W - 1][c] = nxt[c];
        float bk[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) bk[m] = nb[m];
        if (j < j1) {  // the next row's loads go out before this row's arithmetic
            load_row4<R>(e, g, c0, j + R + 1, nxt);
            load_r4(r, g, c0, j + 1, nb);
        }
        float v[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            auto N = [&](int dx, int dy) { return win[R + dy][R + m + dx]; };
            const float uc = win[R][R + m];
            v[m] = fmaf(w, resid_diff32<ST>(N, uc, bk[m]), uc);
        }
        // the 17-point stencil's outer ghosts follow the nodes next to the boundary
        const bool edge = ST == 17 && (c0 == 1 || c0 + 3 >= g.Nx || j == 1 || j == g.Ny);
        if (full && !edge) {
            *reinterpret_cast<float4 *>(out + g.idx(c0, j)) = make_float4(v[0], v[1], v[2], v[3]);
        } else {
#pragma unroll
            for (int m = 0; m < 4; ++m)
                if (c0 + m <= g.Nx) store_node<R, float>(out, g, c0 + m, j, v[m]);
        }
    }
}

template <int ST>
cudaError_t launch_st(const Grid &g, const float *e, const float *r, float *out, float w, cudaStream_t s) {
    static int resident = 0;  // blocks of this kernel resident on the device at once
    if (resident == 0) {
        int dev = 0, sms = 152, per_sm = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep32_vec_kernel<ST>, kBX, 0) != cudaSuccess ||
            per_sm < 1)
            per_sm = 1;
        resident = sms * per_sm;
    }
    const int nbx = (g.Nx + 4 * kBX - 1) / (4 * kBX);
    long long nby = resident / nbx;
    if (nby < 1) nby = 1;
    if (nby > g.Ny) nby = g.Ny;
    int ty = (int)((g.Ny + nby - 1) / nby);
    constexpr int min_ty = ST == 17 ? 8 : 4;  // rows per block, against the 2R rows it re-reads
    if (ty < min_ty) ty = min_ty < g.Ny ? min_ty : g.Ny;
    const dim3 grid(nbx, (g.Ny + ty - 1) / ty);
    sweep32_vec_kernel<ST><<<grid, kBX, 0, s>>>(e, r, out, g, ty, w);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_sweep32(const cj_plan *p, const float *e, const float *r, float *out, float w,
                           cudaStream_t s) {
    switch (p->st) {
        case 5: return launch_st<5>(p->g32, e, r, out, w, s);
        case 9: return launch_st<9>(p->g32, e, r, out, w, s);
        default: return launch_st<17>(p->g32, e, r, out, w, s);
    }
}
