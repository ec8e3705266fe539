// FP32 y-march over four adjacent columns per thread, in the difference form of the FP32
// evaluation (resid_diff32): the vectorised one-sweep stage shared by the single-problem
// FP32 sweep (sweep32.cu) and the batched engine's tiles (engine.cu).
//
// A thread keeps rows j-R .. j+R of columns c0-R .. c0+3+R in registers, loads each new row as
// one 16-byte vector of its own columns plus R scalar side columns on either side (which the
// neighbouring threads' vectors have just brought into L1), and issues the next row's loads
// before the current row's arithmetic.  Columns past the padded row (> Nx + 2) read as 0: they
// only feed results at columns > Nx, which are not stored.
#pragma once

#include "cj_internal.h"
#include "grid_dev.cuh"
#include "stencil_dev.cuh"

namespace {

// Row y at columns c0-R .. c0+3+R into v[0 .. 3+2R].
template <int R>
__device__ __forceinline__ void m4_load_row(const float *__restrict__ a, const Grid &g, int c0, int y, float *v) {
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
__device__ __forceinline__ void m4_load_r(const float *__restrict__ a, const Grid &g, int c0, int y, float *v) {
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

// Rows j0..j1 of columns c0..c0+3 (c0 - 1 a multiple of 4, c0 <= Nx): calls
// op(j, res, uc) with res[m] = (L e - r)(c0+m, j) and uc[m] = e(c0+m, j).
template <int ST, class Op>
__device__ __forceinline__ void march4(const float *__restrict__ e, const float *__restrict__ r, const Grid &g,
                                       int c0, int j0, int j1, Op &op) {
    constexpr int R = ST == 17 ? 2 : 1, W = 2 * R + 1, WC = 4 + 2 * R;
    // win[dy + R][dx + R]: row j + dy, column c0 + dx
    float win[W][WC];
#pragma unroll
    for (int dy = -R; dy < R; ++dy) m4_load_row<R>(e, g, c0, j0 + dy, win[dy + R + 1]);
    float nxt[WC], nb[4];
    m4_load_row<R>(e, g, c0, j0 + R, nxt);
    m4_load_r(r, g, c0, j0, nb);
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
            m4_load_row<R>(e, g, c0, j + R + 1, nxt);
            m4_load_r(r, g, c0, j + 1, nb);
        }
        float res[4], uc[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            auto N = [&](int dx, int dy) { return win[R + dy][R + m + dx]; };
            uc[m] = win[R][R + m];
            res[m] = resid_diff32<ST>(N, uc[m], bk[m]);
        }
        op(j, res, uc);
    }
}

// Stores e' = e + w res at columns c0..c0+3 (those <= Nx): one vector store, or node by node
// where the 17-point stencil's outer ghosts must follow a node next to the boundary.
template <int ST>
struct M4Store {
    float *out;
    const Grid *g;
    int c0;
    float w;
    __device__ __forceinline__ void operator()(int j, const float *res, const float *uc) {
        float v[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) v[m] = fmaf(w, res[m], uc[m]);
        const Grid &G = *g;
        const bool edge = ST == 17 && (c0 == 1 || c0 + 3 >= G.Nx || j == 1 || j == G.Ny);
        if (c0 + 3 <= G.Nx && !edge) {
            *reinterpret_cast<float4 *>(out + G.idx(c0, j)) = make_float4(v[0], v[1], v[2], v[3]);
        } else {
#pragma unroll
            for (int m = 0; m < 4; ++m)
                if (c0 + m <= G.Nx) store_node<(ST == 17 ? 2 : 1), float>(out, G, c0 + m, j, v[m]);
        }
    }
};

}  // namespace
