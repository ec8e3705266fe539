// Device arithmetic shared by the kernel translation units: the stencil evaluation in the
// fixed order of the FP64 reference (y-marching and direct forms), the double-FP64 defect,
// and the shared-memory stage of the temporal-blocked FP32 sweep.
#pragma once

#include "cj_internal.h"
#include "grid_dev.cuh"

namespace {

template <typename T>
struct Ar;
template <>
struct Ar<double> {
    static __device__ __forceinline__ double add(double a, double b, double one) {
        return fma(a, one, b);
    }
    static __device__ __forceinline__ double fm(double a, double b, double c) { return fma(a, b, c); }
};
template <>
struct Ar<float> {
    static __device__ __forceinline__ float add(float a, float b, float) { return a + b; }
    static __device__ __forceinline__ float fm(float a, float b, float c) { return fmaf(a, b, c); }
};

// Stencil coefficients of h^2 Delta_h (Table 3; Eq. 1 and Fig. 1 left; Eq. 2 and Fig. 1
// right), rounded once to the working type.
template <typename T>
struct Co;
template <>
struct Co<double> {
    static __device__ __forceinline__ double c5() { return -4.0; }
    static __device__ __forceinline__ double ax9() { return 4.0 / 6.0; }
    static __device__ __forceinline__ double dg9() { return 1.0 / 6.0; }
    static __device__ __forceinline__ double cc9() { return -20.0 / 6.0; }
    static __device__ __forceinline__ double a1() { return 64.0 / 72.0; }
    static __device__ __forceinline__ double a2() { return -4.0 / 72.0; }
    static __device__ __forceinline__ double d1() { return 16.0 / 72.0; }
    static __device__ __forceinline__ double d2() { return -1.0 / 72.0; }
    static __device__ __forceinline__ double cc17() { return -300.0 / 72.0; }
};
template <>
struct Co<float> {
    static __device__ __forceinline__ float c5() { return -4.0f; }
    static __device__ __forceinline__ float ax9() { return 4.0f / 6.0f; }
    static __device__ __forceinline__ float dg9() { return 1.0f / 6.0f; }
    static __device__ __forceinline__ float cc9() { return -20.0f / 6.0f; }
    static __device__ __forceinline__ float a1() { return 64.0f / 72.0f; }
    static __device__ __forceinline__ float a2() { return -4.0f / 72.0f; }
    static __device__ __forceinline__ float d1() { return 16.0f / 72.0f; }
    static __device__ __forceinline__ float d2() { return -1.0f / 72.0f; }
    static __device__ __forceinline__ float cc17() { return -300.0f / 72.0f; }
};

template <typename T>
__device__ __forceinline__ T ld(const T *p) {
    return __ldg(p);
}

// Walks rows j0..j1 of column i and calls op(j, r, u(i,j)) with r = (L u - b)(i, j).
template <int ST, typename T, class Op>
__device__ __forceinline__ void march(const T *__restrict__ u, const T *__restrict__ b,
                                      const Grid &g, int i, int j0, int j1, T one, Op &op) {
    using A = Ar<T>;
    using C = Co<T>;
    const long long P = g.pitch;
    const T *col = u + g.idx(i, 0);  // node (i, 0); row k at col + k * P
    const T *bcol = b + g.idx(i, 0);
    if (ST == 5) {
        T um = ld(col + (long long)(j0 - 1) * P);
        T uc = ld(col + (long long)j0 * P);
        for (int j = j0; j <= j1; ++j) {
            const T *row = col + (long long)j * P;
            T up = ld(row + P);
            T p0 = A::add(ld(row - 1), ld(row + 1), one);
            T v1 = A::add(um, up, one);
            T bk = ld(bcol + (long long)j * P);
            T a = A::add(p0, v1, one);
            T r = A::add(a, A::fm(C::c5(), uc, -bk), one);
            op(j, r, uc);
            um = uc;
            uc = up;
        }
    } else if (ST == 9) {
        const T *row = col + (long long)(j0 - 1) * P;
        T um = ld(row);
        T pm = A::add(ld(row - 1), ld(row + 1), one);
        row += P;
        T uc = ld(row);
        T pc = A::add(ld(row - 1), ld(row + 1), one);
        for (int j = j0; j <= j1; ++j) {
            row = col + (long long)(j + 1) * P;
            T up = ld(row);
            T pp = A::add(ld(row - 1), ld(row + 1), one);
            T bk = ld(bcol + (long long)j * P);
            T v1 = A::add(um, up, one);
            T a = A::add(pc, v1, one);
            T d = A::add(pm, pp, one);
            T r = A::fm(C::ax9(), a, A::fm(C::dg9(), d, A::fm(C::cc9(), uc, -bk)));
            op(j, r, uc);
            um = uc;
            uc = up;
            pm = pc;
            pc = pp;
        }
    } else {
        // rows j-2 .. j+1 in registers on entry to each iteration; row j+2 loaded in it
        T u_[4], p_[4], Q_[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const T *row = col + (long long)(j0 - 2 + k) * P;
            u_[k] = ld(row);
            p_[k] = A::add(ld(row - 1), ld(row + 1), one);
            Q_[k] = A::add(ld(row - 2), ld(row + 2), one);
        }
        for (int j = j0; j <= j1; ++j) {
            const T *row = col + (long long)(j + 2) * P;
            T u4 = ld(row);
            T p4 = A::add(ld(row - 1), ld(row + 1), one);
            T Q4 = A::add(ld(row - 2), ld(row + 2), one);
            T bk = ld(bcol + (long long)j * P);
            // u_[0..3] = rows j-2, j-1, j, j+1; u4 = row j+2
            T v1 = A::add(u_[1], u_[3], one);
            T v2 = A::add(u_[0], u4, one);
            T a1 = A::add(p_[2], v1, one);
            T a2 = A::add(Q_[2], v2, one);
            T d1 = A::add(p_[1], p_[3], one);
            T d2 = A::add(Q_[0], Q4, one);
            T r = A::fm(C::a1(), a1,
                        A::fm(C::a2(), a2,
                              A::fm(C::d1(), d1, A::fm(C::d2(), d2, A::fm(C::cc17(), u_[2], -bk)))));
            op(j, r, u_[2]);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                u_[k] = u_[k + 1];
                p_[k] = p_[k + 1];
                Q_[k] = Q_[k + 1];
            }
            u_[3] = u4;
            p_[3] = p4;
            Q_[3] = Q4;
        }
    }
}



// FP32 residual in second-difference form, L e - rk, from the horizontal and vertical second
// differences at spacing s, X_s(dy) = (e(s, dy) - e(0, dy)) - (e(0, dy) - e(-s, dy)) and
// Y_s = (e(0, s) - e_C) - (e_C - e(0, -s)): every value enters through a neighbour difference,
// so the smooth low modes keep their digits on fine grids where neighbour sums would cancel
// against the centre.  The forms are exact rewritings of the stencils: 5-point X_1(0) + Y_1;
// 9-point (Eq. 1) (X_1(-1) + X_1(1) + 4 X_1(0))/6 + Y_1 ([1 4 1; 4 -20 4; 1 4 1] is [1 4 1]
// across x times [1 4 1] across y, less 36 at the centre); 17-point (Eq. 2) 16/72 of the
// 9-point form times 6 less 1/72 of the same at spacing 2.  N(di, dj) returns the neighbour
// at offset (di, dj); the operation order is the FP32 reference's.
template <int ST, class F>
__device__ __forceinline__ float resid_diff32(F N, float uC, float rk) {
    auto X = [&](int sp, int dy) {
        const float c = N(0, dy);
        return (N(sp, dy) - c) - (c - N(-sp, dy));
    };
    const float Y1 = (N(0, 1) - uC) - (uC - N(0, -1));
    const float X1c = (N(1, 0) - uC) - (uC - N(-1, 0));
    if (ST == 5) return (X1c + Y1) - rk;
    const float X1s = X(1, -1) + X(1, 1);
    if (ST == 9) return fmaf(1.0f / 6.0f, X1s, fmaf(2.0f / 3.0f, X1c, Y1 - rk));
    const float Y2 = (N(0, 2) - uC) - (uC - N(0, -2));
    const float X2c = (N(2, 0) - uC) - (uC - N(-2, 0));
    const float X2s = X(2, -2) + X(2, 2);
    return fmaf(2.0f / 9.0f, X1s,
                fmaf(8.0f / 9.0f, X1c,
                     fmaf(4.0f / 3.0f, Y1,
                          fmaf(-1.0f / 72.0f, X2s, fmaf(-1.0f / 18.0f, X2c, fmaf(-1.0f / 12.0f, Y2, -rk))))));
}


// (L u - b)(i, j) evaluated directly from a node accessor U(di, dj), in the same order as
// march (so the two agree bit for bit).
template <int ST, typename T, class F>
__device__ __forceinline__ T resid_direct(F U, T bk) {
    const T uC = U(0, 0);
    const T v1 = U(0, -1) + U(0, 1);
    const T p0 = U(-1, 0) + U(1, 0);
    if (ST == 5) return (p0 + v1) + Ar<T>::fm(Co<T>::c5(), uC, -bk);
    const T pm = U(-1, -1) + U(1, -1);
    const T pp = U(-1, 1) + U(1, 1);
    if (ST == 9)
        return Ar<T>::fm(Co<T>::ax9(), p0 + v1,
                         Ar<T>::fm(Co<T>::dg9(), pm + pp, Ar<T>::fm(Co<T>::cc9(), uC, -bk)));
    const T v2 = U(0, -2) + U(0, 2);
    const T P0 = U(-2, 0) + U(2, 0);
    const T Pm = U(-2, -2) + U(2, -2);
    const T Pp = U(-2, 2) + U(2, 2);
    return Ar<T>::fm(Co<T>::a1(), p0 + v1,
                     Ar<T>::fm(Co<T>::a2(), P0 + v2,
                               Ar<T>::fm(Co<T>::d1(), pm + pp,
                                         Ar<T>::fm(Co<T>::d2(), Pm + Pp, Ar<T>::fm(Co<T>::cc17(), uC, -bk)))));
}

__device__ __forceinline__ void two_sum(double a, double b, double &s, double &e) {
    double x = a + b;
    double z = x - a;
    e = (a - (x - z)) + (b - z);
    s = x;
}

struct Sum2 {
    double S = 0.0, E = 0.0;
    __device__ __forceinline__ void add(double t) {
        double e;
        two_sum(S, t, S, e);
        E += e;
    }
};

// Plain FP64 L u at node (i, j) in the evaluation order of the sweep kernels (b = 0).
template <int ST>
__device__ __forceinline__ double plain_L(const double *u, const Grid &g, int i, int j) {
    auto U = [&](int di, int dj) { return u[g.idx(i + di, j + dj)]; };
    return resid_direct<ST, double>(U, 0.0);
}

// R = L (uh + ul) - bk at node (i, j), rounded to FP64 (term order as documented above).
template <int ST>
__device__ __forceinline__ double resid_dd(const double *uh, const double *ul, const Grid &g,
                                           int i, int j, double bk) {
    auto H = [&](int di, int dj) { return uh[g.idx(i + di, j + dj)]; };
    const double uC = H(0, 0);
    Sum2 s;
    double D;
    if (ST == 5) {
        D = 1.0;
        s.add(H(-1, 0));
        s.add(H(1, 0));
        s.add(H(0, -1));
        s.add(H(0, 1));
        s.add(-4.0 * uC);
        s.add(-bk);
    } else if (ST == 9) {
        D = 6.0;
        s.add(4.0 * H(-1, 0));
        s.add(4.0 * H(1, 0));
        s.add(4.0 * H(0, -1));
        s.add(4.0 * H(0, 1));
        s.add(H(-1, -1));
        s.add(H(1, -1));
        s.add(H(-1, 1));
        s.add(H(1, 1));
        s.add(-16.0 * uC);
        s.add(-4.0 * uC);
        s.add(-4.0 * bk);
        s.add(-2.0 * bk);
    } else {
        D = 72.0;
        s.add(64.0 * H(-1, 0));
        s.add(64.0 * H(1, 0));
        s.add(64.0 * H(0, -1));
        s.add(64.0 * H(0, 1));
        s.add(-4.0 * H(-2, 0));
        s.add(-4.0 * H(2, 0));
        s.add(-4.0 * H(0, -2));
        s.add(-4.0 * H(0, 2));
        s.add(16.0 * H(-1, -1));
        s.add(16.0 * H(1, -1));
        s.add(16.0 * H(-1, 1));
        s.add(16.0 * H(1, 1));
        s.add(-H(-2, -2));
        s.add(-H(2, -2));
        s.add(-H(-2, 2));
        s.add(-H(2, 2));
        s.add(-256.0 * uC);
        s.add(-32.0 * uC);
        s.add(-8.0 * uC);
        s.add(-4.0 * uC);
        s.add(-64.0 * bk);
        s.add(-8.0 * bk);
    }
    const double Llo = plain_L<ST>(ul, g, i, j);
    return (s.S + (s.E + D * Llo)) / D;
}

template <int ST>
__device__ __forceinline__ float resid_smem(const float *A, int SX, int x, int y, float rk) {
    auto N = [&](int dx, int dy) { return A[(y + dy) * SX + (x + dx)]; };
    return resid_diff32<ST>(N, A[y * SX + x], rk);
}

// One tile of the temporal-blocked FP32 sweep, run by the whole block: `depth` sweeps with
// weights w[0..depth-1] on the tile whose first interior node is (i0, j0), TX x TY nodes,
// staged with a halo of r * depth in shared memory `sm` (3 (TX+2H)(TY+2H) floats).  The
// caller owns the synchronisation before sm is reused.
template <int ST>
__device__ __forceinline__ void tb_tile(const float *__restrict__ e, const float *__restrict__ r,
                                        float *__restrict__ out, const Grid &g, int depth,
                                        const float *w, int i0, int j0, int TX, int TY, float *sm) {
    constexpr int R = ST == 17 ? 2 : 1;
    const int nt = blockDim.x;
    const int H = R * depth;
    const int SX = TX + 2 * H, SY = TY + 2 * H, NS = SX * SY;
    float *A = sm, *B = sm + NS, *Rs = sm + 2 * NS;
    // node (gx0 + x, gy0 + y) sits at staged cell (x, y)
    const int gx0 = i0 - H, gy0 = j0 - H;
    const int Nx = g.Nx, Ny = g.Ny;

    for (int c = threadIdx.x; c < NS; c += nt) {
        const int x = c % SX, y = c / SX, gi = gx0 + x, gj = gy0 + y;
        float a = 0.0f, q = 0.0f;
        if (gi >= -1 && gi <= Nx + 2 && gj >= -1 && gj <= Ny + 2) {
            const long long k = g.idx(gi, gj);
            a = __ldg(e + k);
            q = __ldg(r + k);
        }
        A[c] = a;
        B[c] = a;
        Rs[c] = q;
    }
    __syncthreads();

    for (int s = 1; s <= depth; ++s) {
        const float ws = w[s - 1];
        const int lo = R * s, wx = SX - 2 * lo, wy = SY - 2 * lo;
        for (int c = threadIdx.x; c < wx * wy; c += nt) {
            const int x = lo + c % wx, y = lo + c / wx, gi = gx0 + x, gj = gy0 + y;
            if (gi >= 1 && gi <= Nx && gj >= 1 && gj <= Ny) {
                const float uc = A[y * SX + x];
                B[y * SX + x] = fmaf(ws, resid_smem<ST>(A, SX, x, y, Rs[y * SX + x]), uc);
            }
        }
        __syncthreads();
        if (R == 2) {
            // outer ghost layer of the new values: odd reflection of the interior
            for (int c = threadIdx.x; c < wx * wy; c += nt) {
                const int x = lo + c % wx, y = lo + c / wx, gi = gx0 + x, gj = gy0 + y;
                const bool gx = gi == -1 || gi == Nx + 2, gy = gj == -1 || gj == Ny + 2;
                if (!(gx || gy)) continue;
                if (gi < -1 || gi > Nx + 2 || gj < -1 || gj > Ny + 2) continue;
                if (gi == 0 || gi == Nx + 1 || gj == 0 || gj == Ny + 1) continue;
                const int mx = gi == -1 ? x + 2 : gi == Nx + 2 ? x - 2 : x;
                const int my = gj == -1 ? y + 2 : gj == Ny + 2 ? y - 2 : y;
                const float v = B[my * SX + mx];
                B[y * SX + x] = (gx != gy) ? -v : v;
            }
            __syncthreads();
        }
        float *t = A;
        A = B;
        B = t;
    }

    for (int c = threadIdx.x; c < TX * TY; c += nt) {
        const int x = H + c % TX, y = H + c / TX, gi = gx0 + x, gj = gy0 + y;
        if (gi <= Nx && gj <= Ny) store_node<R, float>(out, g, gi, gj, A[y * SX + x]);
    }
}

}  // namespace
