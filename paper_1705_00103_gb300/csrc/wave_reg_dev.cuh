// Register wavefront temporal blocking of the FP32 inner sweep: the per-warp stage (wr_run) shared
// by the single-grid kernel (wave_reg.cu) and the batched engine (engine.cu): K consecutive
// weighted sweeps e <- e + w_n (L e - r) per HBM round trip, each with its own weight, with
// no shared-memory exchange and no barrier.
//
// Every warp owns a strip of 128 staged columns (four adjacent columns per lane, loaded and
// stored as 16-byte vectors) and streams down a block of rows.  Each iteration brings in one
// input row and advances all K stages by one row: stage s computes row y_in - s (R + 1) from
// rows y - R .. y + R of stage s-1, which sit in a register ring of 2R + 2 rows per stage
// (the loop is unrolled by the ring length, so every ring index is a constant).  The one row
// of skew beyond the stencil radius makes the K stages of an iteration independent of one
// another (stage s never reads the row stage s-1 produces in the same iteration): all K are
// computed first, and their new rows then enter the rings together.  The R columns on either
// side of a lane's four come from the neighbouring lanes by warp shuffles when a row enters.
// A strip's two side lanes are garbage after K stages (H = R K <= 4 columns from the edge), so
// lanes 1 .. 30 (120 columns) are stored; strip 0 starts at column 1 and stores lanes 0 .. 30.
// In y, a row block's outputs need H input rows before and after it.
//
// Boundaries: in x, the lanes next to the Dirichlet columns keep them in registers at every
// stage (column 0 and Nx + 1 at 0; for the 17-point stencil column -1 at -u(1) and Nx + 2 at
// -u(Nx)), the values the homogeneous boundary gives; lanes past Nx are never read.  In y, the
// stages run on the odd extension of the grid (fold_dev.cuh): every operation of the sweep is
// an odd function of its inputs under round-to-nearest, so values on reflected rows stay the
// exact negatives of their mirrors.  Interior results equal one-sweep launches bit for bit;
// the residual is evaluated in difference form with resid_diff32's operation order.
//
// e and r arrive by cp.async, kWrAhead rows ahead, into lane-private shared-memory rings (each
// lane reads back only what it copied, so no synchronisation is needed); r(y) is needed by
// every stage at a different iteration and stays in its ring for 16 rows.
//
// HBM traffic per update: about (8 B in + 4 B out) / K, plus the strip's 8-column and the row
// block's 2H-row overlap with its neighbours.
#pragma once

#include <type_traits>

#include "cj_internal.h"
#include "fold_dev.cuh"
#include "grid_dev.cuh"
#include "stencil_dev.cuh"

namespace {


constexpr int kWrWarps = 4;              // warps per block; each warp is an independent strip
constexpr int kWrThreads = 32 * kWrWarps;
constexpr int kWrERing = 8;              // rows of e in each lane's ring (a power of 2)
constexpr int kWrRRing = 16;             // rows of r in each lane's ring (a power of 2)
constexpr int kWrAhead = 6;              // input rows in flight ahead of the one consumed

struct WrWeights {
    float w[4];
};

__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Folded index and sign of row y (warp-uniform).
__device__ __forceinline__ int wr_row(int y, int Ny, float &sy) {
    if (y >= 1 && y <= Ny) {
        sy = 1.0f;
        return y;
    }
    return fold(y, Ny, sy);
}

// Starts the copies of row y of e and r (this lane's four columns) into ring rows de, dr;
// a Dirichlet row (sign 0) is stored as 0 at once, and a mirrored row is copied from the row
// it mirrors (its sign is applied when it is consumed).
__device__ __forceinline__ void wr_issue(const float *__restrict__ e, const float *__restrict__ r, const Grid &g,
                                         int c0, int y, float4 *de, float4 *dr) {
    float sy;
    const int fy = wr_row(y, g.Ny, sy);
    if (sy == 0.0f) {
        *de = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        *dr = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        return;
    }
    const long long k = g.idx(c0, fy);
    cp_async16(de, e + k);
    cp_async16(dr, r + k);
}

// Dirichlet columns of a new row.  Every row of every stage keeps column Nx + 1 at 0 and, for
// the 5-wide stencil, column Nx + 2 at -u(Nx) (the values the odd extension gives them
// exactly), and on the left column 0 at 0 and column -1 at -u(1).  Columns past Nx + R are
// never read by a node in 1 .. Nx.
struct WrEdge {
    bool left;       // this lane holds column 1 (its left side columns are 0 and -1)
    unsigned zero;   // bit m: column c0 + m is Nx + 1;   bit 4 + q: side column c0 + 3 + q is
    unsigned neg;    // bit m: column c0 + m is Nx + 2;   bit 4 + q: side column c0 + 3 + q is
};

// The lane's own four values, before they are shared with the neighbouring lanes.
template <int R>
__device__ __forceinline__ float4 wr_edge_own(const WrEdge &ed, float4 v) {
    float a[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        if (ed.zero >> m & 1u) a[m] = 0.0f;
        if (R == 2 && m >= 2 && (ed.neg >> m & 1u)) a[m] = -a[m - 2];
    }
    return make_float4(a[0], a[1], a[2], a[3]);
}

// The side columns after the shuffles.
template <int R, int WC>
__device__ __forceinline__ void wr_edge_side(const WrEdge &ed, float (&row)[WC]) {
    if (ed.left) {
        row[R - 1] = 0.0f;
        if (R == 2) row[0] = -row[R];
    }
#pragma unroll
    for (int q = 1; q <= R; ++q) {
        if (ed.zero >> (3 + q) & 1u) row[R + 3 + q] = 0.0f;
        if (R == 2 && (ed.neg >> (3 + q) & 1u)) row[R + 3 + q] = -row[R + 1 + q];
    }
}

// Puts the four values v of a new row into window row `row` (columns c0 - R .. c0 + 3 + R),
// with the side columns from the neighbouring lanes; `edge`: this warp's strip touches a
// Dirichlet column (warp-uniform).
template <int R, int WC>
__device__ __forceinline__ void wr_put(float (&row)[WC], float4 v, bool edge, const WrEdge &ed) {
    if (edge) v = wr_edge_own<R>(ed, v);
    row[R] = v.x;
    row[R + 1] = v.y;
    row[R + 2] = v.z;
    row[R + 3] = v.w;
    const float vs[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int q = 1; q <= R; ++q) {
        row[R - q] = __shfl_up_sync(0xffffffffu, vs[4 - q], 1);
        row[R + 3 + q] = __shfl_down_sync(0xffffffffu, vs[q - 1], 1);
    }
    if (edge) wr_edge_side<R, WC>(ed, row);
}

// Per-row differences of one stage's input at this lane's columns, alternating between
// iterations: dN[m] = e(c0+m, y+1) - e(c0+m, y) for the row pair (y, y+1), and (9-point) X[m],
// the horizontal second difference of row y + 1.  Node (i, y) uses dN for its upper
// neighbour and node (i, y+1), one iteration later, for its lower one (the two signs of the
// same difference: e(a) - e(b) = -(e(b) - e(a)) exactly under round-to-nearest); a row's X
// serves the three rows whose stencils include it.
struct WrPair {
    float dN[4], X[4];
};

// (L e - r) at this lane's four nodes of the centre row rc (upper row rn; lo: the entries of
// the previous iteration, dN of (y-1, y) and X of row y; hi: on entry the entries of two
// iterations back, whose X is that of row y - 1; filled here with dN of (y, y+1) and X of row
// y + 1), in the operation order of resid_diff32, so each node's result is bit-identical to it.
template <int ST, int R, int WC>
__device__ __forceinline__ void wr_resid(const float (&rc)[WC], const float (&rn)[WC], const WrPair &lo,
                                         WrPair &hi, const float (&rk)[4], float (&res)[4]) {
    float dN[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) dN[m] = rn[R + m] - rc[R + m];
    if (ST == 5) {
        float dE[5];  // dE[j] = e(c0 + j) - e(c0 - 1 + j) of the centre row
#pragma unroll
        for (int j = 0; j < 5; ++j) dE[j] = rc[R + j] - rc[R + j - 1];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const float Y1 = dN[m] - lo.dN[m];
            const float X1c = dE[m + 1] - dE[m];
            res[m] = (X1c + Y1) - rk[m];
            hi.dN[m] = dN[m];
        }
    } else {
        float dE[5];  // of the upper row
#pragma unroll
        for (int j = 0; j < 5; ++j) dE[j] = rn[R + j] - rn[R + j - 1];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const float Xn = dE[m + 1] - dE[m];
            const float Y1 = dN[m] - lo.dN[m];
            const float X1s = hi.X[m] + Xn;
            res[m] = fmaf(1.0f / 6.0f, X1s, fmaf(2.0f / 3.0f, lo.X[m], Y1 - rk[m]));
            hi.dN[m] = dN[m];
            hi.X[m] = Xn;
        }
    }
}

// The 17-point stencil's per-row entries of one stage's input, in rings indexed by the
// iteration (the window's ring length is 6, so every index below is a constant): X1 and X2,
// the horizontal second differences at spacings 1 and 2 of the row that is two above the
// centre when it is formed, serve the centre rows within one (X1) and at 0 or 2 (X2) rows of
// it.  The vertical differences are formed from the window's rows at each centre.
struct Wr17 {
    float x1[3][4], x2[6][4];
};

// (L e - r) of the 17-point stencil at this lane's four nodes of the centre row rc (rows below
// it rm2, rm1, above it r1, r2) at iteration Q (mod 6), in the operation order of resid_diff32.
template <int Q, int WC>
__device__ __forceinline__ void wr_resid17(const float (&rm2)[WC], const float (&rm1)[WC], const float (&rc)[WC],
                                           const float (&r1)[WC], const float (&r2)[WC], Wr17 &z, const float (&rk)[4],
                                           float (&res)[4]) {
    constexpr int R = 2;
    constexpr int n3 = Q % 3, c3 = (Q + 1) % 3, u3 = (Q + 2) % 3;  // X1 of rows y-1 (then y+2), y, y+1
    float dE1[5], dE2[6];  // dE1[j] = e(c0+j) - e(c0+j-1), dE2[q] = e(c0+q) - e(c0+q-2) of row y + 2
#pragma unroll
    for (int j = 0; j < 5; ++j) dE1[j] = r2[R + j] - r2[R + j - 1];
#pragma unroll
    for (int q = 0; q < 6; ++q) dE2[q] = r2[R + q] - r2[R + q - 2];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const float X1n = dE1[m + 1] - dE1[m];
        const float X2n = dE2[m + 2] - dE2[m];
        const float d1 = r1[R + m] - rc[R + m];
        const float d2 = r2[R + m] - rc[R + m];
        const float Y1 = d1 - (rc[R + m] - rm1[R + m]);
        const float Y2 = d2 - (rc[R + m] - rm2[R + m]);
        const float X1s = z.x1[n3][m] + z.x1[u3][m];
        const float X2s = z.x2[(Q + 2) % 6][m] + X2n;
        res[m] = fmaf(2.0f / 9.0f, X1s,
                      fmaf(8.0f / 9.0f, z.x1[c3][m],
                           fmaf(4.0f / 3.0f, Y1,
                                fmaf(-1.0f / 72.0f, X2s,
                                     fmaf(-1.0f / 18.0f, z.x2[(Q + 4) % 6][m], fmaf(-1.0f / 12.0f, Y2, -rk[m]))))));
        z.x1[n3][m] = X1n;
        z.x2[Q][m] = X2n;
    }
}

// Calls f(std::integral_constant<int, I>) for I = B .. E-1, each with its index a constant.
template <int B, int E, class F>
__device__ __forceinline__ void wr_static_for(F &&f) {
    if constexpr (B < E) {
        f(std::integral_constant<int, B>{});
        wr_static_for<B + 1, E>(f);
    }
}

// First staged column of strip x: strip 0 starts at column 1 and stores lanes 0 .. 30, the
// others start 4 columns before their first output column and store lanes 1 .. 30.
__host__ __device__ __forceinline__ int wr_strip_x0(int x) { return x == 0 ? 1 : 121 + 120 * (x - 1); }

__host__ __device__ __forceinline__ int wr_strips(int Nx) { return Nx <= 124 ? 1 : 1 + (Nx - 124 + 119) / 120; }

// One warp's work: K sweeps of strip `strip` over row block `rb` (blocks of `rows` rows) of the
// grid g, with this warp's shared-memory rings er (kWrERing x 32) and rr (kWrRRing x 32).  The
// arguments are warp-uniform; no block barrier is used.
template <int ST, int K>
__device__ __forceinline__ void wr_run(const float *__restrict__ e, const float *__restrict__ r,
                                       float *__restrict__ out, const Grid &g, const WrWeights &wt, int rows,
                                       int strip, int rb, float4 *er, float4 *rr) {
    constexpr int R = ST == 17 ? 2 : 1;
    constexpr int H = R * K;
    static_assert(H <= 4, "the valid strip after K stages is lanes 1 .. 30");
    constexpr int SK = R + 1;      // rows between consecutive stages
    constexpr int W = 2 * R + 2;   // window rows per stage input
    constexpr int WC = 4 + 2 * R;  // window columns
    constexpr int D = kWrAhead;
    static_assert(W % 2 == 0, "the pair differences alternate with the iteration's parity");
    static_assert(D < kWrERing && K * SK + D < kWrRRing, "ring rows still in use would be overwritten");
    const int lane = (int)threadIdx.x & 31;
    const int Nx = g.Nx, Ny = g.Ny;
    const int c0 = wr_strip_x0(strip) + 4 * lane;  // first of this lane's columns
    const bool live = c0 <= Nx;                    // lanes past Nx hold nothing that is read
    const int y0 = rb * rows + 1;
    const int y1 = min(y0 + rows - 1, Ny);  // last output row
    const int ystart = y0 - H, ylast = y1 + H;
    const int T = (y1 - y0 + 1) + H + K * SK;  // output row y1 leaves at iteration T - 1
    const bool out_lane = live && lane <= 30 && (lane >= 1 || strip == 0);
    // warp-uniform: the strip holds column 1, or one of its 128 columns lies past Nx (then
    // the lane holding Nx keeps the Dirichlet columns; the last strip, and the one before it
    // when Nx falls in its side lane)
    const bool edge = strip == 0 || wr_strip_x0(strip) + 127 > Nx;
    WrEdge ed;
    ed.left = strip == 0 && lane == 0;
    ed.zero = ed.neg = 0u;
#pragma unroll
    for (int m = 0; m < 4 + R; ++m) {  // own columns m < 4, side columns c0 + 3 + q at bit 3 + q
        const int c = c0 + m;
        if (c == Nx + 1) ed.zero |= 1u << m;
        if (R == 2 && c == Nx + 2) ed.neg |= 1u << m;
    }

    const float4 z4 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll
    for (int q = 0; q < kWrERing; ++q) er[q * 32 + lane] = z4;
#pragma unroll
    for (int q = 0; q < kWrRRing; ++q) rr[q * 32 + lane] = z4;

    // win[s][q][c]: input of stage s+1 as a ring of W rows (the row produced at iteration t
    // sits at q = t mod W), columns c0 - R .. c0 + 3 + R
    float win[K][W][WC];
    // per-row differences of each stage's input, alternating between iterations (k & 1): the
    // entries computed at one iteration are the lower ones of the next
    WrPair pr2[K][2];
    Wr17 z17[ST == 17 ? K : 1];
    if (ST == 17) {
        float *zp = &z17[0].x1[0][0];
#pragma unroll
        for (int q = 0; q < (int)(sizeof(z17) / sizeof(float)); ++q) zp[q] = 0.0f;
    }
#pragma unroll
    for (int s = 0; s < K; ++s)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
#pragma unroll
            for (int m = 0; m < 4; ++m) pr2[s][h].dN[m] = pr2[s][h].X[m] = 0.0f;
        }
#pragma unroll
    for (int s = 0; s < K; ++s)
#pragma unroll
        for (int q = 0; q < W; ++q)
#pragma unroll
            for (int c = 0; c < WC; ++c) win[s][q][c] = 0.0f;

#pragma unroll
    for (int d = 0; d < D; ++d) {
        if (live && ystart + d <= ylast) wr_issue(e, r, g, c0, ystart + d, &er[d * 32 + lane], &rr[d * 32 + lane]);
        cp_async_commit();
    }

    // Iterations ts .. te-1 (ts a multiple of W) are the steady state: the row entering is inside
    // the grid and within the row block's reach, the row consumed is not mirrored, and the row
    // leaving is an output row; they run without those tests (FAST), the warm-up and the drain
    // with them.  The arithmetic is the same in both.
    const int ts = (H + K * SK + W - 1) / W * W;
    int te = min(T, min(Ny - y0 + H - D + 1, (y1 - y0) + 2 * H - D + 1));
    te = te > ts ? ts + (te - ts) / W * W : ts;
    const bool vec_lane = out_lane && c0 + 3 <= Nx && !(ST == 17 && (c0 == 1 || c0 + 3 >= Nx));
    auto iter = [&](auto kc, auto fastc, int t0) {
        constexpr int k = decltype(kc)::value;       // t mod W: the windows' ring positions are constants
        constexpr bool FAST = decltype(fastc)::value;
        const int t = t0 + k;
        if (!FAST && t >= T) return;
        const int yin = ystart + t;
        if (FAST) {
            if (live) {
                const long long q = g.idx(c0, yin + D);
                cp_async16(&er[((t + D) & (kWrERing - 1)) * 32 + lane], e + q);
                cp_async16(&rr[((t + D) & (kWrRRing - 1)) * 32 + lane], r + q);
            }
        } else if (live && yin + D <= ylast) {
            wr_issue(e, r, g, c0, yin + D, &er[((t + D) & (kWrERing - 1)) * 32 + lane],
                     &rr[((t + D) & (kWrRRing - 1)) * 32 + lane]);
        }
        cp_async_commit();
        cp_async_wait<D>();  // row yin has landed
        float4 ve = er[(t & (kWrERing - 1)) * 32 + lane];
        if (!FAST && (yin < 1 || yin > Ny)) {  // a mirrored row: apply its sign once, for every stage
            float sy;
            wr_row(yin, Ny, sy);
            float4 *pr = &rr[(t & (kWrRRing - 1)) * 32 + lane];
            const float4 vr = *pr;
            ve = make_float4(sy * ve.x, sy * ve.y, sy * ve.z, sy * ve.w);
            *pr = make_float4(sy * vr.x, sy * vr.y, sy * vr.z, sy * vr.w);
        }
        // stage s: row yin - s SK from the rows of ages SK - R .. SK + R of its window; the
        // row of age 0 is the one this iteration produces, so the K stages are computed
        // first and the new rows (ve and the stages' outputs) enter the windows afterwards
        float4 nr[K];  // new row of each window: nr[0] = ve, nr[s] = stage s's output
        nr[0] = ve;
        float4 ov;     // stage K's output
#pragma unroll
        for (int s = 1; s <= K; ++s) {
            const float4 rq = rr[((t - s * SK) & (kWrRRing - 1)) * 32 + lane];
            const float rk[4] = {rq.x, rq.y, rq.z, rq.w};
            float nv[4];
            if (ST == 17) {
                float res[4];
                wr_resid17<k, WC>(win[s - 1][(k - SK - 2 + 2 * W) % W], win[s - 1][(k - SK - 1 + 2 * W) % W],
                                  win[s - 1][(k - SK + 2 * W) % W], win[s - 1][(k - SK + 1 + 2 * W) % W],
                                  win[s - 1][(k - SK + 2 + 2 * W) % W], z17[s - 1], rk, res);
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    const float uc = win[s - 1][(k - SK + 2 * W) % W][R + m];
                    nv[m] = fmaf(wt.w[s - 1], res[m], uc);
                }
            } else {
                float res[4];
                wr_resid<ST, R, WC>(win[s - 1][(k - SK + 2 * W) % W], win[s - 1][(k - SK + 1 + 2 * W) % W],
                                    pr2[s - 1][(k + 1) & 1], pr2[s - 1][k & 1], rk, res);
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    const float uc = win[s - 1][(k - SK + 2 * W) % W][R + m];
                    nv[m] = fmaf(wt.w[s - 1], res[m], uc);
                }
            }
            if (s < K)
                nr[s] = make_float4(nv[0], nv[1], nv[2], nv[3]);
            else
                ov = make_float4(nv[0], nv[1], nv[2], nv[3]);
        }
        // the new rows enter the windows, with the Dirichlet columns under one branch
        if (edge) {
#pragma unroll
            for (int s = 0; s < K; ++s) nr[s] = wr_edge_own<R>(ed, nr[s]);
        }
#pragma unroll
        for (int s = 0; s < K; ++s) wr_put<R, WC>(win[s][k], nr[s], false, ed);
        if (edge) {
#pragma unroll
            for (int s = 0; s < K; ++s) wr_edge_side<R, WC>(ed, win[s][k]);
        }
        const int yo = yin - K * SK;
        if (FAST && ST != 17) {  // yo is an output row
            if (vec_lane) {
                *reinterpret_cast<float4 *>(out + g.idx(c0, yo)) = ov;
            } else if (out_lane) {
                const float o4[4] = {ov.x, ov.y, ov.z, ov.w};
#pragma unroll
                for (int m = 0; m < 4; ++m)
                    if (c0 + m <= Nx) store_node<R, float>(out, g, c0 + m, yo, o4[m]);
            }
        } else if (out_lane && yo >= y0 && yo <= y1) {
            const bool bnd = ST == 17 && (c0 == 1 || c0 + 3 >= Nx || yo == 1 || yo == Ny);
            if (c0 + 3 <= Nx && !bnd) {
                *reinterpret_cast<float4 *>(out + g.idx(c0, yo)) = ov;
            } else {
                const float o4[4] = {ov.x, ov.y, ov.z, ov.w};
#pragma unroll
                for (int m = 0; m < 4; ++m)
                    if (c0 + m <= Nx) store_node<R, float>(out, g, c0 + m, yo, o4[m]);
            }
        }
    };
    for (int t0 = 0; t0 < T; t0 += W) {
        if (t0 == ts && ts < te) {
            for (; t0 < te; t0 += W) wr_static_for<0, W>([&](auto kc) { iter(kc, std::true_type{}, t0); });
            if (t0 >= T) break;
        }
        wr_static_for<0, W>([&](auto kc) { iter(kc, std::false_type{}, t0); });
    }
    cp_async_wait<0>();
}

}  // namespace
