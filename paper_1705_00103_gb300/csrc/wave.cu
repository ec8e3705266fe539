// Wavefront temporal blocking of the FP32 inner sweep (sm_103a): K consecutive weighted
// sweeps e <- e + w_n (L e - r) per HBM round trip, each with its own weight.  The register
// wavefront (wave_reg.cu) serves depths 2-4 of the 5- and 9-point stencils and depth 2 of the
// 17-point one; this kernel serves depth 8 and the 17-point depth 4.
//
// A block of kWaveW threads owns a strip of kWaveW staged columns (one per thread: kWaveW - 2H output
// columns plus an x-halo of H = r K on each side, r = stencil radius) and streams down a
// block of rows.  Every iteration loads one new input row and pushes the K stages one row
// further: stage s computes row y_in - r s from the rows y_in - r s - r .. y_in - r s + r of
// stage s-1.  Each thread keeps its own column's values and horizontal pair sums of those
// rows in registers, so only the newest row of each stage goes through shared memory (one
// row buffer per stage, read by the next stage for the horizontal neighbours); the output
// of stage K is written back.
// There is no halo in y (rows are streamed, not tiled), so each block redoes only the H
// columns on each side and the 2H warm-up rows of its row block.
//
// Boundaries: the grid is extended by the odd reflection the homogeneous Dirichlet boundary
// implies (u and r odd about nodes 0 and N+1, which stay 0).  Every operation of the sweep
// is an odd function of its inputs under round-to-nearest (differences, sums, fma with
// constant coefficients and weights), so the values computed on reflected rows and columns
// are the exact negatives of their mirrors, and interior values equal those of one-sweep
// launches bit for bit -- with no per-stage ghost refresh.
//
// Per node and stage: 2 (5/9-point) or 4 (17-point) shared-memory loads for the horizontal
// neighbours, which each thread keeps, with its own column's values, in register windows
// down the rows; the residual is evaluated in difference form (resid_diff32), as in the
// one-sweep FP32 kernel.  HBM traffic per update: about (4 e + 4 r + 4 e') / K bytes plus
// the halo.
#include "cj_internal.h"
#include "fold_dev.cuh"
#include "grid_dev.cuh"
#include "stencil_dev.cuh"

namespace {

constexpr int kWaveW = 128;   // threads = staged columns per block (measured best of 128, 256, 512)

struct WaveWeights {
    float w[kTbMaxDepth];
};

// True when row y of the odd extension is a Dirichlet row (a node 0 or N+1 image).
__device__ __forceinline__ bool boundary_row(int y, int N) {
    if (y >= 1 && y <= N) return false;
    float sg;
    fold(y, N, sg);
    return sg == 0.0f;
}

// Value of e or r at node (ci, row y) of the odd extension (0 on the boundary rows/columns).
__device__ __forceinline__ float load_ext(const float *__restrict__ a, const Grid &g, int ci, float csign,
                                          int y) {
    float rs;
    const int ry = fold(y, g.Ny, rs);
    const float s = rs * csign;
    return s == 0.0f ? 0.0f : s * __ldg(a + g.idx(ci, ry));
}

template <int ST, int K>
__global__ void __launch_bounds__(kWaveW) sweep_wave_kernel(const float *__restrict__ e,
                                                            const float *__restrict__ r,
                                                            float *__restrict__ out, Grid g,
                                                            WaveWeights wt, int rows) {
    constexpr int R = ST == 17 ? 2 : 1;
    constexpr int H = R * K;
    constexpr int TX = kWaveW - 2 * H;  // output columns per block
    constexpr int RING = 2 * R + 1;     // rows in a register window
    constexpr int RW = kWaveW + 2 * R;  // row buffer width (R pad columns each side)
    constexpr int D = RING;             // rows of e and r loaded ahead
    constexpr int RQ = H + 1;           // r of rows yin .. yin - H, one slot per row
    __shared__ float ring[K][RW];
    __shared__ float rline[RQ][kWaveW];

    const int tid = threadIdx.x;
    const int gi = (int)blockIdx.x * TX + 1 - H + tid;  // this thread's column
    const int y0 = (int)blockIdx.y * rows + 1;           // first output row
    const int Nx = g.Nx, Ny = g.Ny;
    float csign;
    const int ci = fold(gi, Nx, csign);  // column of the original grid this one mirrors
    const bool col_bc = csign == 0.0f;

    for (int k = tid; k < K * RW; k += kWaveW) (&ring[0][0])[k] = 0.0f;
    for (int k = 0; k < RQ; ++k) rline[k][tid] = 0.0f;

    // register windows of each stage's input (stage s reads stage s-1): the values of the
    // last 2R+1 rows (index 2R = newest) at this thread's column and at the columns R
    // to either side (wv[s][c][q]: column offset c - R)
    float wv[K][2 * R + 1][RING];
#pragma unroll
    for (int s = 0; s < K; ++s)
#pragma unroll
        for (int c = 0; c < 2 * R + 1; ++c)
#pragma unroll
            for (int q = 0; q < RING; ++q) wv[s][c][q] = 0.0f;
    // loads in flight: eq[d], rq[d] hold rows yin + d
    float eq[D], rq[D];
    const int ystart = y0 - H;
#pragma unroll
    for (int d = 0; d < D; ++d) {
        eq[d] = load_ext(e, g, ci, csign, ystart + d);
        rq[d] = load_ext(r, g, ci, csign, ystart + d);
    }

    __syncthreads();
    int tend = rows + 2 * H;
    if (ystart + tend - 1 > Ny + H) tend = Ny + H - ystart + 1;  // rows past the last output's needs
    int slot = 0;                                                // rline slot of row yin
    // unrolled by the window length, so the window shifts become register renames
#pragma unroll RING
    for (int t = 0; t < tend; ++t) {
        const int yin = ystart + t;
        float v = col_bc ? 0.0f : eq[0];
        rline[slot][tid] = rq[0];
#pragma unroll
        for (int d = 0; d < D - 1; ++d) {
            eq[d] = eq[d + 1];
            rq[d] = rq[d + 1];
        }
        eq[D - 1] = load_ext(e, g, ci, csign, yin + D);
        rq[D - 1] = load_ext(r, g, ci, csign, yin + D);
        ring[0][tid + R] = v;
        __syncthreads();
#pragma unroll
        for (int s = 1; s <= K; ++s) {
            // push stage s-1's newest row (row yin - R (s-1)) into stage s's window
            const float *row = &ring[s - 1][tid + R];
#pragma unroll
            for (int c = 0; c < 2 * R + 1; ++c) {
#pragma unroll
                for (int q = 0; q < RING - 1; ++q) wv[s - 1][c][q] = wv[s - 1][c][q + 1];
                wv[s - 1][c][RING - 1] = c == R ? v : row[c - R];
            }
            // stage s: row y = yin - R s, window rows y-R .. y+R; r(y) from the r line
            const int y = yin - R * s;
            const bool bc_row = boundary_row(y, Ny);
            float nv = 0.0f;
            if (!bc_row && !col_bc) {
                int rs = slot - R * s;
                if (rs < 0) rs += RQ;
                const float rk = rline[rs][tid];
                auto N = [&](int dx, int dy) { return wv[s - 1][R + dx][R + dy]; };
                const float uc = wv[s - 1][R][R];
                const float res = resid_diff32<ST>(N, uc, rk);
                nv = fmaf(wt.w[s - 1], res, uc);
            }
            v = nv;
            if (s < K) {
                // the next stage reads this row; the row it replaces was last read before
                // the barrier that followed this iteration's input load
                ring[s][tid + R] = v;
                __syncthreads();
            }
        }
        // stage K produced row yin - H
        const int yo = yin - H;
        if (yo >= y0 && yo < y0 + rows && yo <= Ny && tid >= H && tid < kWaveW - H && gi >= 1 &&
            gi <= Nx)
            store_node<R, float>(out, g, gi, yo, v);
        slot = slot + 1 == RQ ? 0 : slot + 1;
    }
}

// Rows per block so that the grid is one wave of resident blocks (at least 2H + 1, so the
// warm-up rows stay a minority).
template <int ST, int K>
int wave_rows(const Grid &g, int nstrips) {
    static const int resident = [] {  // computed once, thread-safely
        int dev = 0, sms = 152, per_sm = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep_wave_kernel<ST, K>, kWaveW, 0) !=
                cudaSuccess ||
            per_sm < 1)
            per_sm = 1;
        return sms * per_sm;
    }();
    constexpr int H = (ST == 17 ? 2 : 1) * K;
    int nby = resident / nstrips;
    if (nby < 1) nby = 1;
    int rows = (g.Ny + nby - 1) / nby;
    if (rows < 2 * H + 1) rows = 2 * H + 1;
    return rows;
}

template <int ST, int K>
cudaError_t launch_wave_k(const Grid &g, const float *e, const float *r, float *out,
                          const float *w, cudaStream_t s) {
    constexpr int R = ST == 17 ? 2 : 1;
    constexpr int TX = kWaveW - 2 * R * K;
    WaveWeights wt{};
    for (int k = 0; k < K; ++k) wt.w[k] = w[k];
    const int nstrips = (g.Nx + TX - 1) / TX;
    const int rows = wave_rows<ST, K>(g, nstrips);
    const dim3 grid(nstrips, (g.Ny + rows - 1) / rows);
    sweep_wave_kernel<ST, K><<<grid, kWaveW, 0, s>>>(e, r, out, g, wt, rows);
    return cudaGetLastError();
}

template <int ST>
cudaError_t launch_wave_st(const Grid &g, const float *e, const float *r, float *out,
                           const float *w, int k, cudaStream_t s) {
    switch (k) {
        case 2: return launch_wave_k<ST, 2>(g, e, r, out, w, s);
        case 4: return launch_wave_k<ST, 4>(g, e, r, out, w, s);
        case 8: return launch_wave_k<ST, 8>(g, e, r, out, w, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

int wave_depth_supported(int k) { return k == 2 || k == 4 || k == 8; }

cudaError_t launch_sweep32_wave(const cj_plan *p, const float *e, const float *r, float *out,
                                const float *w, int k, cudaStream_t s) {
    switch (p->st) {
        case 5: return launch_wave_st<5>(p->g32, e, r, out, w, k, s);
        case 9: return launch_wave_st<9>(p->g32, e, r, out, w, k, s);
        default: return launch_wave_st<17>(p->g32, e, r, out, w, k, s);
    }
}
