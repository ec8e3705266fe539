// One FP32 weighted sweep e' = e + w (L e - r) of the inner CJM cycles, in the difference form
// of the FP32 evaluation (resid_diff32): four adjacent columns per thread (march4).
//
// The sweep moves 12 bytes per update (read e and r, write e') and does ~20 FP32 operations,
// so it is bound by HBM; what limits a one-column-per-thread march is the number of bytes in
// flight.  Here each thread loads the four columns of a row as one 16-byte vector, stores its
// four results as one vector, issues the next row's loads before it computes the current row,
// and walks down `ty` rows.  The grid is exactly one wave of resident blocks.
//
// Boundaries are those of the padded FP32 grids: nodes 0 and N+1 hold 0 and, for the 17-point
// stencil, the outer ghost layer holds the odd reflection, which store_node rewrites whenever a
// boundary-adjacent node changes.  Results equal the one-column march's bit for bit (same
// formula per node).
#include "march4_dev.cuh"

namespace {

// The 17-point kernel is held to 85 registers (6 blocks per SM): measured 422 Gupd/s on 8192^2
// against 365 at its unconstrained 119 registers (4 blocks) and 407 at 5 blocks.  (Minimum blocks
// 0 leaves the 5- and 9-point kernels to the compiler's own register choice.)
template <int ST>
__global__ void __launch_bounds__(kBX, ST == 17 ? 6 : 0) sweep32_vec_kernel(const float *__restrict__ e, const float *__restrict__ r,
                                                          float *__restrict__ out, Grid g, int ty, float w) {
    const int c0 = ((int)blockIdx.x * kBX + (int)threadIdx.x) * 4 + 1;  // first of this thread's columns
    const int j0 = (int)blockIdx.y * ty + 1;
    const int j1 = min(j0 + ty - 1, g.Ny);
    if (c0 > g.Nx) return;
    M4Store<ST> op{out, &g, c0, w};
    march4<ST>(e, r, g, c0, j0, j1, op);
}

template <int ST>
cudaError_t launch_st(const Grid &g, const float *e, const float *r, float *out, float w, cudaStream_t s) {
    // blocks of this kernel resident on the device at once (computed once, thread-safely)
    static const int resident = [] {
        int dev = 0, sms = 152, per_sm = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep32_vec_kernel<ST>, kBX, 0) != cudaSuccess ||
            per_sm < 1)
            per_sm = 1;
        return sms * per_sm;
    }();
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
