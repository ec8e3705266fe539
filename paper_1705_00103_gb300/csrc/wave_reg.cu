// The register wavefront (wave_reg_dev.cuh) over one whole grid: K = 2-4 FP32 inner sweeps per
// launch, every warp one (strip, row block) of the grid, one wave of warps.
#include "wave_reg_dev.cuh"

namespace {

// Registers: the 9-point depth-4 kernel carries about 240 (windows and pair differences of
// four stages), so it runs 2 blocks per SM; 3 blocks (12 warps, 168 registers each, as the register
// file is split between the SM's four schedulers) would spill.
template <int ST, int K>
__global__ void __launch_bounds__(kWrThreads, ST == 17 || (ST == 9 && K == 4) ? 2 : 3)
    sweep_wave_reg_kernel(const float *__restrict__ e, const float *__restrict__ r, float *__restrict__ out,
                          Grid g, WrWeights wt, int rows, int nrb, int nstrips) {
    __shared__ float4 ering[kWrWarps][kWrERing][32];
    __shared__ float4 rring[kWrWarps][kWrRRing][32];

    const int wid = (int)threadIdx.x >> 5;
    const int gw = (int)blockIdx.x * kWrWarps + wid;  // (strip, row block) of this warp
    if (gw >= nstrips * nrb) return;                   // whole warp: no block barrier is used
    const int strip = gw % nstrips, rb = gw / nstrips;
    wr_run<ST, K>(e, r, out, g, wt, rows, strip, rb, ering[wid][0], rring[wid][0]);
}

// Warps of this kernel resident on the device at once (computed once, thread-safely).
template <int ST, int K>
int wr_resident_warps() {
    static const int n = [] {
        int dev = 0, sms = 152, per_sm = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep_wave_reg_kernel<ST, K>, kWrThreads, 0) !=
                cudaSuccess ||
            per_sm < 1)
            per_sm = 1;
        return sms * per_sm * kWrWarps;
    }();
    return n;
}

template <int ST, int K>
cudaError_t launch_k(const Grid &g, const float *e, const float *r, float *out, const float *w, cudaStream_t s) {
    constexpr int H = (ST == 17 ? 2 : 1) * K;
    WrWeights wt{};
    for (int k = 0; k < K; ++k) wt.w[k] = w[k];
    const int nstrips = wr_strips(g.Nx);
    // at most one wave of warps; row blocks of at least 4H rows so the warm-up stays a minority
    int nrb = wr_resident_warps<ST, K>() / nstrips;
    if (nrb < 1) nrb = 1;
    int rows = (g.Ny + nrb - 1) / nrb;
    if (rows < 4 * H) rows = 4 * H;
    nrb = (g.Ny + rows - 1) / rows;
    const long long warps = (long long)nstrips * nrb;
    const int blocks = (int)((warps + kWrWarps - 1) / kWrWarps);
    sweep_wave_reg_kernel<ST, K><<<blocks, kWrThreads, 0, s>>>(e, r, out, g, wt, rows, nrb, nstrips);
    return cudaGetLastError();
}

}  // namespace

int wave_reg_supported(int st, int k) { return k == 2 || ((k == 3 || k == 4) && st != 17); }

cudaError_t launch_sweep32_wave_reg(const cj_plan *p, const float *e, const float *r, float *out,
                                    const float *w, int k, cudaStream_t s) {
    if (!wave_reg_supported(p->st, k)) return cudaErrorInvalidValue;
    switch (p->st) {
        case 5:
            return k == 2 ? launch_k<5, 2>(p->g32, e, r, out, w, s)
                   : k == 3 ? launch_k<5, 3>(p->g32, e, r, out, w, s)
                            : launch_k<5, 4>(p->g32, e, r, out, w, s);
        case 9:
            return k == 2 ? launch_k<9, 2>(p->g32, e, r, out, w, s)
                   : k == 3 ? launch_k<9, 3>(p->g32, e, r, out, w, s)
                            : launch_k<9, 4>(p->g32, e, r, out, w, s);
        default: return launch_k<17, 2>(p->g32, e, r, out, w, s);
    }
}
