// Temporal blocking of the FP32 inner sweep (sm_103a): up to kTbMaxDepth consecutive
// weighted sweeps e <- e + w_n (L e - r), each with its own weight, per HBM round trip.
//
// A block owns an output tile of kTbX x kTbY nodes.  It stages the tile plus a halo of
// r * depth nodes (r = stencil radius) of e and of r in shared memory, runs the sweeps there
// -- stage s recomputes a region that shrinks by r on every side, so the tile's centre is
// exact after the last stage -- and writes only the centre back.  Between stages the ghost
// nodes inside the staged region are refreshed: Dirichlet nodes 0 and N+1 hold 0, and for
// the 17-point stencil the outer ghost layer is the odd reflection of the new interior.
// Each node of each stage is evaluated with the same arithmetic, in the same order, as the
// one-sweep kernel, so a depth-K launch equals K one-sweep launches bit for bit.
//
// HBM traffic per update falls from 12 bytes (read e and r, write e) to about
// (2 (X+2H)(Y+2H) + X Y) * 4 / (K X Y) bytes, H = r K; the work moves to shared memory and
// the FP32 pipes, which have far more headroom on GB300 than HBM.  (The FP64 sweep does not
// use this: it is bound by the FP64 pipe, and the halo recomputation would only add work.)
#include "cj_internal.h"
#include "grid_dev.cuh"
#include "stencil_dev.cuh"

namespace {

constexpr int kTbX = 128, kTbY = 32, kTbThreads = 256;

struct Weights {
    float w[kTbMaxDepth];
};

template <int ST>
__global__ void __launch_bounds__(kTbThreads) sweep_tb_kernel(const float *__restrict__ e,
                                                              const float *__restrict__ r,
                                                              float *__restrict__ out, Grid g,
                                                              int depth, Weights wt) {
    extern __shared__ float sm[];
    tb_tile<ST>(e, r, out, g, depth, wt.w, blockIdx.x * kTbX + 1, blockIdx.y * kTbY + 1, kTbX, kTbY,
                sm);
}

bool g_tb_attr_set[3] = {false, false, false};

}  // namespace

size_t tb_smem_bytes(int st, int depth) {
    const int R = st == 17 ? 2 : 1, H = R * depth;
    return (size_t)3 * (kTbX + 2 * H) * (kTbY + 2 * H) * sizeof(float);
}

cudaError_t launch_sweep32_tb(const cj_plan *p, const float *e, const float *r, float *out,
                              const float *w, int depth, cudaStream_t s) {
    if (depth < 1 || depth > kTbMaxDepth) return cudaErrorInvalidValue;
    Weights wt{};
    for (int k = 0; k < depth; ++k) wt.w[k] = w[k];
    const dim3 grid((p->Nx + kTbX - 1) / kTbX, (p->Ny + kTbY - 1) / kTbY);
    const size_t smem = tb_smem_bytes(p->st, depth);
    const size_t smem_max = tb_smem_bytes(p->st, kTbMaxDepth);
    const int which = p->st == 5 ? 0 : p->st == 9 ? 1 : 2;
    cudaError_t err = cudaSuccess;
    if (!g_tb_attr_set[which]) {
        switch (p->st) {
            case 5: err = cudaFuncSetAttribute(sweep_tb_kernel<5>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max); break;
            case 9: err = cudaFuncSetAttribute(sweep_tb_kernel<9>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max); break;
            default: err = cudaFuncSetAttribute(sweep_tb_kernel<17>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max); break;
        }
        if (err != cudaSuccess) return err;
        g_tb_attr_set[which] = true;
    }
    switch (p->st) {
        case 5: sweep_tb_kernel<5><<<grid, kTbThreads, smem, s>>>(e, r, out, p->g32, depth, wt); break;
        case 9: sweep_tb_kernel<9><<<grid, kTbThreads, smem, s>>>(e, r, out, p->g32, depth, wt); break;
        default: sweep_tb_kernel<17><<<grid, kTbThreads, smem, s>>>(e, r, out, p->g32, depth, wt); break;
    }
    return cudaGetLastError();
}
