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

namespace {

constexpr int kTbX = 128, kTbY = 32, kTbThreads = 256;

template <int ST>
__device__ __forceinline__ float resid_smem(const float *A, int SX, int x, int y, float rk) {
    auto U = [&](int dx, int dy) { return A[(y + dy) * SX + (x + dx)]; };
    const float uC = U(0, 0);
    const float v1 = U(0, -1) + U(0, 1);
    const float p0 = U(-1, 0) + U(1, 0);
    if (ST == 5) return (p0 + v1) + fmaf(-4.0f, uC, -rk);
    const float pm = U(-1, -1) + U(1, -1);
    const float pp = U(-1, 1) + U(1, 1);
    if (ST == 9)
        return fmaf(4.0f / 6.0f, p0 + v1, fmaf(1.0f / 6.0f, pm + pp, fmaf(-20.0f / 6.0f, uC, -rk)));
    const float v2 = U(0, -2) + U(0, 2);
    const float P0 = U(-2, 0) + U(2, 0);
    const float Pm = U(-2, -2) + U(2, -2);
    const float Pp = U(-2, 2) + U(2, 2);
    return fmaf(64.0f / 72.0f, p0 + v1,
                fmaf(-4.0f / 72.0f, P0 + v2,
                     fmaf(16.0f / 72.0f, pm + pp,
                          fmaf(-1.0f / 72.0f, Pm + Pp, fmaf(-300.0f / 72.0f, uC, -rk)))));
}

struct Weights {
    float w[kTbMaxDepth];
};

template <int ST>
__global__ void __launch_bounds__(kTbThreads) sweep_tb_kernel(const float *__restrict__ e,
                                                              const float *__restrict__ r,
                                                              float *__restrict__ out, Grid g,
                                                              int depth, Weights wt) {
    constexpr int R = ST == 17 ? 2 : 1;
    extern __shared__ float sm[];
    const int H = R * depth;
    const int SX = kTbX + 2 * H, SY = kTbY + 2 * H, NS = SX * SY;
    float *A = sm, *B = sm + NS, *Rs = sm + 2 * NS;
    // node (gx0 + x, gy0 + y) sits at staged cell (x, y)
    const int gx0 = blockIdx.x * kTbX + 1 - H, gy0 = blockIdx.y * kTbY + 1 - H;
    const int Nx = g.Nx, Ny = g.Ny;

    for (int c = threadIdx.x; c < NS; c += kTbThreads) {
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
        const float w = wt.w[s - 1];
        const int lo = R * s, wx = SX - 2 * lo, wy = SY - 2 * lo;
        for (int c = threadIdx.x; c < wx * wy; c += kTbThreads) {
            const int x = lo + c % wx, y = lo + c / wx, gi = gx0 + x, gj = gy0 + y;
            if (gi >= 1 && gi <= Nx && gj >= 1 && gj <= Ny) {
                const float uc = A[y * SX + x];
                B[y * SX + x] = fmaf(w, resid_smem<ST>(A, SX, x, y, Rs[y * SX + x]), uc);
            }
        }
        __syncthreads();
        if (R == 2) {
            // outer ghost layer of the new values: odd reflection of the interior
            for (int c = threadIdx.x; c < wx * wy; c += kTbThreads) {
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

    for (int c = threadIdx.x; c < kTbX * kTbY; c += kTbThreads) {
        const int x = H + c % kTbX, y = H + c / kTbX, gi = gx0 + x, gj = gy0 + y;
        if (gi <= Nx && gj <= Ny) store_node<R, float>(out, g, gi, gj, A[y * SX + x]);
    }
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
