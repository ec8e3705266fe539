// CUDA graphs of the FP64 sweeps for grids whose sweeps are shorter than a host-side launch.
//
// On grids of up to 2^22 nodes one FP64 sweep takes a few to a few tens of microseconds, about
// what the host needs to issue one kernel, so a cycle of M single-sweep launches is bound by the
// host, not the GPU.  A plan for such a grid builds, once, an instantiated graph of G sweeps
// (G = min(M, 128), a power of two, so an even chain that starts and ends in the buffer u0),
// followed by one node that advances a device-side position in the weight table by G.  A
// cycle is then a reset of the position and M / G graph launches.  The sweeps read their weight
// w_n from a device copy of the plan's table at index position + k; otherwise they are the
// one-sweep kernels' arithmetic (same march, same evaluation order), so results are identical.
#include "cj_internal.h"
#include "grid_dev.cuh"
#include "stencil_dev.cuh"

namespace {

constexpr long long kGraphMaxNodes = 1LL << 22;  // grids up to 2048 x 2048 use the graph
constexpr int kGraphChain = 128;                  // sweeps per graph launch (at most)

template <int ST, bool MIRROR>
struct TabSweepOp {
    double *out;
    const Grid *g;
    int i;
    double w;
    __device__ __forceinline__ void operator()(int j, double r, double uc) {
        store_node<((ST == 17 && MIRROR) ? 2 : 1)>(out, *g, i, j, Ar<double>::fm(w, r, uc));
    }
};

// One FP64 sweep whose weight is wtab[*pos + k] (a broadcast load, the same for every thread).
template <int ST, bool MIRROR>
__global__ void __launch_bounds__(kBX) sweep64_tab_kernel(const double *__restrict__ u,
                                                          const double *__restrict__ b,
                                                          double *__restrict__ out, Grid g, int ty,
                                                          const double *__restrict__ wtab,
                                                          const long long *__restrict__ pos, int k,
                                                          double one) {
    const int i = blockIdx.x * kBX + threadIdx.x + 1;
    const int j0 = blockIdx.y * ty + 1;
    const int j1 = min(j0 + ty - 1, g.Ny);
    if (i > g.Nx) return;
    TabSweepOp<ST, MIRROR> op{out, &g, i, wtab[*pos + k]};
    march<ST, double>(u, b, g, i, j0, j1, one, op);
}

// Moves the table position on by one graph's worth of sweeps, modulo the cycle length.
__global__ void advance_pos_kernel(long long *pos, long long G, long long M) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *pos = (*pos + G) % M;
}

void *tab_kernel(const cj_plan *p) {
    switch (p->st) {
        case 5: return (void *)sweep64_tab_kernel<5, true>;
        case 9: return (void *)sweep64_tab_kernel<9, true>;
        default:
            return p->bc == CJ_BC_DIRICHLET ? (void *)sweep64_tab_kernel<17, false>
                                            : (void *)sweep64_tab_kernel<17, true>;
    }
}

}  // namespace

bool sweep_graph_wanted(const cj_plan *p) {
    return p->M >= 2 && (long long)p->Nx * p->Ny <= kGraphMaxNodes;
}

cudaError_t make_sweep_graph(cj_plan *p) {
    const int G = (int)(p->M < kGraphChain ? p->M : kGraphChain);
    cudaError_t e = cudaMalloc((void **)&p->w_dev, sizeof(double) * (size_t)p->M);
    if (e == cudaSuccess) e = cudaMalloc((void **)&p->pos, sizeof(long long));
    if (e == cudaSuccess)
        e = cudaMemcpy(p->w_dev, p->w.data(), sizeof(double) * (size_t)p->M, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(p->pos, 0, sizeof(long long));
    if (e != cudaSuccess) return e;
    cudaGraph_t graph = nullptr;
    e = cudaGraphCreate(&graph, 0);
    if (e != cudaSuccess) return e;
    void *fn = tab_kernel(p);
    const dim3 grid(p->m64.nbx, p->m64.nby), block(kBX);
    const double *bb = p->b;
    Grid g = p->g64;
    int ty = p->m64.ty;
    const double *wt = p->w_dev;
    const long long *ps = p->pos;
    double one = 1.0;
    cudaGraphNode_t prev = nullptr;
    for (int k = 0; k < G && e == cudaSuccess; ++k) {
        const double *in = (k & 1) ? p->u1 : p->u0;
        double *out = (k & 1) ? p->u0 : p->u1;
        int kk = k;
        void *args[] = {(void *)&in, (void *)&bb, (void *)&out, (void *)&g, (void *)&ty,
                        (void *)&wt, (void *)&ps, (void *)&kk, (void *)&one};
        cudaKernelNodeParams kp{};
        kp.func = fn;
        kp.gridDim = grid;
        kp.blockDim = block;
        kp.sharedMemBytes = 0;
        kp.kernelParams = args;
        cudaGraphNode_t node;
        e = cudaGraphAddKernelNode(&node, graph, prev ? &prev : nullptr, prev ? 1 : 0, &kp);
        prev = node;
    }
    if (e == cudaSuccess) {
        long long *pp = p->pos;
        long long GG = G, MM = p->M;
        void *args[] = {(void *)&pp, (void *)&GG, (void *)&MM};
        cudaKernelNodeParams kp{};
        kp.func = (void *)advance_pos_kernel;
        kp.gridDim = dim3(1);
        kp.blockDim = dim3(32);
        kp.kernelParams = args;
        cudaGraphNode_t node;
        e = cudaGraphAddKernelNode(&node, graph, &prev, 1, &kp);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&p->graph, graph, 0);
    cudaGraphDestroy(graph);
    if (e == cudaSuccess) p->graph_G = G;
    return e;
}

cudaError_t launch_sweep_cycle_graph(const cj_plan *p, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(p->pos, 0, sizeof(long long), s);
    for (long long r = 0; r < p->M / p->graph_G && e == cudaSuccess; ++r) e = cudaGraphLaunch(p->graph, s);
    return e;
}
