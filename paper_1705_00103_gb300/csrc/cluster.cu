// Whole plain-FP64 CJM solves of small grids in one launch, resident in one thread-block cluster.
//
// On a grid of up to 2^14 nodes one FP64 sweep is a few microseconds of work spread over the
// whole GPU, so a solve of M-sweep cycles launched from the host (or replayed as a graph) is
// bound by launches, not arithmetic.  Here one cluster of C CTAs (up to 16, on C SMs) holds the
// grid in shared memory for the whole solve: CTA c owns a band of rows, with two ghost rows above
// and below, in two ping-pong buffers of full padded width (columns -1 .. Nx+2).  A sweep is:
// every CTA computes its rows from one buffer into the other (the weight w_n from the plan's
// table), storing each node of its first and last R rows (R the stencil radius) also into the
// neighbouring CTA's ghost rows of that buffer through distributed shared memory.  Those boundary
// rows are computed first, then the arrive half of the cluster barrier (release), the interior rows,
// and the wait half (acquire), so the barrier's latency overlaps the interior work.  A neighbour
// reads its ghost rows only for its own boundary rows, which it computes before it arrives, so the
// next sweep's stores never overwrite rows it still needs.  The residual test
// before every cycle reduces (sum r^2, max |r|, sum u^2) per CTA, and every CTA then reads all
// CTAs' triples in rank order through distributed shared memory, so all take the identical stop
// decision and leave the loop together.  No thread waits on a flag: the only waits are the
// hardware cluster barrier and the block barrier.
//
// Node arithmetic is the sweep kernels' (resid_direct, fma(w, r, u)), so the iterates equal the
// plan's other launch modes bit for bit; on the grid's boundary rows and columns the 17-point
// stencil's odd-reflection ghosts are rewritten with each node (store_node's rule), or, with
// Dirichlet data, the ring is loaded once and left alone.
#include <cooperative_groups.h>

#include <cstdio>

#include "cj_internal.h"
#include "grid_dev.cuh"
#include "stencil_dev.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr int kClThreads = 256;
constexpr long long kClusterMaxNodes = 1LL << 14;
constexpr size_t kClMaxSmem = 200 * 1024;  // dynamic shared memory per CTA, at most

struct ClArgs {
    double *u;            // padded FP64 grid (the plan's u0): initial guess in, solution out
    const double *b;      // padded b = h^2 f
    const double *w;      // M sweep coefficients
    double *res;          // [0] status, [1] sweeps, [2] cycles, [3] rho, [4] rinf, [5] fl
    Grid g;
    const double *bstat;  // (sum b^2, max |b|) from the import's reduction
    long long M, max_sweeps;
    double tol, S;
    int method;           // CJ_CJM or CJ_JACOBI
    int mirror;           // 17-point odd reflection at the boundary (homogeneous plans)
};

// rows of CTA c: first row (1-based) and count, the first Ny mod C bands one row longer
__device__ __forceinline__ void cl_band(int Ny, int C, int c, int &r0, int &nr) {
    const int q = Ny / C, rem = Ny % C;
    nr = q + (c < rem ? 1 : 0);
    r0 = 1 + c * q + (c < rem ? c : rem);
}

template <int ST>
__global__ void __launch_bounds__(kClThreads) cluster_solve_kernel(ClArgs a) {
    cg::cluster_group cl = cg::this_cluster();
    const int c = (int)cl.block_rank(), C = (int)cl.num_blocks();
    const int Nx = a.g.Nx, Ny = a.g.Ny, W = Nx + 4;
    int r0, nr;
    cl_band(Ny, C, c, r0, nr);
    int nr_max, dummy;
    cl_band(Ny, C, 0, dummy, nr_max);
    const int rows = nr_max + 4;  // buffer rows: q = 0, 1 ghosts above, 2 .. nr+1 own, then 2 ghosts
    extern __shared__ double sm[];
    double *const buf0 = sm, *const buf1 = sm + (long long)rows * W;
    double *bs = sm + 2LL * rows * W;            // own rows of b, nr_max x Nx
    double *red = bs + (long long)nr_max * Nx;   // 3 doubles: this CTA's residual triple; +3: scratch
    __shared__ double wred[kClThreads / 32][3];
    const int t = (int)threadIdx.x;

    // load rows r0-2 .. r0+nr+1 (ghost rows of the padded grid at the edges), full width, into
    // both buffers, and the own rows of b
    for (long long k = t; k < (long long)(nr + 4) * W; k += kClThreads) {
        const int q = (int)(k / W), x = (int)(k % W);
        const double v = a.u[a.g.idx(x - 1, r0 - 2 + q)];
        buf0[(long long)q * W + x] = v;
        buf1[(long long)q * W + x] = v;
    }
    for (long long k = t; k < (long long)nr * Nx; k += kClThreads) {
        const int q = (int)(k / Nx), i = (int)(k % Nx) + 1;
        bs[k] = a.b[a.g.idx(i, r0 + q)];
    }
    __syncthreads();

    int cur = 0, status = -1, stall = 0;
    long long sweeps = 0, cycles = 0;
    double prev = 0.0, rho = 0.0, rinf = 0.0, fl = 0.0;
    const double eps = 1.1102230246251565e-16;
    const double bn = sqrt(a.bstat[0]), bmax = a.bstat[1];
    for (;;) {
        // residual test: this CTA's triple, then all CTAs' in rank order
        double s2 = 0.0, mx = 0.0, u2 = 0.0;
        const double *U0 = cur ? buf1 : buf0;
        for (long long k = t; k < (long long)nr * Nx; k += kClThreads) {
            const int q = (int)(k / Nx) + 2, x = (int)(k % Nx) + 2;
            auto U = [&](int di, int dj) { return U0[(long long)(q + dj) * W + x + di]; };
            const double r = resid_direct<ST, double>(U, bs[k]);
            const double uc = U(0, 0);
            s2 = fma(r, r, s2);
            mx = (mx != mx || mx > fabs(r)) ? mx : fabs(r);
            u2 = fma(uc, uc, u2);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            s2 += __shfl_down_sync(0xffffffffu, s2, o);
            const double m2 = __shfl_down_sync(0xffffffffu, mx, o);
            mx = (mx != mx || mx > m2) ? mx : m2;
            u2 += __shfl_down_sync(0xffffffffu, u2, o);
        }
        if ((t & 31) == 0) {
            wred[t >> 5][0] = s2;
            wred[t >> 5][1] = mx;
            wred[t >> 5][2] = u2;
        }
        __syncthreads();
        if (t == 0) {
            double A = 0.0, Mx = 0.0, U2 = 0.0;
            for (int k = 0; k < kClThreads / 32; ++k) {
                A += wred[k][0];
                Mx = (Mx != Mx || Mx > wred[k][1]) ? Mx : wred[k][1];
                U2 += wred[k][2];
            }
            red[0] = A;
            red[1] = Mx;
            red[2] = U2;
        }
        cl.sync();
        if (t == 0) {
            double A = 0.0, Mx = 0.0, U2 = 0.0;
            for (int k = 0; k < C; ++k) {
                const double *rk = cl.map_shared_rank(red, k);
                A += rk[0];
                Mx = (Mx != Mx || Mx > rk[1]) ? Mx : rk[1];
                U2 += rk[2];
            }
            const double rn = sqrt(A), un = sqrt(U2);
            rho = bn > 0.0 ? rn / bn : rn;
            rinf = bmax > 0.0 ? Mx / bmax : Mx;
            fl = bn > 0.0 ? eps * a.S * un / bn : eps * a.S * un;
            int st = -1;
            if (rho <= a.tol) st = CJ_OK;
            else if (!(rho == rho) || rho > 1e300) st = CJ_ERR_DIVERGED;
            else if (rho <= 4.0 * fl) st = CJ_FLOOR;
            else if (cycles > 0) {
                if (a.method == CJ_JACOBI) {
                    if (rho >= prev) st = CJ_STALLED;
                } else {
                    stall = rho > 0.5 * prev ? stall + 1 : 0;
                    if (stall >= 1) st = CJ_STALLED;
                }
            }
            if (st == -1 && sweeps + a.M > a.max_sweeps) st = CJ_ERR_NOT_CONVERGED;
            red[3] = (double)st;
        }
        __syncthreads();
        status = (int)red[3];
        cl.sync();  // every CTA has read the triples before any CTA writes new ones
        if (status != -1) break;
        prev = rho;
        constexpr int R = ST == 17 ? 2 : 1;
        const int nbt = R < nr ? R : nr, nbb = R < nr - nbt ? R : nr - nbt;  // boundary rows
        for (long long n = 0; n < a.M; ++n) {
            const double w = a.w[n];
            const double *Ui = cur ? buf1 : buf0;
            double *Uo = cur ? buf0 : buf1;
            double *up_base = nullptr, *dn_base = nullptr;  // ghost rows of the neighbours' Uo
            if (c > 0) {
                int pr0, pnr;
                cl_band(Ny, C, c - 1, pr0, pnr);
                up_base = cl.map_shared_rank(Uo, c - 1) + (long long)(pnr + 2) * W;
            }
            if (c < C - 1) dn_base = cl.map_shared_rank(Uo, c + 1);
            // node (q, x) of the new buffer; the first and last R rows also go to the neighbours'
            // ghost rows: my rows 2 .. R+1 are rows pnr+2 .. of the CTA above (rank c-1), my rows
            // nr-R+2 .. nr+1 are rows 2-R .. 1 of the CTA below (rank c+1)
            auto node = [&](int q, int x) {
                auto U = [&](int di, int dj) { return Ui[(long long)(q + dj) * W + x + di]; };
                const double v = fma(w, resid_direct<ST, double>(U, bs[(long long)(q - 2) * Nx + x - 2]), U(0, 0));
                Uo[(long long)q * W + x] = v;
                double *up = nullptr, *dn = nullptr;
                if (c > 0 && q < 2 + R) up = up_base + (long long)(q - 2) * W;
                if (c < C - 1 && q > nr + 1 - R) dn = dn_base + (long long)(q - nr) * W;
                if (up) up[x] = v;
                if (dn) dn[x] = v;
                if (ST == 17 && a.mirror) {  // store_node's reflection rule, in band coordinates
                    const int i = x - 1, j = r0 + q - 2;
                    const double nv = -v;
                    if (i == 1) {
                        Uo[(long long)q * W + 0] = nv;
                        if (up) up[0] = nv;
                        if (dn) dn[0] = nv;
                    }
                    if (i == Nx) {
                        Uo[(long long)q * W + Nx + 3] = nv;
                        if (up) up[Nx + 3] = nv;
                        if (dn) dn[Nx + 3] = nv;
                    }
                    if (j == 1) {
                        Uo[(long long)(q - 2) * W + x] = nv;
                        if (i == 1) Uo[(long long)(q - 2) * W + 0] = v;
                        if (i == Nx) Uo[(long long)(q - 2) * W + Nx + 3] = v;
                    }
                    if (j == Ny) {
                        Uo[(long long)(q + 2) * W + x] = nv;
                        if (i == 1) Uo[(long long)(q + 2) * W + 0] = v;
                        if (i == Nx) Uo[(long long)(q + 2) * W + Nx + 3] = v;
                    }
                }
            };
            // the rows the neighbours need first (rows 2 .. 1+nbt and nr+2-nbb .. nr+1), then the
            // arrive half of the cluster barrier, the interior rows while the others arrive, and
            // the wait half: the interior rows read no ghost row, so a neighbour still finishing
            // them is never disturbed by the next sweep's stores into its ghost rows
            // (one index space over the boundary rows, then the interior rows: a thread with no
            // boundary node left arrives at once and starts on the interior, so every thread works
            // while the boundary rows are computed)
            const long long nbn = (long long)(nbt + nbb) * Nx, nall = (long long)nr * Nx;
            long long k = t;
            for (; k < nbn; k += kClThreads) {
                const int row = (int)(k / Nx), x = (int)(k % Nx) + 2;
                node(row < nbt ? 2 + row : nr + 2 - nbb + (row - nbt), x);
            }
            asm volatile("barrier.cluster.arrive.release;\n" ::: "memory");
            for (; k < nall; k += kClThreads) {
                const long long ki = k - nbn;
                node(2 + nbt + (int)(ki / Nx), (int)(ki % Nx) + 2);
            }
            __syncthreads();  // the interior rows, written after the arrive, for the next sweep
            asm volatile("barrier.cluster.wait.acquire;\n" ::: "memory");
            cur ^= 1;
        }
        sweeps += a.M;
        cycles += 1;
    }
    // the solution's own rows back to the padded grid
    for (long long k = t; k < (long long)nr * Nx; k += kClThreads) {
        const int q = (int)(k / Nx) + 2, x = (int)(k % Nx) + 2;
        a.u[a.g.idx(x - 1, r0 + q - 2)] = (cur ? buf1 : buf0)[(long long)q * W + x];
    }
    if (c == 0 && t == 0) {
        a.res[0] = (double)status;
        a.res[1] = (double)sweeps;
        a.res[2] = (double)cycles;
        a.res[3] = rho;
        a.res[4] = rinf;
        a.res[5] = fl;
    }
    cl.sync();  // no CTA leaves while another may still read its shared memory
}

void *cl_kernel(int st) {
    return st == 5 ? (void *)cluster_solve_kernel<5> : st == 9 ? (void *)cluster_solve_kernel<9>
                                                                : (void *)cluster_solve_kernel<17>;
}

size_t cl_smem(int Nx, int Ny, int C) {
    const int nr_max = Ny / C + (Ny % C ? 1 : 0);
    return sizeof(double) * (2ULL * (nr_max + 4) * (Nx + 4) + (size_t)nr_max * Nx + 4);
}

}  // namespace

int cluster_solve_size(const cj_plan *p) {
    if (p->precision != CJ_FP64 || p->pattern != 0 || (long long)p->Nx * p->Ny > kClusterMaxNodes) return 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    int cluster_ok = 0;
    if (cudaDeviceGetAttribute(&cluster_ok, cudaDevAttrClusterLaunch, dev) != cudaSuccess || !cluster_ok) return 0;
    void *fn = cl_kernel(p->st);
    // the same values for every plan, so plans of different sizes never undo each other's setting
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess ||
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kClMaxSmem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    for (int C = 16; C >= 1; C /= 2) {
        if (C > 1 && p->Ny < 2 * C) continue;  // every band needs two rows for its neighbours' ghosts
        const size_t smem = cl_smem(p->Nx, p->Ny, C);
        if (smem > kClMaxSmem) continue;
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3(C);
        cfg.blockDim = dim3(kClThreads);
        cfg.dynamicSmemBytes = smem;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = C;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int nclusters = 0;
        if (cudaOccupancyMaxActiveClusters(&nclusters, fn, &cfg) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        if (nclusters >= 1) return C;
    }
    return 0;
}

cudaError_t launch_cluster_solve(const cj_plan *p, double *res_dev, cudaStream_t s) {
    const int C = p->cluster_C;
    ClArgs a;
    a.u = p->u0;
    a.b = p->b;
    a.w = p->w_dev;
    a.res = res_dev;
    a.g = p->g64;
    a.M = p->M;
    a.max_sweeps = p->max_sweeps;
    a.tol = p->tol;
    a.S = p->S;
    a.bstat = p->red + 3;
    a.method = p->method;
    a.mirror = p->bc == CJ_BC_DIRICHLET0;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(C);
    cfg.blockDim = dim3(kClThreads);
    cfg.dynamicSmemBytes = cl_smem(p->Nx, p->Ny, C);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    void *args[] = {(void *)&a};
    return cudaLaunchKernelExC(&cfg, cl_kernel(p->st), args);
}
