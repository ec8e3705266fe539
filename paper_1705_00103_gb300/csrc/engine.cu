// Kernels of the batched / served CJM engine (sm_103a).
//
// Many independent problems of different sizes, stencils and tolerances are solved
// together by the mixed-precision CJM (FP32 inner cycles inside an FP64 or double-FP64
// defect-correction loop).  One engine step is six launches over fixed, persistent grids:
//   correct  -- slots starting an outer step add the last inner cycle's correction to u;
//   defect   -- they form the defect r = b - L u (FP64 or double-FP64), its FP32 copy and
//               per-tile partial norms, and zero the inner iterate;
//   decide   -- per slot: reduce the partials in a fixed order, apply the stop rule on the
//               device, start the next inner cycle or finish the slot;
//   sweep    -- every slot in an inner cycle advances min(depth, left) FP32 sweeps over all
//               of its tiles (one-sweep march4, or temporal blocking; depth-4 slots of 5 and
//               9 points on the register wavefront); a step runs several sweep launches, the
//               q-th reading where the slot stands from the step's starting counter and q,
//               so the per-step launches are spread over more sweeps;
//   export   -- finished slots copy u into the caller's buffer;
//   advance  -- per slot: move the cycle counter and the ping-pong by the step's sweeps,
//               retire exported slots, publish a compact status record for the host.
// The launches read the tile list and the slots' phases from device memory, so a CUDA graph
// of many steps is captured once and replayed unchanged while problems come and go.  No
// kernel waits on another block: every dependency is a kernel boundary.
//
// Per node, every kernel evaluates the same arithmetic, in the same order, as the
// single-problem solver, so a problem's result does not depend on what it is batched with.
#include <mutex>

#include "engine.cuh"
#include "grid_dev.cuh"
#include "march4_dev.cuh"
#include "stencil_dev.cuh"
#include "wave_reg_dev.cuh"

namespace {

constexpr int kEngThreads = 128;  // = kEngTX: one thread per tile column

struct TileRef {
    int slot, i0, j0, i1, j1;  // nodes i0..i1 x j0..j1 (clipped to the grid)
};

__device__ __forceinline__ TileRef tile_ref(const SlotDev &S, int slot, int lt) {
    TileRef t;
    t.slot = slot;
    const int tx = lt % S.ntx, tyi = lt / S.ntx;
    t.i0 = tx * kEngTX + 1;
    t.j0 = tyi * S.ty + 1;
    t.i1 = min(t.i0 + kEngTX - 1, S.Nx);
    t.j1 = min(t.j0 + S.ty - 1, S.Ny);
    return t;
}

// Rows of the wavefront items' row blocks (16 rows of warm-up per block at depth 4).
constexpr int kEngWaveRows = 128;

// Slots whose sweeps run on the register wavefront: 5- and 9-point slots at depth 4 (their inner
// cycles are a multiple of 4 sweeps long: admission runs shorter ones at depth 1).
__device__ __forceinline__ bool eng_wave_slot(const SlotDev &S) {
    return S.depth == 4 && (S.st == 5 || S.st == 9);
}

// Where sweep launch q of a step (0-based) stands for a slot in its inner cycle: the slot's counter
// and ping-pong are those of the step's start (the step's last kernel advances them), launch q
// sweeps k = min(depth, left) sweeps from counter + what the earlier launches swept, and every
// earlier launch that swept flipped the ping-pong once.
struct StepPos {
    long long counter;  // weight index of launch q's first sweep
    int cur;            // its input buffer
    int k;              // sweeps of launch q (0: the cycle is already done)
};

__device__ __forceinline__ StepPos eng_pos(const SlotDev &S, int q) {
    const long long left = S.M_in - S.counter, d = S.depth;
    const long long done = (long long)q * d < left ? (long long)q * d : left;
    const long long busy = (left + d - 1) / d;  // launches with sweeps in this cycle
    const long long lw = q < busy ? q : busy;
    StepPos P;
    P.counter = S.counter + done;
    P.cur = S.cur ^ (int)(lw & 1);
    P.k = (int)(left - done < d ? left - done : d);
    return P;
}

template <int R>
__device__ __forceinline__ void correct_node(SlotDev &S, int i, int j, const float *e) {
    const long long k = S.g64.idx(i, j);
    const double ev = (double)e[S.g32.idx(i, j)];
    if (S.mode == CJ_FP32_INNER_DD) {
        double hi, err, h2, l2;
        two_sum(S.u[k], ev, hi, err);
        two_sum(hi, S.ulo[k] + err, h2, l2);
        store_node<R, double>(S.u, S.g64, i, j, h2);
        store_node<R, double>(S.ulo, S.g64, i, j, l2);
    } else {
        store_node<R, double>(S.u, S.g64, i, j, S.u[k] + ev);
    }
}

__global__ void __launch_bounds__(kEngThreads) eng_correct(EngineDev E) {
    const int n = *E.ntiles;
    for (int t = blockIdx.x; t < n; t += gridDim.x) {
        const int2 ref = E.tiles[t];
        SlotDev &S = E.slots[ref.x];
        if (S.phase != PHASE_OUTER || S.outer == 0) continue;
        const TileRef T = tile_ref(S, ref.x, ref.y);
        const int i = T.i0 + threadIdx.x;
        if (i > T.i1) continue;
        const float *e = S.cur ? S.e1 : S.e0;
        for (int j = T.j0; j <= T.j1; ++j) {
            if (S.st == 17)
                correct_node<2>(S, i, j, e);
            else
                correct_node<1>(S, i, j, e);
        }
    }
}

template <int ST>
__device__ __forceinline__ double defect_value(const SlotDev &S, int i, int j) {
    const double bk = S.b[S.g64.idx(i, j)];
    if (S.mode == CJ_FP32_INNER_DD) return resid_dd<ST>(S.u, S.ulo, S.g64, i, j, bk);
    auto U = [&](int di, int dj) { return S.u[S.g64.idx(i + di, j + dj)]; };
    return resid_direct<ST, double>(U, bk);
}

__global__ void __launch_bounds__(kEngThreads) eng_defect(EngineDev E) {
    const int n = *E.ntiles;
    for (int t = blockIdx.x; t < n; t += gridDim.x) {
        const int2 ref = E.tiles[t];
        SlotDev &S = E.slots[ref.x];
        if (S.phase != PHASE_OUTER) continue;  // uniform over the block
        const TileRef T = tile_ref(S, ref.x, ref.y);
        const int i = T.i0 + threadIdx.x;
        double s2 = 0.0, mx = 0.0, u2 = 0.0;
        if (i <= T.i1) {
            for (int j = T.j0; j <= T.j1; ++j) {
                const double r = S.st == 5 ? defect_value<5>(S, i, j)
                               : S.st == 9 ? defect_value<9>(S, i, j)
                                           : defect_value<17>(S, i, j);
                const double uc = S.u[S.g64.idx(i, j)];
                s2 = fma(r, r, s2);
                mx = fmax(mx, fabs(r));
                u2 = fma(uc, uc, u2);
                S.rt[S.g32.idx(i, j)] = (float)(-r);
                if (S.st == 17)
                    store_node<2, float>(S.e0, S.g32, i, j, 0.0f);
                else
                    S.e0[S.g32.idx(i, j)] = 0.0f;
            }
        }
        // block partials of this tile into the slot's part[3 * lt ..]
        __shared__ double sh[kEngThreads / 32][3];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            s2 += __shfl_down_sync(0xffffffffu, s2, o);
            mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
            u2 += __shfl_down_sync(0xffffffffu, u2, o);
        }
        if ((threadIdx.x & 31) == 0) {
            sh[threadIdx.x >> 5][0] = s2;
            sh[threadIdx.x >> 5][1] = mx;
            sh[threadIdx.x >> 5][2] = u2;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double a = 0.0, m = 0.0, c = 0.0;
            for (int w = 0; w < kEngThreads / 32; ++w) {
                a += sh[w][0];
                m = fmax(m, sh[w][1]);
                c += sh[w][2];
            }
            S.part[3 * (long long)ref.y + 0] = a;
            S.part[3 * (long long)ref.y + 1] = m;
            S.part[3 * (long long)ref.y + 2] = c;
        }
        __syncthreads();
    }
}

// Stop rule of the solver (tol, rounding floor, two consecutive outer steps that fail to halve
// the residual above it, outer-step budget); -1 = continue.
__device__ __forceinline__ int eng_stop(SlotDev &S) {
    if (S.rho <= S.tol) return CJ_OK;
    if (!(S.rho == S.rho) || S.rho > 1e300) return CJ_ERR_DIVERGED;
    if (S.rho <= 4.0 * S.fl) return CJ_FLOOR;
    if (S.outer > 0) {
        S.stall = S.rho > 0.5 * S.prev ? S.stall + 1 : 0;
        if (S.stall >= 2) return CJ_STALLED;
    }
    if (S.outer >= S.max_outer) return CJ_ERR_NOT_CONVERGED;
    return -1;
}

__global__ void __launch_bounds__(kEngThreads) eng_decide(EngineDev E) {
    __shared__ double sa[kEngThreads], sm[kEngThreads], sc[kEngThreads];
    for (int q = blockIdx.x; q < E.max_slots; q += gridDim.x) {
        SlotDev &S = E.slots[q];
        if (S.phase != PHASE_OUTER) continue;
        double a = 0.0, m = 0.0, c = 0.0;
        for (int k = threadIdx.x; k < S.ntiles; k += kEngThreads) {
            a += S.part[3 * (long long)k + 0];
            m = fmax(m, S.part[3 * (long long)k + 1]);
            c += S.part[3 * (long long)k + 2];
        }
        sa[threadIdx.x] = a;
        sm[threadIdx.x] = m;
        sc[threadIdx.x] = c;
        __syncthreads();
        for (int s = kEngThreads / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s) {
                sa[threadIdx.x] += sa[threadIdx.x + s];
                sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + s]);
                sc[threadIdx.x] += sc[threadIdx.x + s];
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            const double bn = sqrt(S.bsq), rn = sqrt(sa[0]), un = sqrt(sc[0]);
            const double eps = S.mode == CJ_FP32_INNER_DD ? 1.2325951644078309e-32 : 1.1102230246251565e-16;
            S.rho = bn > 0.0 ? rn / bn : rn;
            S.rinf = S.bmax > 0.0 ? sm[0] / S.bmax : sm[0];
            S.fl = bn > 0.0 ? eps * S.S * un / bn : eps * S.S * un;
            const int st = eng_stop(S);
            if (st != -1) {
                S.status = st;
                S.phase = PHASE_DONE;
            } else {
                S.prev = S.rho;
                S.counter = 0;
                S.cur = 0;
                S.phase = PHASE_SWEEP;
            }
        }
        __syncthreads();
    }
}

// sweep: one-sweep march for depth 1, temporal blocking otherwise
template <int ST>
__device__ __forceinline__ void sweep_tile(SlotDev &S, const TileRef &T, const StepPos &P, float *sm) {
    const int k = P.k;
    const float *ein = P.cur ? S.e1 : S.e0;
    float *eout = P.cur ? S.e0 : S.e1;
    if (k == 1) {
        // four warps split the tile's rows; each lane takes four adjacent columns (march4)
        const int rows_per_warp = (S.ty + kEngThreads / 32 - 1) / (kEngThreads / 32);
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        const int c0 = T.i0 + 4 * lane;
        const int js = T.j0 + warp * rows_per_warp;
        const int je = min(js + rows_per_warp - 1, T.j1);
        if (c0 > T.i1 || js > je) return;
        M4Store<ST> op{eout, &S.g32, c0, S.w32[P.counter]};
        march4<ST>(ein, S.rt, S.g32, c0, js, je, op);
    } else {
        float w[kTbMaxDepth];
        for (int s = 0; s < k; ++s) w[s] = S.w32[P.counter + s];
        tb_tile<ST>(ein, S.rt, eout, S.g32, k, w, T.i0, T.j0, kEngTX, S.ty, sm);
    }
}

// Sweep launches: tiles whose slot advances one sweep now (k = 1: march4, no shared memory)
// and tiles of temporally blocked slots (k > 1: tb_tile in dynamic shared memory) go to two
// kernels, so that the blocked tiles' shared memory does not lower the occupancy of the rest.
// (64 registers for the one-sweep tiles: 8 blocks per SM stay resident, which measured 1.4x faster on
// the 512-problem batch than the 95-register, 5-blocks-per-SM build)
template <bool BLOCKED>
__global__ void __launch_bounds__(kEngThreads, BLOCKED ? 1 : 8) eng_sweep(EngineDev E, int q) {
    extern __shared__ float sm[];
    const int n = *E.ntiles;
    for (int t = blockIdx.x; t < n; t += gridDim.x) {
        const int2 ref = E.tiles[t];
        SlotDev &S = E.slots[ref.x];
        if (S.phase != PHASE_SWEEP || eng_wave_slot(S)) continue;
        const StepPos P = eng_pos(S, q);
        if (P.k == 0 || (P.k > 1) != BLOCKED) continue;
        const TileRef T = tile_ref(S, ref.x, ref.y);
        if (BLOCKED) __syncthreads();  // the previous tile's shared-memory stage is finished
        if (S.st == 5)
            sweep_tile<5>(S, T, P, sm);
        else if (S.st == 9)
            sweep_tile<9>(S, T, P, sm);
        else
            sweep_tile<17>(S, T, P, sm);
    }
}

// Sweep launches, wavefront part: each warp takes (slot, strip, row block) items of the wave list
// and advances them 4 sweeps (wr_run: the single-grid wavefront's per-warp stage, the same node
// arithmetic, so the results equal one-sweep tiles bit for bit); the tile kernels leave these
// slots alone.
// (one kernel per stencil: both stage bodies in one kernel overflow the instruction cache)
template <int ST>
__global__ void __launch_bounds__(kWrThreads, 2) eng_sweep_wave(EngineDev E, int q) {
    __shared__ float4 ering[kWrWarps][kWrERing][32];
    __shared__ float4 rring[kWrWarps][kWrRRing][32];
    const int wid = (int)threadIdx.x >> 5;
    const int n = *E.nwaves;
    for (int it = (int)blockIdx.x * kWrWarps + wid; it < n; it += (int)gridDim.x * kWrWarps) {
        const int4 w = E.waves[it];
        SlotDev &S = E.slots[w.x];
        if (S.st != ST || S.phase != PHASE_SWEEP || !eng_wave_slot(S)) continue;  // warp-uniform
        const StepPos P = eng_pos(S, q);
        if (P.k != 4) continue;
        WrWeights wt;
#pragma unroll
        for (int k = 0; k < 4; ++k) wt.w[k] = S.w32[P.counter + k];
        const float *ein = P.cur ? S.e1 : S.e0;
        float *eout = P.cur ? S.e0 : S.e1;
        wr_run<ST, 4>(ein, S.rt, eout, S.g32, wt, kEngWaveRows, w.y, w.z, ering[wid][0], rring[wid][0]);
    }
}

__global__ void __launch_bounds__(kEngThreads) eng_export(EngineDev E) {
    const int n = *E.ntiles;
    for (int t = blockIdx.x; t < n; t += gridDim.x) {
        const int2 ref = E.tiles[t];
        SlotDev &S = E.slots[ref.x];
        if (S.phase != PHASE_DONE) continue;
        const TileRef T = tile_ref(S, ref.x, ref.y);
        const int i = T.i0 + threadIdx.x;
        if (i > T.i1) continue;
        for (int j = T.j0; j <= T.j1; ++j)
            S.out[(long long)(j - 1) * S.ld_out + (i - 1)] = S.u[S.g64.idx(i, j)];
    }
}

// Per slot at the end of a step: the step's `launches` sweep launches move the cycle counter and
// the ping-pong (eng_pos), an inner cycle that ended becomes an outer step, exported slots retire,
// and the status records are published.
__global__ void eng_advance(EngineDev E, int launches) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < E.max_slots; q += gridDim.x * blockDim.x) {
        SlotDev &S = E.slots[q];
        if (S.phase == PHASE_SWEEP) {
            const StepPos P = eng_pos(S, launches);  // where a launch after the last would start
            S.sweeps += P.counter - S.counter;
            S.counter = P.counter;
            S.cur = P.cur;
            if (S.counter >= S.M_in) {
                S.phase = PHASE_OUTER;
                S.outer += 1;
            }
        } else if (S.phase == PHASE_DONE) {
            S.phase = PHASE_RETIRED;
        }
        SlotStatus st;
        st.phase = S.phase;
        st.status = S.status;
        st.sweeps = S.sweeps;
        st.outer = S.outer;
        st.rho = S.rho;
        st.rinf = S.rinf;
        st.fl = S.fl;
        E.status[q] = st;
    }
}

// admission: b = h^2 f, u = u0 with its reflection ghosts, partial (sum b^2, max|b|)
__global__ void __launch_bounds__(kEngThreads) eng_import(EngineDev E, int slot, int ntiles,
                                                          const double *f, long long ldf,
                                                          const double *u0, long long ldu) {
    SlotDev &S = E.slots[slot];
    for (int lt = blockIdx.x; lt < ntiles; lt += gridDim.x) {
        const TileRef T = tile_ref(S, slot, lt);
        const int i = T.i0 + threadIdx.x;
        double s = 0.0, m = 0.0;
        if (i <= T.i1) {
            for (int j = T.j0; j <= T.j1; ++j) {
                const double bk = S.h2 * f[(long long)(j - 1) * ldf + (i - 1)];
                S.b[S.g64.idx(i, j)] = bk;
                s = fma(bk, bk, s);
                m = fmax(m, fabs(bk));
                const double uv = u0[(long long)(j - 1) * ldu + (i - 1)];
                if (S.st == 17)
                    store_node<2, double>(S.u, S.g64, i, j, uv);
                else
                    S.u[S.g64.idx(i, j)] = uv;
            }
        }
        __shared__ double sh[kEngThreads / 32][2];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            s += __shfl_down_sync(0xffffffffu, s, o);
            m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
        }
        if ((threadIdx.x & 31) == 0) {
            sh[threadIdx.x >> 5][0] = s;
            sh[threadIdx.x >> 5][1] = m;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double a = 0.0, mm = 0.0;
            for (int w = 0; w < kEngThreads / 32; ++w) {
                a += sh[w][0];
                mm = fmax(mm, sh[w][1]);
            }
            S.part[3 * (long long)lt + 0] = a;
            S.part[3 * (long long)lt + 1] = mm;
            S.part[3 * (long long)lt + 2] = 0.0;
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kEngThreads) eng_admit(EngineDev E, int slot) {
    __shared__ double sa[kEngThreads], sm[kEngThreads];
    SlotDev &S = E.slots[slot];
    double a = 0.0, m = 0.0;
    for (int k = threadIdx.x; k < S.ntiles; k += kEngThreads) {
        a += S.part[3 * (long long)k + 0];
        m = fmax(m, S.part[3 * (long long)k + 1]);
    }
    sa[threadIdx.x] = a;
    sm[threadIdx.x] = m;
    __syncthreads();
    for (int s = kEngThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            sa[threadIdx.x] += sa[threadIdx.x + s];
            sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + s]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        S.bsq = sa[0];
        S.bmax = sm[0];
        S.phase = PHASE_OUTER;
        S.status = CJ_PENDING;
        S.cur = 0;
        S.stall = 0;
        S.counter = 0;
        S.outer = 0;
        S.sweeps = 0;
        S.prev = 0.0;
        S.rho = S.rinf = S.fl = 0.0;
    }
}

}  // namespace

size_t eng_sweep_smem(int max_depth) {
    if (max_depth <= 1) return 0;
    const int H = 2 * max_depth;  // radius 2 covers every stencil
    return (size_t)3 * (kEngTX + 2 * H) * (kEngTYMax + 2 * H) * sizeof(float);
}

bool eng_is_tile_kernel(const void *fn) {
    return fn == (const void *)eng_correct || fn == (const void *)eng_defect || fn == (const void *)eng_sweep<false> ||
           fn == (const void *)eng_sweep<true> || fn == (const void *)eng_export;
}

int eng_sweep_blocks_per_sm() {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, eng_sweep<false>, kEngThreads, 0) != cudaSuccess || n < 1)
        n = 1;
    return n;
}

// The blocked sweep kernel's dynamic shared-memory limit is one attribute of the function, shared by
// every engine in the process (the server's lanes are several): it is only ever raised, so an engine
// created later with a shallower depth never takes it from one that needs it.
cudaError_t eng_prepare(size_t sweep_smem) {
    static std::mutex mu;
    static size_t granted = 0;
    std::lock_guard<std::mutex> lk(mu);
    if (sweep_smem <= granted) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(eng_sweep<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sweep_smem);
    if (e == cudaSuccess) granted = sweep_smem;
    return e;
}

int eng_wave_items(int slot, int Nx, int Ny, int st, int depth, std::vector<int4> &items) {
    if (depth != 4 || (st != 5 && st != 9)) return 0;
    const int nstrips = wr_strips(Nx), nrb = (Ny + kEngWaveRows - 1) / kEngWaveRows;
    for (int rb = 0; rb < nrb; ++rb)
        for (int x = 0; x < nstrips; ++x) items.push_back(make_int4(slot, x, rb, 0));
    return nstrips * nrb;
}

int eng_wave_grid() {
    static const int n = [] {
        int dev = 0, sms = 152, per_sm = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, eng_sweep_wave<9>, kWrThreads, 0) != cudaSuccess ||
            per_sm < 1)
            per_sm = 1;
        return sms * per_sm;
    }();
    return n;
}

cudaError_t eng_launch_step(const EngineDev &e, int grid_tiles, int grid_slots, size_t sweep_smem,
                            int sweeps, int wave_grid, cudaStream_t s) {
    const int grid_adv = (e.max_slots + 127) / 128;
    eng_correct<<<grid_tiles, kEngThreads, 0, s>>>(e);
    eng_defect<<<grid_tiles, kEngThreads, 0, s>>>(e);
    eng_decide<<<grid_slots, kEngThreads, 0, s>>>(e);
    for (int q = 0; q < sweeps; ++q) {
        eng_sweep<false><<<grid_tiles, kEngThreads, 0, s>>>(e, q);
        if (sweep_smem > 0) eng_sweep<true><<<grid_tiles, kEngThreads, sweep_smem, s>>>(e, q);
        if (wave_grid > 0) {
            eng_sweep_wave<5><<<wave_grid, kWrThreads, 0, s>>>(e, q);
            eng_sweep_wave<9><<<wave_grid, kWrThreads, 0, s>>>(e, q);
        }
    }
    eng_export<<<grid_tiles, kEngThreads, 0, s>>>(e);
    eng_advance<<<grid_adv, 128, 0, s>>>(e, sweeps);
    return cudaGetLastError();
}

cudaError_t eng_launch_import(const EngineDev &e, int slot, int ntiles, const double *f,
                              long long ldf, const double *u0, long long ldu, cudaStream_t s) {
    int grid = ntiles < 1024 ? ntiles : 1024;
    eng_import<<<grid, kEngThreads, 0, s>>>(e, slot, ntiles, f, ldf, u0, ldu);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    eng_admit<<<1, kEngThreads, 0, s>>>(e, slot);
    return cudaGetLastError();
}
