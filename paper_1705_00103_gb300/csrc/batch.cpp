// Host side of the batched / served CJM engine: slot admission (plan math, device memory,
// import), the captured CUDA graph of engine steps, completion polling, and the C ABI of
// cj_solve_batch and of the request server (cj_server_* / cj_submit / cj_poll).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstddef>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "engine.cuh"

namespace {

// FP32 sweep launches per engine step, and steps per captured graph: a replay advances a slot by
// up to 32 sweeps, as with one sweep per step and 32 steps, with fewer launches per sweep
// (measured: 4 sweeps per step 5.68 s for the 512-problem batch, 8: 5.52 s, 16: 5.45 s).
constexpr int kSweepsPerStep = 8;
// Shorter side from which 5- and 9-point problems sweep on the register wavefront by default.
constexpr int kEngWaveMinSide = 512;

using Clock = std::chrono::steady_clock;

#define ENG_TRY(call, where)                \
    do {                                    \
        cudaError_t e_ = (call);            \
        if (e_ != cudaSuccess) {            \
            set_cuda_error(e_, where);      \
            return CJ_ERR_CUDA;             \
        }                                   \
    } while (0)

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// What a slot needs besides its device state: the allocation behind it.
struct SlotMem {
    char *base = nullptr;
    size_t bytes = 0;
};

struct Spec {
    int Nx, Ny, st, mode, inner_cycle, depth, ty;
    double tol;
    long long max_sweeps;
};

// Device bytes a problem occupies in the engine (FP64 u, b [, u_lo], FP32 e0, e1, rt,
// weights, partials).
size_t slot_bytes(const Spec &sp, long long M_in) {
    const Grid g64 = make_grid(sp.Nx, sp.Ny, 8), g32 = make_grid(sp.Nx, sp.Ny, 4);
    const long long ntiles = (long long)((sp.Nx + kEngTX - 1) / kEngTX) * ((sp.Ny + sp.ty - 1) / sp.ty);
    size_t n = 0;
    n += align256(g64.elems() * 8) * (sp.mode == CJ_FP32_INNER_DD ? 3 : 2);
    n += align256(g32.elems() * 4) * 3;
    n += align256((size_t)M_in * 4);
    n += align256((size_t)ntiles * 3 * 8);
    return n;
}

class Engine {
  public:
    ~Engine() { destroy(); }

    // priority_rank 0 = the device's default stream priority; k > 0 = k levels above it
    // (clamped to the device's range): a lane of small requests is scheduled ahead of the others.
    // tile_grid: launch the tile kernels with one block per tile of the current tile list (the
    // captured graph's grids are updated when the list changes) instead of 8 blocks per SM that
    // stride over it; short-lived blocks let another stream's higher-priority kernels onto the SMs
    // within microseconds, where resident striding blocks would hold them for a whole launch.
    // blocked_depth: the deepest depth of the tiles' shared-memory temporal blocking (17-point slots,
    // depths 2 and 3); -1: max_depth.  Depth-4 slots of 5 and 9 points sweep on the wavefront.
    // wave_share: the share of the SMs' wavefront blocks the wavefront kernel launches (1 = a whole
    // wave; the server's larger lanes leave room for the smaller lanes' blocks).
    cj_status init(int max_slots, int max_depth, int priority_rank = 0, bool tile_grid = false,
                   int blocked_depth = -1, double wave_share = 1.0) {
        if (max_slots < 1 || max_depth < 1 || max_depth > kTbMaxDepth) return CJ_ERR_INVALID_ARG;
        max_slots_ = max_slots;
        max_depth_ = max_depth;
        ENG_TRY(cudaGetDevice(&dev_), "cudaGetDevice");
        int least = 0, greatest = 0;
        ENG_TRY(cudaDeviceGetStreamPriorityRange(&least, &greatest), "stream priorities");
        const int prio = std::max(greatest, least - priority_rank);  // numerically lower = higher
        ENG_TRY(cudaStreamCreateWithPriority(&s_, cudaStreamNonBlocking, prio), "engine stream");
        int sms = 152;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev_);
        grid_tiles_ = sms * 8;
        tile_grid_ = tile_grid;
        grid_slots_ = std::min(max_slots, sms * 4);
        smem_ = eng_sweep_smem(blocked_depth < 0 ? max_depth : blocked_depth);
        wave_ = max_depth >= 4;  // depth-4 slots of 5 and 9 points sweep on the register wavefront
        wave_grid_ = wave_ ? std::max(1, (int)(wave_share * eng_wave_grid())) : 0;
        ENG_TRY(eng_prepare(smem_), "engine smem attribute");
        host_.assign(max_slots, SlotDev{});
        mem_.assign(max_slots, SlotMem{});
        used_.assign(max_slots, 0);
        tiles_off_.assign(max_slots, 0);
        ENG_TRY(cudaMalloc(&d_.slots, sizeof(SlotDev) * max_slots), "engine slots");
        ENG_TRY(cudaMemset(d_.slots, 0, sizeof(SlotDev) * max_slots), "engine slots");
        ENG_TRY(cudaMalloc(&d_.status, sizeof(SlotStatus) * max_slots), "engine status");
        ENG_TRY(cudaMemset(d_.status, 0, sizeof(SlotStatus) * max_slots), "engine status");
        ENG_TRY(cudaMalloc(&d_.ntiles, sizeof(int)), "engine tile count");
        ENG_TRY(cudaMemset(d_.ntiles, 0, sizeof(int)), "engine tile count");
        ENG_TRY(cudaMalloc(&d_.nwaves, sizeof(int)), "engine wave count");
        ENG_TRY(cudaMemset(d_.nwaves, 0, sizeof(int)), "engine wave count");
        wave_cap_ = 0;
        d_.waves = nullptr;
        tile_cap_ = 0;
        d_.tiles = nullptr;
        d_.max_slots = max_slots;
        ENG_TRY(cudaMallocHost(&h_status_, sizeof(SlotStatus) * max_slots), "engine status (host)");
        ENG_TRY(cudaMallocHost(&h_ntiles_, sizeof(int)), "engine tile count (host)");
        ENG_TRY(cudaMallocHost(&h_nwaves_, sizeof(int)), "engine wave count (host)");
        return ensure_tile_capacity(1024);
    }

    void destroy() {
        if (!s_) return;
        cudaSetDevice(dev_);  // the engine's device, whichever thread tears it down
        cudaStreamSynchronize(s_);
        for (int q = 0; q < max_slots_; ++q)
            if (mem_[q].base) cudaFree(mem_[q].base);
        if (gexec_) cudaGraphExecDestroy(gexec_);
        if (graph_) cudaGraphDestroy(graph_);
        cudaFree(d_.slots);
        cudaFree(d_.status);
        cudaFree(d_.ntiles);
        cudaFree(d_.nwaves);
        cudaFree(d_.waves);
        cudaFree(d_.tiles);
        if (h_status_) cudaFreeHost(h_status_);
        if (h_ntiles_) cudaFreeHost(h_ntiles_);
        if (h_nwaves_) cudaFreeHost(h_nwaves_);
        cudaStreamDestroy(s_);
        s_ = nullptr;
    }

    cudaStream_t stream() const { return s_; }
    int free_slots() const { return (int)std::count(used_.begin(), used_.end(), 0); }

    // Plan numbers of a problem: (kmin, kmax, M_in), with the FP64 cycle length as the cap.
    static cj_status plan(const Spec &sp, double *kmin, double *kmax, long long *M_in) {
        plan_kappa_bounds(sp.st, sp.Nx + 1.0, sp.Ny + 1.0, kmin, kmax);
        if (!(*kmin > 0.0 && *kmin < *kmax)) return CJ_ERR_INVALID_ARG;
        const long long M = plan_cycle_length(*kmin, *kmax, sp.tol);
        *M_in = sp.inner_cycle ? sp.inner_cycle : plan_inner_cycle(*kmin, *kmax, M);
        return CJ_OK;
    }

    // Admit a problem into a free slot: f, u0 device grids (u0 may be NULL = zero), out:
    // caller grid for the result.  Enqueued on the engine stream; takes effect at the next
    // run().
    // With out_to_b the result is exported into the interior of the slot's own b buffer
    // (no longer needed once the slot is done), for callers without a device output grid.
    cj_status admit(const Spec &sp, const double *f, long long ldf, const double *u0, long long ldu,
                    double *out, long long ld_out, int *slot_out, bool out_to_b = false) {
        int q = -1;
        for (int k = 0; k < max_slots_; ++k)
            if (!used_[k]) {
                q = k;
                break;
            }
        if (q < 0) return CJ_ERR_BUDGET;
        double kmin, kmax;
        long long M_in;
        cj_status st = plan(sp, &kmin, &kmax, &M_in);
        if (st != CJ_OK) return st;
        const size_t bytes = slot_bytes(sp, M_in);
        char *base = nullptr;
        ENG_TRY(cudaMallocAsync((void **)&base, bytes, s_), "slot memory");
        ENG_TRY(cudaMemsetAsync(base, 0, bytes, s_), "slot memory");
        SlotDev S{};
        S.Nx = sp.Nx;
        S.Ny = sp.Ny;
        S.st = sp.st;
        S.mode = sp.mode;
        // a depth the engine has no shared memory for (an autotuned one in the server, whose
        // engine sweeps one at a time) runs at the engine's maximum
        S.depth = std::min(sp.depth, max_depth_);
        // the wavefront takes 4 sweeps at a time: an inner cycle of 1 or 2 sweeps runs at depth 1
        if (S.depth == 4 && (sp.st == 5 || sp.st == 9) && M_in % 4 != 0) S.depth = 1;
        S.ty = sp.ty;
        S.ntx = (sp.Nx + kEngTX - 1) / kEngTX;
        S.ntiles = S.ntx * ((sp.Ny + sp.ty - 1) / sp.ty);
        S.M_in = M_in;
        const long long max_sweeps = sp.max_sweeps ? sp.max_sweeps : 64 * M_in;
        S.max_outer = max_sweeps / M_in;
        S.tol = sp.tol;
        S.S = plan_abs_coeff_sum(sp.st);
        const double h = 1.0 / (double)(sp.Nx + 1);
        S.h2 = h * h;
        S.g64 = make_grid(sp.Nx, sp.Ny, 8);
        S.g32 = make_grid(sp.Nx, sp.Ny, 4);
        char *p = base;
        const size_t b64 = align256(S.g64.elems() * 8), b32 = align256(S.g32.elems() * 4);
        S.u = (double *)p;
        p += b64;
        S.b = (double *)p;
        p += b64;
        if (sp.mode == CJ_FP32_INNER_DD) {
            S.ulo = (double *)p;
            p += b64;
        }
        S.e0 = (float *)p;
        p += b32;
        S.e1 = (float *)p;
        p += b32;
        S.rt = (float *)p;
        p += b32;
        float *w32 = (float *)p;
        p += align256((size_t)M_in * 4);
        S.part = (double *)p;
        if (out_to_b) {
            S.out = S.b + S.g64.idx(1, 1);
            S.ld_out = S.g64.pitch;
        } else {
            S.out = out;
            S.ld_out = ld_out;
        }
        std::vector<double> w;
        plan_sweep_coeffs(sp.st, kmin, kmax, M_in, w);
        wstage_.assign(w.size(), 0.0f);
        for (size_t k = 0; k < w.size(); ++k) wstage_[k] = (float)w[k];
        S.w32 = w32;
        host_[q] = S;
        ENG_TRY(cudaMemcpyAsync(w32, wstage_.data(), wstage_.size() * 4, cudaMemcpyHostToDevice, s_), "weights");
        ENG_TRY(cudaMemcpyAsync(d_.slots + q, &host_[q], sizeof(SlotDev), cudaMemcpyHostToDevice, s_), "slot upload");
        ENG_TRY(cudaStreamSynchronize(s_), "admit sync");  // host staging buffers reused next time
        const double *u0p = u0;
        if (!u0p) {
            // zero initial guess: the slot's u is already zero; import reads it in place
            u0p = S.u + S.g64.idx(1, 1);
            ldu = S.g64.pitch;
        }
        ENG_TRY(eng_launch_import(d_, q, S.ntiles, f, ldf, u0p, ldu, s_), "import");
        mem_[q].base = base;
        mem_[q].bytes = bytes;
        used_[q] = 1;
        tiles_off_[q] = 0;
        tiles_dirty_ = true;
        *slot_out = q;
        return CJ_OK;
    }

    // Device pointer to the interior of slot q's b buffer and its pitch (elements).
    void b_interior(int q, double **ptr, long long *pitch) const {
        *ptr = host_[q].b + host_[q].g64.idx(1, 1);
        *pitch = host_[q].g64.pitch;
    }

    size_t slot_mem(int q) const { return mem_[q].bytes; }

    // Takes a retired slot's tiles out of the tile list (its memory and status stay): every
    // engine kernel scans the list, so a batch's tail runs only over the slots still working.
    void drop_tiles(int q) {
        if (q >= 0 && q < max_slots_ && used_[q] && !tiles_off_[q]) {
            tiles_off_[q] = 1;
            tiles_dirty_ = true;
        }
    }

    // Frees slot q (after its result has been read).
    cj_status release(int q) {
        if (q < 0 || q >= max_slots_ || !used_[q]) return CJ_ERR_INVALID_ARG;
        const int free_phase = PHASE_FREE;
        ENG_TRY(cudaMemcpyAsync((char *)(d_.slots + q) + offsetof(SlotDev, phase), &free_phase,
                                sizeof(int), cudaMemcpyHostToDevice, s_), "slot release");
        ENG_TRY(cudaFreeAsync(mem_[q].base, s_), "slot free");
        ENG_TRY(cudaStreamSynchronize(s_), "release sync");
        mem_[q] = SlotMem{};
        used_[q] = 0;
        tiles_dirty_ = true;
        return CJ_OK;
    }

    // Runs `replays` graph replays of the engine steps, then refreshes the host status.
    cj_status run(int replays) {
        if (tiles_dirty_) {
            cj_status st = upload_tiles();
            if (st != CJ_OK) return st;
        }
        if (!gexec_) {
            cj_status st = capture();
            if (st != CJ_OK) return st;
        }
        if (tile_grid_) {
            const int want = std::max(1, *h_ntiles_);
            if (want != cur_grid_) {
                cj_status st = set_tile_grid(want);
                if (st != CJ_OK) return st;
            }
        }
        for (int k = 0; k < replays; ++k) ENG_TRY(cudaGraphLaunch(gexec_, s_), "graph launch");
        launches_ += (long long)replays * steps_per_graph_ * (5 + ((smem_ > 0 ? 2 : 1) + (wave_ ? 2 : 0)) * kSweepsPerStep);
        ENG_TRY(cudaMemcpyAsync(h_status_, d_.status, sizeof(SlotStatus) * max_slots_,
                                cudaMemcpyDeviceToHost, s_), "status readback");
        ENG_TRY(cudaStreamSynchronize(s_), "step sync");
        return CJ_OK;
    }

    const SlotStatus &status(int q) const { return h_status_[q]; }
    bool used(int q) const { return used_[q] != 0; }
    long long launches() const { return launches_; }
    int steps_per_graph() const { return steps_per_graph_; }

  private:
    cj_status ensure_tile_capacity(int n) {
        if (n <= tile_cap_) return CJ_OK;
        int cap = std::max(n, 2 * tile_cap_);
        int2 *t = nullptr;
        ENG_TRY(cudaMalloc(&t, sizeof(int2) * cap), "tile table");
        cudaFree(d_.tiles);
        d_.tiles = t;
        tile_cap_ = cap;
        if (gexec_) {  // the graph bakes the table pointer in: capture again
            cudaGraphExecDestroy(gexec_);
            gexec_ = nullptr;
            cudaGraphDestroy(graph_);
            graph_ = nullptr;
        }
        return CJ_OK;
    }

    cj_status upload_tiles() {
        tiles_.clear();
        waves_.clear();
        for (int q = 0; q < max_slots_; ++q)
            if (used_[q] && !tiles_off_[q]) {
                for (int t = 0; t < host_[q].ntiles; ++t) tiles_.push_back(make_int2(q, t));
                if (wave_) eng_wave_items(q, host_[q].Nx, host_[q].Ny, host_[q].st, host_[q].depth, waves_);
            }
        cj_status st = ensure_tile_capacity((int)tiles_.size() + 1);
        if (st != CJ_OK) return st;
        st = ensure_wave_capacity((int)waves_.size() + 1);
        if (st != CJ_OK) return st;
        *h_ntiles_ = (int)tiles_.size();
        *h_nwaves_ = (int)waves_.size();
        if (!tiles_.empty())
            ENG_TRY(cudaMemcpyAsync(d_.tiles, tiles_.data(), sizeof(int2) * tiles_.size(),
                                    cudaMemcpyHostToDevice, s_), "tile upload");
        if (!waves_.empty())
            ENG_TRY(cudaMemcpyAsync(d_.waves, waves_.data(), sizeof(int4) * waves_.size(),
                                    cudaMemcpyHostToDevice, s_), "wave upload");
        ENG_TRY(cudaMemcpyAsync(d_.ntiles, h_ntiles_, sizeof(int), cudaMemcpyHostToDevice, s_), "tile count");
        ENG_TRY(cudaMemcpyAsync(d_.nwaves, h_nwaves_, sizeof(int), cudaMemcpyHostToDevice, s_), "wave count");
        ENG_TRY(cudaStreamSynchronize(s_), "tile sync");
        tiles_dirty_ = false;
        return CJ_OK;
    }

    cj_status ensure_wave_capacity(int n) {
        if (n <= wave_cap_) return CJ_OK;
        int cap = std::max(n, 2 * wave_cap_);
        int4 *t = nullptr;
        ENG_TRY(cudaMalloc(&t, sizeof(int4) * cap), "wave table");
        cudaFree(d_.waves);
        d_.waves = t;
        wave_cap_ = cap;
        if (gexec_) {  // the graph bakes the table pointer in: capture again
            cudaGraphExecDestroy(gexec_);
            gexec_ = nullptr;
            cudaGraphDestroy(graph_);
            graph_ = nullptr;
        }
        return CJ_OK;
    }

    cj_status capture() {
        cudaGraph_t g = nullptr;
        ENG_TRY(cudaStreamBeginCapture(s_, cudaStreamCaptureModeThreadLocal), "begin capture");
        cudaError_t err = cudaSuccess;
        for (int k = 0; k < steps_per_graph_ && err == cudaSuccess; ++k)
            err = eng_launch_step(d_, grid_tiles_, grid_slots_, smem_, kSweepsPerStep, wave_grid_, s_);
        cudaError_t e2 = cudaStreamEndCapture(s_, &g);
        if (err == cudaSuccess) err = e2;
        if (err == cudaSuccess) err = cudaGraphInstantiate(&gexec_, g, 0);
        tile_nodes_.clear();
        cur_grid_ = grid_tiles_;
        if (err == cudaSuccess && tile_grid_) {  // the nodes whose grid follows the tile list
            size_t n = 0;
            err = cudaGraphGetNodes(g, nullptr, &n);
            std::vector<cudaGraphNode_t> nodes(n);
            if (err == cudaSuccess && n) err = cudaGraphGetNodes(g, nodes.data(), &n);
            for (size_t k = 0; k < n && err == cudaSuccess; ++k) {
                cudaGraphNodeType type;
                err = cudaGraphNodeGetType(nodes[k], &type);
                if (err != cudaSuccess || type != cudaGraphNodeTypeKernel) continue;
                cudaKernelNodeParams kp{};
                err = cudaGraphKernelNodeGetParams(nodes[k], &kp);
                if (err == cudaSuccess && eng_is_tile_kernel(kp.func)) tile_nodes_.push_back(nodes[k]);
            }
        }
        if (err == cudaSuccess) {
            graph_ = g;  // kept: the tile kernels' nodes are updated through it
        } else if (g) {
            cudaGraphDestroy(g);
        }
        ENG_TRY(err, "graph capture");
        return CJ_OK;
    }

    // Every tile kernel of the instantiated graph launches `blocks` blocks from now on.
    cj_status set_tile_grid(int blocks) {
        for (cudaGraphNode_t node : tile_nodes_) {
            cudaKernelNodeParams kp{};
            ENG_TRY(cudaGraphKernelNodeGetParams(node, &kp), "tile node params");
            kp.gridDim = dim3((unsigned)blocks);
            ENG_TRY(cudaGraphExecKernelNodeSetParams(gexec_, node, &kp), "tile grid update");
        }
        cur_grid_ = blocks;
        return CJ_OK;
    }

    int dev_ = 0, max_slots_ = 0, max_depth_ = 1, grid_tiles_ = 0, grid_slots_ = 0;
    int steps_per_graph_ = 4;
    size_t smem_ = 0;
    cudaStream_t s_ = nullptr;
    EngineDev d_{};
    std::vector<SlotDev> host_;
    std::vector<SlotMem> mem_;
    std::vector<char> used_, tiles_off_;
    std::vector<int2> tiles_;
    std::vector<int4> waves_;
    int wave_cap_ = 0;
    int *h_nwaves_ = nullptr;
    std::vector<float> wstage_;
    int tile_cap_ = 0;
    bool tiles_dirty_ = true;
    SlotStatus *h_status_ = nullptr;
    int *h_ntiles_ = nullptr;
    cudaGraphExec_t gexec_ = nullptr;
    cudaGraph_t graph_ = nullptr;
    bool tile_grid_ = false, wave_ = false;
    int wave_grid_ = 0;
    std::vector<cudaGraphNode_t> tile_nodes_;
    int cur_grid_ = 0;
    long long launches_ = 0;
};

// Precision a request gets when it does not name one: FP64 outer steps unless the FP64
// rounding floor of the relative residual (about 2^-53 S / (c kmin)) comes within 4x of
// the tolerance, then double-FP64.
int auto_mode(int st, int Nx, int Ny, double tol) {
    double kmin, kmax;
    plan_kappa_bounds(st, Nx + 1.0, Ny + 1.0, &kmin, &kmax);
    const double fl = 1.1102230246251565e-16 * plan_abs_coeff_sum(st) / (plan_centre(st) * kmin);
    return 4.0 * fl > tol ? CJ_FP32_INNER_DD : CJ_FP32_INNER;
}

// Engine tile rows and temporal depth per (stencil, size class) recorded by
// cj_autotune_engine; 0 = not tuned (tile rows 32, depth 1).
struct EngineTune {
    int ty, depth;
};
std::mutex g_engine_tune_mu;
EngineTune g_engine_tune[3][32] = {};

EngineTune engine_tuned(int st, int Nx, int Ny) {
    std::lock_guard<std::mutex> lk(g_engine_tune_mu);
    return g_engine_tune[stencil_slot(st)][size_class(Nx, Ny)];
}

cj_status check_problem(const cj_problem &pr) {
    if (pr.Nx < 1 || pr.Ny < 1 || pr.Nx > (1 << 20) || pr.Ny > (1 << 20)) return CJ_ERR_INVALID_ARG;
    if (pr.st != CJ_ST5 && pr.st != CJ_ST9 && pr.st != CJ_ST17) return CJ_ERR_INVALID_ARG;
    if (!(pr.tol > 0.0 && pr.tol < 1.0)) return CJ_ERR_INVALID_ARG;
    if (pr.precision != 0 && pr.precision != CJ_FP32_INNER && pr.precision != CJ_FP32_INNER_DD)
        return CJ_ERR_INVALID_ARG;
    if (pr.inner_cycle < 0 || (pr.inner_cycle & (pr.inner_cycle - 1)) != 0) return CJ_ERR_INVALID_ARG;
    if (pr.temporal_depth < 0 || pr.temporal_depth > kTbMaxDepth) return CJ_ERR_INVALID_ARG;
    if (!pr.f || !pr.u || pr.ld_f < pr.Nx || pr.ld_u < pr.Nx) return CJ_ERR_INVALID_ARG;
    return CJ_OK;
}

// Default depth of a problem the autotuner has not seen: the register wavefront (depth 4) for 5-
// and 9-point problems whose shorter side is at least kEngWaveMinSide, else one sweep at a time.
int default_depth(int st, int Nx, int Ny) {
    return (st == CJ_ST5 || st == CJ_ST9) && std::min(Nx, Ny) >= kEngWaveMinSide ? 4 : 1;
}

Spec spec_of(const cj_problem &pr) {
    Spec sp;
    sp.Nx = pr.Nx;
    sp.Ny = pr.Ny;
    sp.st = pr.st;
    sp.tol = pr.tol;
    sp.mode = pr.precision ? pr.precision : auto_mode(pr.st, pr.Nx, pr.Ny, pr.tol);
    sp.inner_cycle = pr.inner_cycle;
    EngineTune t = engine_tuned(pr.st, pr.Nx, pr.Ny);
    sp.depth = pr.temporal_depth ? pr.temporal_depth : (t.depth ? t.depth : default_depth(pr.st, pr.Nx, pr.Ny));
    sp.ty = t.ty ? t.ty : kEngTYDefault;
    sp.max_sweeps = pr.max_sweeps;
    return sp;
}

void fill_result(const SlotStatus &st, cj_result *r) {
    r->sweeps = st.sweeps;
    r->cycles = (int)st.outer;
    r->status = st.status;
    r->rel_res_l2 = st.rho;
    r->rel_res_inf = st.rinf;
    r->floor_est = st.fl;
}

}  // namespace

// ------------------------------------------------------------------ request server

// Size lanes of the server: requests of up to kLaneNodes[k] nodes (and more than the previous
// lane's) run in lane k, an engine of its own on its own stream, driven by its own worker
// thread, so a small request's engine replays sweep only small grids and its latency follows
// its own work rather than the largest grids on the device.  Smaller lanes' streams have higher
// priority.  Admission stays by footprint against the one shared budget, in arrival order
// within a lane.
constexpr int kLanes = 3;
// Share of a wave of wavefront blocks the larger lanes launch (one block per SM of the two that fit).
constexpr double kServerWaveShare = 0.5;
constexpr long long kLaneNodes[kLanes] = {1LL << 20, 1LL << 23, 1LL << 62};
// Every lane launches its tile kernels with one block per tile (Engine::init's tile_grid): with
// blocks that live a few microseconds, the block scheduler puts the smaller lanes' higher-priority
// blocks on the SMs as soon as any block retires, while each lane still fills the device when it
// runs alone.
// The two larger lanes also hold their next graph replay while the smallest lane has requests on
// the device, so its short-lived kernels find the SMs free instead of sharing them with the larger
// lanes' blocks; a replay is 32 sweeps of a lane's slots, so at most one replay of each larger
// lane is in flight when a small request arrives.  (Holding the largest lane for the middle one
// as well raised the p99 latency and lowered the throughput more, for no lower p50.)  The hold is
// paid from an allowance per lane: it starts at kYieldCapS seconds, refills at kYieldRate seconds
// per second and never exceeds kYieldCapS, so under a sustained stream of small requests a larger
// lane still runs at least 1 - kYieldRate of the time.  Only the order in which the lanes'
// replays reach the GPU changes: every request's arithmetic is the same.
constexpr double kYieldCapS = 1.0;
constexpr double kYieldRate = 0.5;

int lane_of(const Spec &sp) {
    const long long n = (long long)sp.Nx * sp.Ny;
    int k = 0;
    while (k < kLanes - 1 && n > kLaneNodes[k]) ++k;
    return k;
}

struct cj_server {
    struct Request {
        uint64_t ticket;
        Spec sp;
        std::vector<double> f;     // host copy of the right-hand side
        std::vector<double> u;     // host result
        int slot = -1, lane = 0;
        size_t bytes = 0;
        int state = 0;             // 0 queued, 1 running, 2 done
        cj_status rc = CJ_PENDING;
        cj_result res{};
        Clock::time_point t_submit, t_admit, t_done;
    };

    // Pinned staging buffer of each lane: request data crosses the bus through it in chunks on
    // the lane's stream, so a large request's copies neither stage through the driver's pageable
    // path nor hold up the other lanes' work.
    static constexpr size_t kStageBytes = (size_t)16 << 20;

    struct Lane {
        Engine eng;
        std::deque<uint64_t> queue;
        std::map<int, uint64_t> by_slot;
        std::thread worker;
        char *stage = nullptr;
        double allowance = kYieldCapS;  // seconds this lane may still hold for smaller lanes
        Clock::time_point refilled{};
        ~Lane() {
            if (stage) cudaFreeHost(stage);
        }
    };

    Lane lanes[kLanes];
    size_t budget = 0, in_use = 0;
    int max_slots = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::map<uint64_t, Request> reqs;
    uint64_t next_ticket = 1;
    bool stop = false;
    cj_status fatal = CJ_OK;
    int device = 0;
    long long steps = 0, admitted = 0, completed = 0, peak_active = 0;
    size_t peak_bytes = 0;

    long long active_all() const {
        long long n = 0;
        for (const Lane &L : lanes) n += (long long)L.by_slot.size();
        return n;
    }

    long long queued_all() const {
        long long n = 0;
        for (const Lane &L : lanes) n += (long long)L.queue.size();
        return n;
    }

    bool small_lane_busy() const { return !lanes[0].by_slot.empty(); }

    // Before a replay of a larger lane: waits while the smallest lane has requests on the device,
    // as long as the lane's allowance lasts (the caller holds mu through lk).
    void hold_for_small_lane(int lane, std::unique_lock<std::mutex> &lk) {
        Lane &L = lanes[lane];
        const Clock::time_point now = Clock::now();
        if (L.refilled == Clock::time_point{}) L.refilled = now;
        L.allowance = std::min(kYieldCapS,
                               L.allowance + kYieldRate * std::chrono::duration<double>(now - L.refilled).count());
        L.refilled = now;
        if (L.allowance <= 0.0 || !small_lane_busy()) return;
        const auto until = now + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(L.allowance));
        cv.wait_until(lk, until, [&] { return stop || !small_lane_busy(); });
        const double waited = std::chrono::duration<double>(Clock::now() - now).count();
        L.allowance -= waited;
    }

    // Marks every running request of lane L failed (after a CUDA error of its engine).
    void fail_lane(Lane &L) {
        fatal = CJ_ERR_CUDA;
        for (auto &kv : L.by_slot) {
            Request &r = reqs[kv.second];
            r.state = 2;
            r.rc = CJ_ERR_CUDA;
            in_use -= r.bytes;
        }
        L.by_slot.clear();
        cv.notify_all();
    }

    void loop(int lane) {
        cudaSetDevice(device);
        Lane &L = lanes[lane];
        for (;;) {
            std::vector<uint64_t> admit_now;
            {
                std::unique_lock<std::mutex> lk(mu);
                cv.wait(lk, [&] { return stop || !L.queue.empty() || !L.by_slot.empty(); });
                if (stop) return;
                // admission by footprint and free slots, in arrival order
                while (!L.queue.empty()) {
                    Request &r = reqs[L.queue.front()];
                    double kmin, kmax;
                    long long M_in;
                    if (Engine::plan(r.sp, &kmin, &kmax, &M_in) != CJ_OK) {
                        r.state = 2;
                        r.rc = CJ_ERR_INVALID_ARG;
                        L.queue.pop_front();
                        continue;
                    }
                    const size_t need = slot_bytes(r.sp, M_in);
                    if (need > budget) {
                        r.state = 2;
                        r.rc = CJ_ERR_BUDGET;
                        L.queue.pop_front();
                        continue;
                    }
                    if (in_use + need > budget || (int)(L.by_slot.size() + admit_now.size()) >= max_slots)
                        break;
                    r.bytes = need;
                    in_use += need;
                    admit_now.push_back(L.queue.front());
                    L.queue.pop_front();
                }
            }
            for (uint64_t t : admit_now) {
                Request *r;
                {
                    std::lock_guard<std::mutex> lk(mu);
                    r = &reqs[t];
                }
                cj_status st = admit(L, *r);
                std::lock_guard<std::mutex> lk(mu);
                if (st != CJ_OK) {
                    r->state = 2;
                    r->rc = st;
                    in_use -= r->bytes;
                    if (st == CJ_ERR_CUDA) fatal = st;
                    cv.notify_all();
                } else {
                    r->state = 1;
                    r->t_admit = Clock::now();
                    L.by_slot[r->slot] = t;
                    ++admitted;
                    peak_active = std::max<long long>(peak_active, active_all());
                    peak_bytes = std::max(peak_bytes, in_use);
                }
            }
            bool active;
            {
                std::unique_lock<std::mutex> lk(mu);
                if (lane > 0 && !L.by_slot.empty()) hold_for_small_lane(lane, lk);
                if (stop) return;
                active = !L.by_slot.empty();
            }
            if (!active) continue;
            if (L.eng.run(1) != CJ_OK) {
                std::lock_guard<std::mutex> lk(mu);
                fail_lane(L);
                return;
            }
            std::vector<std::pair<int, uint64_t>> done;
            {
                std::lock_guard<std::mutex> lk(mu);
                steps += L.eng.steps_per_graph();
                for (auto &kv : L.by_slot)
                    if (L.eng.status(kv.first).phase == PHASE_RETIRED) done.push_back(kv);
            }
            // release finished problems
            for (auto &d : done) {
                Request *r;
                {
                    std::lock_guard<std::mutex> lk(mu);
                    r = &reqs[d.second];
                }
                const SlotStatus &ss = L.eng.status(d.first);
                double *bin;
                long long pitch;
                L.eng.b_interior(d.first, &bin, &pitch);
                std::vector<double> u((size_t)r->sp.Nx * r->sp.Ny, 0.0);
                cudaError_t e = download(L, u.data(), bin, pitch, r->sp.Nx, r->sp.Ny);
                cj_result res{};
                fill_result(ss, &res);
                L.eng.release(d.first);
                std::lock_guard<std::mutex> lk(mu);
                r->u.swap(u);
                r->res = res;
                r->t_done = Clock::now();
                r->res.seconds = std::chrono::duration<double>(r->t_done - r->t_submit).count();
                r->res.sweep_seconds = std::chrono::duration<double>(r->t_done - r->t_admit).count();
                r->rc = e != cudaSuccess ? CJ_ERR_CUDA : (cj_status)ss.status;
                r->state = 2;
                in_use -= r->bytes;
                L.by_slot.erase(d.first);
                ++completed;
                cv.notify_all();
            }
        }
    }

    // Stages f on the device, admits the request, and points its result at the slot's own b
    // interior (read back by the worker when the slot retires).
    // Host -> device of n bytes through the lane's staging buffer (whole rows of nothing: a flat copy).
    cudaError_t upload(Lane &L, void *dst, const void *src, size_t n) {
        for (size_t off = 0; off < n; off += kStageBytes) {
            const size_t k = std::min(kStageBytes, n - off);
            std::memcpy(L.stage, (const char *)src + off, k);
            cudaError_t e = cudaMemcpyAsync((char *)dst + off, L.stage, k, cudaMemcpyHostToDevice, L.eng.stream());
            if (e == cudaSuccess) e = cudaStreamSynchronize(L.eng.stream());  // before the buffer is reused
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }

    // Device (Ny rows of Nx doubles, row pitch `pitch` elements) -> host (dense) through the staging
    // buffer, a band of whole rows at a time.
    cudaError_t download(Lane &L, double *dst, const double *src, long long pitch, int Nx, int Ny) {
        const size_t row = (size_t)Nx * 8;
        const int band = (int)std::max<size_t>(1, kStageBytes / row);
        for (int j = 0; j < Ny; j += band) {
            const int rows = std::min(band, Ny - j);
            cudaError_t e = cudaMemcpy2DAsync(L.stage, row, src + (size_t)j * pitch, (size_t)pitch * 8, row, rows,
                                              cudaMemcpyDeviceToHost, L.eng.stream());
            if (e == cudaSuccess) e = cudaStreamSynchronize(L.eng.stream());
            if (e != cudaSuccess) return e;
            std::memcpy(dst + (size_t)j * Nx, L.stage, row * rows);
        }
        return cudaSuccess;
    }

    cj_status admit(Lane &L, Request &r) {
        Engine &eng = L.eng;
        double *fd = nullptr;
        const size_t fbytes = (size_t)r.sp.Nx * r.sp.Ny * 8;
        ENG_TRY(cudaMallocAsync((void **)&fd, fbytes, eng.stream()), "request f");
        ENG_TRY(upload(L, fd, r.f.data(), fbytes), "request H2D");
        int slot = -1;
        cj_status st = eng.admit(r.sp, fd, r.sp.Nx, nullptr, 0, nullptr, 0, &slot, true);
        cudaError_t e = cudaFreeAsync(fd, eng.stream());
        if (st == CJ_OK && e != cudaSuccess) {
            set_cuda_error(e, "request f free");
            st = CJ_ERR_CUDA;
        }
        r.slot = slot;
        std::vector<double>().swap(r.f);
        return st;
    }
};

// ------------------------------------------------------------------ C ABI

extern "C" {

cj_status cj_solve_batch(const cj_problem *problems, int n, void *stream, cj_result *results) {
    if (!problems || n < 1 || !results) return CJ_ERR_INVALID_ARG;
    int max_depth = 1, blocked_depth = 1;
    for (int k = 0; k < n; ++k) {
        cj_status st = check_problem(problems[k]);
        if (st != CJ_OK) return st;
        const int d = spec_of(problems[k]).depth;  // requested or autotuned
        max_depth = std::max(max_depth, d);
        if (problems[k].st == CJ_ST17 || d == 2 || d == 3) blocked_depth = std::max(blocked_depth, d);
    }
    auto t0 = Clock::now();
    Engine eng;
    cj_status st = eng.init(n, max_depth, 0, false, blocked_depth);
    if (st != CJ_OK) return st;
    cudaEvent_t ev;
    ENG_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "event");
    ENG_TRY(cudaEventRecord(ev, (cudaStream_t)stream), "event");
    ENG_TRY(cudaStreamWaitEvent(eng.stream(), ev, 0), "event wait");
    std::vector<int> slot(n, -1);
    long long max_steps = 0;
    for (int k = 0; k < n; ++k) {
        const cj_problem &pr = problems[k];
        const Spec sp = spec_of(pr);
        st = eng.admit(sp, pr.f, pr.ld_f, pr.u, pr.ld_u, pr.u, pr.ld_u, &slot[k]);
        if (st != CJ_OK) {
            cudaEventDestroy(ev);
            return st;
        }
        double kmin, kmax;
        long long M_in = 1;
        Engine::plan(sp, &kmin, &kmax, &M_in);
        const long long max_sweeps = sp.max_sweeps ? sp.max_sweeps : 64 * M_in;
        const long long outer = max_sweeps / M_in + 1;
        max_steps = std::max(max_steps, outer * (M_in / sp.depth + 2) + 4);
    }
    // every slot retires within max_steps engine steps (its outer-step budget)
    const long long max_replays = max_steps / eng.steps_per_graph() + 2;
    bool all = false;
    for (long long rep = 0; rep < max_replays && !all; ++rep) {
        st = eng.run(1);
        if (st != CJ_OK) {
            cudaEventDestroy(ev);
            return st;
        }
        all = true;
        for (int k = 0; k < n; ++k) {
            if (eng.status(slot[k]).phase != PHASE_RETIRED)
                all = false;
            else
                eng.drop_tiles(slot[k]);
        }
    }
    const double secs = std::chrono::duration<double>(Clock::now() - t0).count();
    for (int k = 0; k < n; ++k) {
        cj_result r{};
        fill_result(eng.status(slot[k]), &r);
        if (!all && eng.status(slot[k]).phase != PHASE_RETIRED) r.status = CJ_ERR_TIMEOUT;
        r.seconds = secs;
        r.launches = eng.launches();
        results[k] = r;
    }
    ENG_TRY(cudaEventRecord(ev, eng.stream()), "event");
    ENG_TRY(cudaStreamWaitEvent((cudaStream_t)stream, ev, 0), "event wait");
    ENG_TRY(cudaStreamSynchronize(eng.stream()), "batch sync");
    cudaEventDestroy(ev);
    return all ? CJ_OK : CJ_ERR_TIMEOUT;
}

cj_status cj_autotune_engine(int Nx, int Ny, cj_stencil st, int *tile_rows, int *depth, double *gupd) {
    if (Nx < 1 || Ny < 1 || Nx > (1 << 20) || Ny > (1 << 20)) return CJ_ERR_INVALID_ARG;
    if (st != CJ_ST5 && st != CJ_ST9 && st != CJ_ST17) return CJ_ERR_INVALID_ARG;
    // candidates, the default (32 rows, depth 1) first so that it wins ties
    const int tys[9] = {32, 16, 64, 32, 16, 64, 32, 16, 64};
    const int dps[9] = {1, 1, 1, 2, 2, 2, 4, 4, 4};
    const int kReplays = 8;  // 8 replays x 8 steps x 4 sweep launches
    double rate[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    // a synthetic problem of this class: f constant (every byte 0x3F, about 4.8e-4), u0 = 0,
    // a tolerance no slot reaches within the timed replays
    const size_t bytes = (size_t)Nx * Ny * sizeof(double);
    double *f = nullptr;
    ENG_TRY(cudaMalloc((void **)&f, bytes), "autotune grid");
    cudaError_t e = cudaMemset(f, 0x3F, bytes);
    if (e != cudaSuccess) {
        cudaFree(f);
        set_cuda_error(e, "autotune grid");
        return CJ_ERR_CUDA;
    }
    // as many copies of the problem as fill the device with tiles (a loaded engine, as in a
    // batch), within 256 slots and 2^24 nodes
    int sms = 152, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long tiles32 = (long long)((Nx + kEngTX - 1) / kEngTX) * ((Ny + 31) / 32);
    long long copies = (8LL * sms + tiles32 - 1) / tiles32;
    copies = std::min<long long>(copies, 256);
    copies = std::max<long long>(1, std::min<long long>(copies, (1LL << 24) / ((long long)Nx * Ny)));
    cj_status rc = CJ_OK;
    for (int c = 0; c < 9 && rc == CJ_OK; ++c) {
        // depth 4 of 5 and 9 points is the register wavefront, whose four-sweep launches of a
        // problem with a side under 512 are latency-bound in a batch (measured on the 512-problem
        // batch: 3.55 s at depth 1 everywhere, 3.45 s at depth 4 everywhere, 3.16 s at depth 4 from
        // a shorter side of 512): not a candidate there
        if (dps[c] == 4 && st != CJ_ST17 && std::min(Nx, Ny) < kEngWaveMinSide) continue;
        // the wavefront's copies: enough (strip, row block) items for two waves of its warps
        long long cp = copies;
        if (dps[c] == 4 && st != CJ_ST17) {
            std::vector<int4> items;
            const long long per = std::max(1, eng_wave_items(0, Nx, Ny, st, 4, items));
            cp = std::max(cp, (2LL * eng_wave_grid() * 4 + per - 1) / per);
            cp = std::min<long long>(cp, 256);
            cp = std::max<long long>(1, std::min<long long>(cp, (1LL << 24) / ((long long)Nx * Ny)));
        }
        Engine eng;
        rc = eng.init((int)cp, dps[c], 0, false, st == CJ_ST17 || dps[c] == 2 || dps[c] == 3 ? dps[c] : 1);
        if (rc != CJ_OK) break;
        Spec sp{};
        sp.Nx = Nx;
        sp.Ny = Ny;
        sp.st = st;
        sp.mode = CJ_FP32_INNER_DD;
        sp.inner_cycle = 0;
        sp.depth = dps[c];
        sp.ty = tys[c];
        sp.tol = 1e-15;
        sp.max_sweeps = 0;
        std::vector<int> q(cp, -1);
        for (long long k = 0; k < cp && rc == CJ_OK; ++k)
            rc = eng.admit(sp, f, Nx, nullptr, 0, nullptr, 0, &q[k], true);  // results into own slot
        if (rc == CJ_OK) rc = eng.run(2);  // capture and warm-up
        if (rc != CJ_OK) break;
        long long s0 = 0, s1 = 0;
        for (long long k = 0; k < cp; ++k) s0 += eng.status(q[k]).sweeps;
        const auto t0 = Clock::now();
        rc = eng.run(kReplays);
        const double secs = std::chrono::duration<double>(Clock::now() - t0).count();
        if (rc != CJ_OK) break;
        for (long long k = 0; k < cp; ++k) s1 += eng.status(q[k]).sweeps;
        rate[c] = (double)Nx * Ny * (double)(s1 - s0) / secs / 1e9;
    }
    cudaFree(f);
    if (rc != CJ_OK) return rc;
    int best = 0;
    for (int c = 1; c < 9; ++c)
        if (rate[c] > rate[best]) best = c;
    {
        std::lock_guard<std::mutex> lk(g_engine_tune_mu);
        g_engine_tune[stencil_slot(st)][size_class(Nx, Ny)] = EngineTune{tys[best], dps[best]};
    }
    if (tile_rows) *tile_rows = tys[best];
    if (depth) *depth = dps[best];
    if (gupd)  // tile rows 16, 32, 64 (major) x depth 1, 2, 4
        for (int c = 0; c < 9; ++c) gupd[(tys[c] == 16 ? 0 : tys[c] == 32 ? 1 : 2) * 3 + (dps[c] == 1 ? 0 : dps[c] == 2 ? 1 : 2)] = rate[c];
    return CJ_OK;
}

void cj_server_destroy(cj_server *sv);

cj_status cj_server_create(size_t hbm_budget_bytes, int max_slots, cj_server **out) {
    if (!out || hbm_budget_bytes == 0 || max_slots < 1) return CJ_ERR_INVALID_ARG;
    *out = nullptr;
    cj_server *sv = new (std::nothrow) cj_server();
    if (!sv) return CJ_ERR_NOMEM;
    sv->budget = hbm_budget_bytes;
    sv->max_slots = max_slots;
    cudaGetDevice(&sv->device);
    for (int k = 0; k < kLanes; ++k) {
        // the two larger lanes sweep 5- and 9-point requests with a side of at least 512 on the
        // register wavefront (depth 4); the smallest sweeps one at a time
        cj_status st = sv->lanes[k].eng.init(max_slots, k == kLanes - 1 ? 4 : 1, kLanes - 1 - k, true, 1, kServerWaveShare);
        if (st == CJ_OK && cudaMallocHost((void **)&sv->lanes[k].stage, cj_server::kStageBytes) != cudaSuccess)
            st = CJ_ERR_NOMEM;
        if (st != CJ_OK) {
            cj_server_destroy(sv);
            return st;
        }
    }
    try {
        for (int k = 0; k < kLanes; ++k) sv->lanes[k].worker = std::thread([sv, k] { sv->loop(k); });
    } catch (...) {
        cj_server_destroy(sv);
        return CJ_ERR_NOMEM;
    }
    *out = sv;
    return CJ_OK;
}

cj_status cj_submit(cj_server *sv, int Nx, int Ny, cj_stencil st, double tol, const double *f_host,
                    uint64_t *ticket) {
    if (!sv || !f_host || !ticket) return CJ_ERR_INVALID_ARG;
    cj_problem pr{};
    pr.Nx = Nx;
    pr.Ny = Ny;
    pr.st = st;
    pr.tol = tol;
    pr.f = f_host;
    pr.u = (double *)f_host;
    pr.ld_f = pr.ld_u = Nx;
    cj_status c = check_problem(pr);
    if (c != CJ_OK) return c;
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->fatal != CJ_OK) return sv->fatal;
    const uint64_t t = sv->next_ticket++;
    cj_server::Request &r = sv->reqs[t];
    r.ticket = t;
    r.sp = spec_of(pr);
    r.lane = lane_of(r.sp);
    r.f.assign(f_host, f_host + (size_t)Nx * Ny);
    r.t_submit = Clock::now();
    sv->lanes[r.lane].queue.push_back(t);
    *ticket = t;
    sv->cv.notify_all();
    return CJ_OK;
}

cj_status cj_poll(cj_server *sv, uint64_t ticket, double *u_host, cj_result *res) {
    if (!sv) return CJ_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(ticket);
    if (it == sv->reqs.end()) return CJ_ERR_INVALID_ARG;
    cj_server::Request &r = it->second;
    if (r.state != 2) return CJ_PENDING;
    if (u_host && !r.u.empty()) std::memcpy(u_host, r.u.data(), r.u.size() * sizeof(double));
    if (res) *res = r.res;
    const cj_status rc = r.rc;
    sv->reqs.erase(it);
    return rc;
}

cj_status cj_server_stats(cj_server *sv, cj_server_stats_t *out) {
    if (!sv || !out) return CJ_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(sv->mu);
    out->queued = sv->queued_all();
    out->active = sv->active_all();
    out->admitted = sv->admitted;
    out->completed = sv->completed;
    out->steps = sv->steps;
    out->peak_active = sv->peak_active;
    out->bytes_in_use = sv->in_use;
    out->peak_bytes = sv->peak_bytes;
    out->budget_bytes = sv->budget;
    return CJ_OK;
}

void cj_server_destroy(cj_server *sv) {
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
        sv->cv.notify_all();
    }
    for (int k = 0; k < kLanes; ++k)
        if (sv->lanes[k].worker.joinable()) sv->lanes[k].worker.join();
    delete sv;
}

}  // extern "C"
