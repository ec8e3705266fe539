// Device-resident state of the batched / served CJM engine (shared by engine.cu and
// batch.cpp).  Each admitted problem occupies one slot; every kernel of an engine step
// reads the slots' phases from device memory, so one captured CUDA graph of steps serves
// whatever set of problems is admitted when it is replayed.
#pragma once

#include <vector>

#include "cj_internal.h"

// Engine tile: the unit of work of every engine kernel, kEngTX columns x (per slot) ty rows of
// nodes; ty is 16, 32 (the default) or 64, chosen per stencil and size class by
// cj_autotune_engine.
constexpr int kEngTX = 128, kEngTYDefault = 32, kEngTYMax = 64;

enum SlotPhase : int {
    PHASE_FREE = 0,     // unused
    PHASE_OUTER = 1,    // next step: correction (after the first cycle) + defect + stop test
    PHASE_SWEEP = 2,    // inner FP32 cycle in progress
    PHASE_DONE = 3,     // stopped; the next step copies u to the caller's buffer
    PHASE_RETIRED = 4   // result delivered; the host may release the slot
};

struct SlotDev {
    // set at admission
    int Nx, Ny, st, mode;          // mode: CJ_FP32_INNER or CJ_FP32_INNER_DD
    int depth, ntx, ntiles, ty;    // ty: tile rows
    long long M_in, max_outer;
    double tol, S, h2;
    Grid g64, g32;
    double *u, *ulo, *b;           // padded FP64 (ulo: CJ_FP32_INNER_DD only)
    float *e0, *e1, *rt;           // padded FP32
    const float *w32;              // inner-cycle weights, M_in of them
    double *part;                  // 3 doubles per tile
    double *out;                   // caller's device grid for the result
    long long ld_out;
    // evolving
    int phase, status, cur, stall;
    long long counter, outer, sweeps;
    double prev, rho, rinf, fl, bsq, bmax;
};

// Compact per-slot record the host polls after each replay.
struct SlotStatus {
    int phase, status;
    long long sweeps, outer;
    double rho, rinf, fl;
};

struct EngineDev {
    SlotDev *slots;        // max_slots entries
    int max_slots;
    int2 *tiles;           // (slot, tile index within the slot)
    int *ntiles;           // device counter of valid entries in tiles
    int4 *waves;           // (slot, strip, row block, 0): register-wavefront items of depth-4 slots
    int *nwaves;           // device counter of valid entries in waves
    SlotStatus *status;    // max_slots entries, refreshed by the advance kernel
};

// launchers (engine.cu)
// one engine step: correct, defect, decide, `sweeps` sweep launches (with wave_grid > 0, each
// also launches the register-wavefront kernel over the wave list with that many blocks), export,
// advance (the step's sweeps applied to the counters at once)
cudaError_t eng_launch_step(const EngineDev &e, int grid_tiles, int grid_slots, size_t sweep_smem,
                            int sweeps, int wave_grid, cudaStream_t s);
// Appends the register-wavefront items of a slot (Nx x Ny, stencil st) to items, if the slot's
// sweeps at depth `depth` run on the wavefront (5- and 9-point slots at depth 4); returns how many.
int eng_wave_items(int slot, int Nx, int Ny, int st, int depth, std::vector<int4> &items);
// Blocks of the wavefront kernel resident on the device at once (one wave).
int eng_wave_grid();
cudaError_t eng_launch_import(const EngineDev &e, int slot, int ntiles, const double *f,
                              long long ldf, const double *u0, long long ldu, cudaStream_t s);
size_t eng_sweep_smem(int max_depth);
// blocks of the one-sweep tile kernel (the engine's heaviest in registers) resident per SM
int eng_sweep_blocks_per_sm();
// true for the kernels that loop over the tile list (their grid may be any size)
bool eng_is_tile_kernel(const void *fn);
cudaError_t eng_prepare(size_t sweep_smem);
