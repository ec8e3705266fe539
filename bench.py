"""Benchmark of the GB300 Chebyshev-Jacobi solver: one JSON line on stdout.

Workload (one step): the CJM solve of Delta_h u = f with the 9-point alpha = 2/3 stencil (Eq. 1)
on a 4096 x 4096 interior grid, homogeneous Dirichlet boundary, to relative residual 1e-10 in
FP64 arithmetic: FP64 CJM cycles inside double-FP64 defect correction (plain FP64 cycles stall
above 1e-10 on this grid, so the residual target needs the double-FP64 outer step; every sweep is
the plain FP64 sweep).  The right-hand side alternates between steps over the two of this
workload: the manufactured f = -2 pi^2 sin(pi x) sin(pi y), and a seeded smooth random f (sine
modes |k| <= 64, Gaussian amplitudes decaying as |k|^-2).  Inputs (134 MB FP64 grids) are larger
than the 129 MB L2, so no flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

value  = interior points x sweeps of all ranks / max-over-ranks device time of the K steps
         (Gupdates/s, grid-point updates per second), inputs resident in HBM;
e2e    = the same metric through cj_solve_host (host arrays, one H2D copy of f and of the
         initial guess, one D2H copy of u inside every step), over min(K, 3) steps;
roofline: the FP64 sweep kernel against the FP64 FMA issue rate measured on the GPU by
         cj_issue_peaks (it is bound by FP64 arithmetic on GB300, not by HBM; its HBM fraction
         is given beside);
vs_plain_fp64: configuration 2's comparisons -- plain FP64 cycles (which stall), FP32 inner
         cycles in FP64 / double-FP64 defect correction (time to 1e-10) -- and
         fp32_sweep_roofline: the FP32 register wavefront kernel (4 sweeps per launch) timed alone
         against the measured FP32 FMA issue rate, and ff_sweep_roofline: the float-float
         FP64-accuracy sweep on the FP32 pipe beside the bit-exact FP64 sweep;
highorder, batch, serve: configurations 3, 4 and 5 (17-point 8192^2 mixed precision to 1e-10;
         the 512-problem batch; an arrival-faithful prefix of the served stream), each with an
         FP64 comparison and its own clock record;
cpu_baseline / --impl reference: the FP64 C oracle (test infrastructure) timed on the
         host on a bounded sample of the same workload.
N > 1 runs independent replicas, one per GPU (the solve does not shard across GPUs).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

N_GRID = 4096
STENCIL = 9
TOL = 1e-10
METRIC = "CJM time-to-1e-10 residual & Gupdates/s vs plain FP64; HBM GB/s; p50/p99 latency"
UNIT = "Gupdates/s"
# FP64 instructions per grid-point update of the sweep (9-point tree: 4 pair/group sums,
# 3 coefficient fmas, 1 update fma) and algorithmic bytes (read u and b, write u')
FP64_OPS_PER_UPDATE = {5: 6, 9: 8, 17: 14}
BYTES_PER_UPDATE_FP64 = 24
# FP64 issue peak: 1.25 TFLOP/s nominal = 2 FP64 FMA per SM per clock x 152 SMs x 2.07 GHz
FP64_PEAK_TOPS = 2 * 152 * 2.07e9 / 1e12


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="cj", choices=["cj", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--workload", default="solve", choices=["solve", "highorder", "paper", "masks", "batch", "serve"],
                    help="solve: the plain FP64 9-point 4096^2 solve (default); highorder: the 17-point "
                         "8192^2 mixed-precision solve; paper: the paper's test problem (Table 1 point and Fig. 4 "
                         "right); masks: coefficient-mask sweeps and a polar solve; batch: the 512-problem batched workload; serve: a "
                         "bounded sample of the request stream")
    ap.add_argument("--serve-requests", type=int, default=64)
    ap.add_argument("--no-extra", action="store_true",
                    help="default workload: skip the highorder, batch and serve keys")
    ap.add_argument("--no-autotune", action="store_true",
                    help="batch workload: keep the engine's default tiles (32 rows) and depth 1")
    ap.add_argument("--no-jacobi", action="store_true",
                    help="paper workload: skip the classical Jacobi solves of Table 1 (minutes)")
    return ap.parse_args(argv)


# ----------------------------------------------------------------- distributed plumbing

def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def dist_init(world, backend):
    import torch.distributed as dist
    if world > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend)
    return dist


def reduce_max_sum(dist, world, tmax: float, tsum: float, device=None):
    """(max over ranks of tmax, sum over ranks of tsum)."""
    if world == 1:
        return tmax, tsum
    import torch
    a = torch.tensor([tmax], dtype=torch.float64, device=device)
    b = torch.tensor([tsum], dtype=torch.float64, device=device)
    dist.all_reduce(a, op=dist.ReduceOp.MAX)
    dist.all_reduce(b, op=dist.ReduceOp.SUM)
    return float(a.item()), float(b.item())


def barrier(dist, world):
    if world > 1:
        dist.barrier()


# ----------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi sampled every 200 ms during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,"
              "clocks.mem,clocks.max.mem")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", "cj_clocks_%d_%d.csv" % (os.getpid(), index))

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons, power, mem, mmax = [], [], set(), [], [], []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
            try:
                mem.append(float(parts[9]))
                mmax.append(float(parts[10]))
            except (ValueError, IndexError):
                pass
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        out = {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
               "power_w_max": max(power), "samples": len(sm)}
        if mem:
            out["mem_mhz"] = statistics.median(mem)
            out["mem_max_mhz"] = max(mmax)
        return out


# ----------------------------------------------------------------- traffic record

KERNEL_SOURCES = ("kernels.cu", "stencil_dev.cuh", "grid_dev.cuh")
# sources of the FP32 register wavefront kernel (temporal blocking)
WAVE_REG_SOURCES = ("wave_reg.cu", "wave_reg_dev.cuh", "fold_dev.cuh", "grid_dev.cuh", "stencil_dev.cuh", "cj_internal.h")
# FP32 instructions per 9-point update of the register wavefront kernel (second-difference form):
# 1.25 first differences along the row (shared between neighbours) and 1 second difference, both
# for the row entering the stencil; 1 vertical difference and 1 second difference; 1 sum of the
# outer rows' second differences, 1 subtraction of r, 2 coefficient fmas, 1 update fma
FP32_OPS_PER_UPDATE_WAVE_REG_9 = 9.25
# FP32 issue peak: 4 schedulers x 32 lanes per SM x 152 SMs x 2.07 GHz (FFMA/FADD issue at one
# warp instruction per scheduler per clock)
FP32_ISSUE_PEAK_TOPS = 4 * 32 * 152 * 2.07e9 / 1e12


# sources of the float-float sweep kernel
FF_SOURCES = ("ff.cu", "grid_dev.cuh", "stencil_dev.cuh", "cj_internal.h")
# FP32 instructions per 9-point update of the float-float sweep in its scaled form
# u' = c1 u + (w/6) (4 a + d - 6 b): 7 float-float adds (11 each: TwoSum 6, low parts 2,
# FastTwoSum 3; the row pair, the vertical pair, a, d, 4 a + d, - 6 b and the final sum), the
# exact scaling by 4 (2) and 2 TwoProduct multiplies (7 each)
FF_OPS_PER_UPDATE_9 = 7 * 11 + 2 + 2 * 7


def kernel_digest(sources=KERNEL_SOURCES) -> str:
    """Digest of the sources a kernel is compiled from."""
    h = hashlib.sha256()
    for name in sources:
        h.update(open(os.path.join(ROOT, "paper_1705_00103_gb300", "csrc", name), "rb").read())
    return h.hexdigest()[:16]


def traffic_per_launch(kernel_key: str, sources=KERNEL_SOURCES):
    """DRAM bytes per launch of a kernel from the committed ncu summary, or None when the
    kernel's sources changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "traffic_per_launch.txt")
    if not os.path.exists(path):
        return None
    digest = kernel_digest(sources)
    for line in open(path):
        parts = line.split()
        if len(parts) >= 3 and not line.startswith("#") and parts[0] == kernel_key:
            return float(parts[1]) if parts[2] == digest else None
    return None


# ----------------------------------------------------------------- workload

def make_rhs(which: int):
    import workloads
    if which == 0:
        return workloads.manufactured_rhs(N_GRID, N_GRID)
    return workloads.smooth_random_rhs(N_GRID, N_GRID, seed=1)


def cpu_oracle_sample(seconds_target: float = 15.0) -> dict:
    """The FP64 C oracle as it stands, single-threaded, timed on FP64 9-point sweeps of the
    4096^2 grid (a bounded sample of the workload: whole sweeps until ~seconds_target)."""
    from oracle import oracle as orc
    f = make_rhs(1)
    b = orc.scale_rhs(f)
    kmin, kmax = orc.kappa_bounds(STENCIL, N_GRID, N_GRID)
    M = orc.cycle_length(kmin, kmax, TOL)
    w = orc.sweep_coeffs(STENCIL, kmin, kmax, M)
    u = np.zeros_like(b)
    t0 = time.perf_counter()
    n = 0
    while True:
        u = orc.sweep(STENCIL, u, b, w[n % M])
        n += 1
        if time.perf_counter() - t0 >= seconds_target:
            break
    dt = time.perf_counter() - t0
    return {"value": N_GRID * N_GRID * n / dt / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "%d FP64 9-point CJM sweeps of the 4096x4096 grid (smooth random RHS), "
                      "single-threaded C oracle, %.1f s" % (n, dt)}


def measured_hbm_gbs():
    """The measured copy bandwidth (MEASURED_PEAKS.json), else the recipe's fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured (MEASURED_PEAKS.json: torch copy)"
    except Exception:
        return 6800.0, "fallback (no MEASURED_PEAKS.json)"


def issue_peaks(cj, stream) -> dict:
    """FP64 and FP32 FMA issue rates measured on this device by cj_issue_peaks (best of 3), with
    the nominal figures from unit counts and the maximum clock beside them."""
    runs = [cj.cj_issue_peaks(stream) for _ in range(3)]
    return {"fp64_tfma_s": max(r["fp64_tfma_s"] for r in runs),
            "fp32_tfma_s": max(r["fp32_tfma_s"] for r in runs),
            "fp64_nominal": FP64_PEAK_TOPS, "fp32_nominal": FP32_ISSUE_PEAK_TOPS,
            "how": "cj_issue_peaks: 8 independent FMA chains per thread, 4 x 256 threads per SM, CUDA events, "
                   "best of 3; nominal = (2 FP64 | 128 FP32) FMA/clk/SM x 152 SMs x 2.07 GHz"}


def run_cj(args):
    import torch

    import paper_1705_00103_gb300 as cj
    rank, world, local = dist_env()
    if world != args.gpus:
        world = max(world, 1)
    torch.cuda.set_device(local)
    dist = dist_init(world, "nccl")
    cj.build.build()
    stream = torch.cuda.current_stream()
    peaks = issue_peaks(cj, stream)
    hbm_peak, hbm_note = measured_hbm_gbs()

    # the headline step: CJM in FP64 arithmetic to 1e-10 (FP64 inner cycles in double-FP64 defect
    # correction; plain FP64 cycles stall above 1e-10 on this grid, see vs_plain_fp64)
    plan = cj.Plan(N_GRID, N_GRID, STENCIL, TOL, precision=cj.CJ_FP64_INNER_DD)
    info = plan.info()
    rhs_host = [np.ascontiguousarray(make_rhs(0)), np.ascontiguousarray(make_rhs(1))]
    rhs_dev = [torch.from_numpy(r).cuda() for r in rhs_host]
    u = torch.zeros((N_GRID, N_GRID), dtype=torch.float64, device="cuda")

    def step(k):
        u.zero_()
        return cj.cj_solve(plan.handle, rhs_dev[k % 2], u, stream)

    for k in range(args.warmup):
        step(k)
    torch.cuda.synchronize()
    barrier(dist, world)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    results = [step(k) for k in range(args.steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(dist, world)
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    updates = sum(r["sweeps"] for r in results) * N_GRID * N_GRID
    ms_max, updates_all = reduce_max_sum(dist, world, ms, float(updates), device="cuda")
    value = updates_all / (ms_max * 1e-3) / 1e9

    # the comparisons below use the smooth-RHS solve: the second timed step, or (one timed step)
    # a solve of it after the timed region
    smooth = results[1] if len(results) > 1 else (step(1) if not args.no_mixed and rank == 0 else None)

    sweeps = sum(r["sweeps"] for r in results)
    sweep_s = sum(r["sweep_seconds"] for r in results)
    avg_sweep_s = sweep_s / sweeps
    ops = FP64_OPS_PER_UPDATE[STENCIL] * N_GRID * N_GRID
    achieved = ops / avg_sweep_s / 1e12
    traffic = traffic_per_launch("sweep_kernel_9_f64_4096")
    hbm_gbs = BYTES_PER_UPDATE_FP64 * N_GRID * N_GRID / avg_sweep_s / 1e9
    roofline = {"bound": "alu", "achieved": achieved, "peak": peaks["fp64_tfma_s"], "unit": "TFP64op/s",
                "frac": achieved / peaks["fp64_tfma_s"], "traffic": traffic,
                "kernel": "sweep_kernel<9,double>", "avg_launch_us": avg_sweep_s * 1e6,
                "peak_note": "FP64 FMA issue rate measured on this GPU by cj_issue_peaks (the sweep issues "
                             "every FP64 operation as an FMA: 8 per 9-point update); of measured",
                "peak_nominal": FP64_PEAK_TOPS, "frac_of_nominal": achieved / FP64_PEAK_TOPS,
                "hbm": {"achieved_gbs": hbm_gbs, "peak_gbs": hbm_peak, "frac": hbm_gbs / hbm_peak,
                        "bytes_per_update": BYTES_PER_UPDATE_FP64, "peak_note": hbm_note},
                "issue_peaks": peaks}

    e2e = None
    if not args.no_e2e:
        n_e2e = min(args.steps, 3)
        pinned_f = [torch.from_numpy(r).pin_memory().numpy() for r in rhs_host]
        pinned_u = torch.zeros((N_GRID, N_GRID), dtype=torch.float64).pin_memory().numpy()
        torch.cuda.synchronize()
        barrier(dist, world)
        t0 = time.perf_counter()
        eres = []
        for k in range(n_e2e):
            pinned_u[...] = 0.0
            eres.append(cj.cj_solve_host(plan.handle, pinned_f[k % 2], pinned_u, stream))
        t_e2e = time.perf_counter() - t0
        t_max, up_all = reduce_max_sum(dist, world, t_e2e,
                                       float(sum(r["sweeps"] for r in eres) * N_GRID * N_GRID), device="cuda")
        e2e = {"value": up_all / t_max / 1e9, "unit": UNIT, "steps": n_e2e,
               "h2d_bytes_per_step": 2 * N_GRID * N_GRID * 8, "d2h_bytes_per_step": N_GRID * N_GRID * 8,
               "api": "cj_solve_host"}
    plan.close()

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "CJM in FP64 arithmetic to relative residual 1e-10: FP64 CJM cycles (inner "
                               "cycle %d) in double-FP64 defect correction, 9-point alpha=2/3 stencil, "
                               "4096x4096 interior, homogeneous Dirichlet; RHS alternating sin*sin / seeded "
                               "smooth random (|k|<=64, |k|^-2). Plain FP64 cycles stall above 1e-10 here "
                               "(vs_plain_fp64.plain_fp64_cycles)" % info["M_inner"],
                   "Nx": N_GRID, "Ny": N_GRID, "stencil": STENCIL, "tol": TOL, "M": info["M"],
                   "inner_cycle": info["M_inner"], "precision": "FP64 inner cycles, double-FP64 outer",
                   "l2_flush": "none needed: 6 resident FP64 grids of 134 MB each exceed the 129 MB L2",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "solves": [{"status": cj.cj_status_string(r["rc"]), "sweeps": r["sweeps"], "outer_steps": r["cycles"],
                    "rel_res_l2": r["rel_res_l2"], "time_s": r["seconds"]} for r in results[:2]],
        "roofline": roofline, "clocks": clk, "gpu_launches": sum(r["launches"] for r in results),
        "e2e": e2e,
    }
    if not args.no_mixed and rank == 0:
        out["vs_plain_fp64"] = keyed(lambda: mixed_paths(cj, rhs_dev[1], stream, smooth, peaks), local)
        out["small_5pt_64"] = small_solve(cj, stream)
    if not args.no_extra and rank == 0:
        out["highorder"] = keyed(lambda: highorder_key(cj, stream), local)
        out["batch"] = keyed(lambda: batch_key(cj, stream, autotune=not args.no_autotune), local)
        out["serve"] = keyed(lambda: serve_key(cj, args.serve_requests), local)
    if rank == 0 and not args.no_cpu:
        out["cpu_baseline"] = cpu_oracle_sample()
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


def keyed(fn, local):
    """Runs one extra measurement with its own clock record."""
    clk = ClockSampler(local)
    clk.start()
    t0 = time.perf_counter()
    d = fn()
    d["clocks"] = clk.stop()
    d["bench_wall_s"] = time.perf_counter() - t0
    return d


def mixed_paths(cj, f, stream, fp64dd, peaks):
    """Configuration 2's comparisons, on its smooth-RHS problem, each solved once: the plain FP64
    cycles (which stall above 1e-10 here), and the FP32-inner paths (FP64 and double-FP64 outer
    steps) -- time to stop, residual reached, and the speed-up over the FP64-arithmetic path that
    does reach 1e-10 (the headline's solve) and over the plain FP64 solve's stall."""
    import torch
    out = {"fp64_inner_dd": {"time_s": fp64dd["seconds"], "rel_res_l2": fp64dd["rel_res_l2"],
                             "status": cj.cj_status_string(fp64dd["rc"]), "fp64_sweeps": fp64dd["sweeps"],
                             "outer_steps": fp64dd["cycles"],
                             "note": "the headline's solve of this RHS: the all-FP64 path to 1e-10"}}
    with cj.Plan(N_GRID, N_GRID, STENCIL, TOL) as p:
        u = torch.zeros((N_GRID, N_GRID), dtype=torch.float64, device="cuda")
        plain = cj.cj_solve(p.handle, f, u, stream)
    out["plain_fp64_cycles"] = {"time_s": plain["seconds"], "rel_res_l2": plain["rel_res_l2"],
                                "floor_est": plain["floor_est"], "status": cj.cj_status_string(plain["rc"]),
                                "sweeps": plain["sweeps"],
                                "note": "plain CJM cycles of M sweeps in FP64: the second cycle fails to halve "
                                        "the residual, which stalls far above 1e-10 and above the FP64 floor"}
    runs = (("fp32_inner_fp64_outer", cj.CJ_FP32_INNER, 0), ("fp32_inner_dd_outer", cj.CJ_FP32_INNER_DD, 0),
            ("fp32_inner_dd_outer_one_sweep_per_launch", cj.CJ_FP32_INNER_DD, 1))
    for name, prec, depth in runs:
        with cj.Plan(N_GRID, N_GRID, STENCIL, TOL, precision=prec, temporal_depth=depth) as p:
            u = torch.zeros((N_GRID, N_GRID), dtype=torch.float64, device="cuda")
            r = cj.cj_solve(p.handle, f, u, stream)
            M_in = p.info()["M_inner"]
        upd_s = N_GRID * N_GRID * r["sweeps"] / r["sweep_seconds"]
        k = depth if depth else 4
        out[name] = {"time_s": r["seconds"], "rel_res_l2": r["rel_res_l2"], "status": cj.cj_status_string(r["rc"]),
                     "fp32_sweeps": r["sweeps"], "outer_steps": r["cycles"], "inner_cycle": M_in,
                     "temporal_depth": depth if depth else "auto (4 for this stencil and size unless "
                                                           "cj_autotune_depth recorded another)",
                     "fp32_gupdates_s": upd_s / 1e9,
                     # algorithmic bytes: one HBM round trip (read e, r; write e') per launch of k sweeps
                     "fp32_hbm_gbs_algorithmic": 12.0 / k * upd_s / 1e9,
                     "speedup_vs_fp64_inner_dd": fp64dd["seconds"] / r["seconds"],
                     "speedup_vs_plain_fp64_stall": plain["seconds"] / r["seconds"]}
    out["fp32_sweep_roofline"] = fp32_sweep_roofline(cj, stream, peaks)
    out["ff_sweep_roofline"] = ff_sweep_roofline(cj, f, stream, peaks)
    return out


def small_solve(cj, stream, runs: int = 5) -> dict:
    """The small case (5-point, 64 x 64, FP64, tol 1e-10, the sin*sin right-hand side): time to
    tolerance of whole cj_solve calls (graph-launched cycles), median of `runs` after 3 warm-up
    solves; the call blocks until the solve ends, so host time is the time to tolerance."""
    import torch
    import workloads
    N = 64
    f = torch.from_numpy(workloads.manufactured_rhs(N, N)).cuda()
    times, res = [], None
    with cj.Plan(N, N, 5, TOL) as p:
        u = torch.zeros_like(f)
        for k in range(3 + runs):
            u.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            res = cj.cj_solve(p.handle, f, u, stream)
            torch.cuda.synchronize()
            if k >= 3:
                times.append(time.perf_counter() - t0)
    return {"us_to_tol_median": statistics.median(times) * 1e6, "sweeps": res["sweeps"],
            "rel_res_l2": res["rel_res_l2"], "status": cj.cj_status_string(res["rc"]), "runs": runs}


def fp32_sweep_roofline(cj, stream, peaks, launches: int = 64) -> dict:
    """The dominant kernel of the FP32-inner paths, the register wavefront at its default depth
    (4 sweeps per launch), timed alone with CUDA events on the launching stream over `launches`
    launches on the 4096^2 grid (three 64 MB FP32 grids, more than the L2), against the FP32
    FMA issue rate measured on this GPU: it is bound by instruction issue, not by HBM."""
    import torch
    with cj.Plan(N_GRID, N_GRID, STENCIL, TOL, precision=cj.CJ_FP32_INNER) as p:
        r = torch.zeros((N_GRID, N_GRID), dtype=torch.float32, device="cuda")
        e = torch.zeros_like(r)
        depth = 4
        cj.cj_sweeps_f32(p.handle, r, e, 0, 4 * depth, stream)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        cj.cj_sweeps_f32(p.handle, r, e, 0, launches * depth, stream)
        e1.record(stream)
        torch.cuda.synchronize()
    per_launch = e0.elapsed_time(e1) * 1e-3 / launches
    upd = depth * N_GRID * N_GRID
    achieved = FP32_OPS_PER_UPDATE_WAVE_REG_9 * upd / per_launch / 1e12
    traffic = traffic_per_launch("sweep_wave_reg_9_d4_4096", WAVE_REG_SOURCES)
    peak = peaks["fp32_tfma_s"]
    return {"kernel": "sweep_wave_reg_kernel<9,4>", "bound": "alu", "achieved": achieved,
            "peak": peak, "unit": "TFP32op/s", "frac": achieved / peak,
            "peak_nominal": FP32_ISSUE_PEAK_TOPS, "frac_of_nominal": achieved / FP32_ISSUE_PEAK_TOPS,
            "traffic": traffic,
            "avg_launch_us": per_launch * 1e6, "sweeps_per_launch": depth,
            "gupdates_s": upd / per_launch / 1e9,
            # DRAM bytes actually moved (ncu traffic per launch) per second and per update
            "dram_gbs_with_temporal_blocking": None if traffic is None else traffic / per_launch / 1e9,
            "dram_bytes_per_update": None if traffic is None else traffic / upd,
            # algorithmic bytes: one round trip of e, r, e' (12 B per node) per launch of 4 sweeps
            "hbm_gbs_algorithmic": 12.0 * N_GRID * N_GRID / per_launch / 1e9,
            "peak_note": "FP32 FMA issue rate measured by cj_issue_peaks, of measured; 9.25 FP32 instructions "
                         "per 9-point update in the kernel's shared second-difference form"}


def ff_sweep_roofline(cj, f, stream, peaks, sweeps: int = 64) -> dict:
    """The float-float sweep (cj_sweeps_ff: the FP64 sweep's expression in pairs of floats on the
    FP32 pipe) beside the bit-exact FP64 sweep, on the 4096^2 9-point grid: `sweeps` sweeps of
    the plan's cycle in one call each (the float-float call includes its 6 in-place conversions
    of the three FP64 grids), timed with CUDA events on the launching stream; and its largest
    deviation from the FP64 kernel over the first sweep from a random iterate, relative to the
    per-sweep scale max|u| + |w| (9 max|u| + max|b|)."""
    import torch
    hbm_peak, hbm_note = measured_hbm_gbs()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with cj.Plan(N_GRID, N_GRID, STENCIL, TOL) as p:
        w = p.info()["w"]
        t = {}
        for name, fn in (("ff", cj.cj_sweeps_ff), ("fp64", cj.cj_sweeps)):
            u = torch.zeros((N_GRID, N_GRID), dtype=torch.float64, device="cuda")
            fn(p.handle, f, u, 0, 8, stream)
            torch.cuda.synchronize()
            e0.record(stream)
            fn(p.handle, f, u, 0, sweeps, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            t[name] = e0.elapsed_time(e1) * 1e-3 / sweeps
        g = torch.Generator(device="cuda").manual_seed(5)
        u0 = torch.randn((N_GRID, N_GRID), dtype=torch.float64, device="cuda", generator=g)
        k = int(np.argmax(w))
        dev = {}
        for name, fn in (("ff", cj.cj_sweeps_ff), ("fp64", cj.cj_sweeps)):
            u = u0.clone()
            fn(p.handle, f, u, k, 1, stream)
            dev[name] = u
        torch.cuda.synchronize()
        dmax = float((dev["ff"] - dev["fp64"]).abs().max())
        umax = float(u0.abs().max())
        bmax = float(f.abs().max()) / ((N_GRID + 1) ** 2)
        scale = umax + abs(float(w[k])) * (9.0 * umax + bmax)
    upd = N_GRID * N_GRID
    gupd = upd / t["ff"] / 1e9
    hbm = BYTES_PER_UPDATE_FP64 * upd / t["ff"] / 1e9
    ops = FF_OPS_PER_UPDATE_9 * upd / t["ff"] / 1e12
    return {"kernel": "sweep_ff_kernel<9>", "bound": "hbm", "achieved": hbm, "peak": hbm_peak, "unit": "GB/s",
            "frac": hbm / hbm_peak, "traffic": traffic_per_launch("sweep_ff_9_4096", FF_SOURCES),
            "bytes_per_update": BYTES_PER_UPDATE_FP64,
            "peak_note": hbm_note + "; of measured",
            "fp32_issue": {"achieved": ops, "peak": peaks["fp32_tfma_s"], "unit": "TFP32op/s",
                           "frac": ops / peaks["fp32_tfma_s"], "ops_per_update": FF_OPS_PER_UPDATE_9,
                           "note": "FP32 FMA issue rate measured by cj_issue_peaks, of measured"},
            "avg_sweep_us": t["ff"] * 1e6, "gupdates_s": gupd,
            "fp64_sweep_avg_us": t["fp64"] * 1e6, "fp64_sweep_gupdates_s": upd / t["fp64"] / 1e9,
            "speedup_vs_fp64_sweep": t["fp64"] / t["ff"],
            "max_dev_vs_fp64_sweep": dmax, "max_dev_rel_to_sweep_scale": dmax / scale,
            "dev_weight_index": k,
            "note": "FP64-accuracy (48-bit float-float) sweep, not bit-equal to the FP64 sweep; per-sweep "
                    "deviation held to 1e-12 of the sweep scale by the parity tests; timings include the "
                    "in-place conversions of the three grids, amortised over the call's sweeps"}


def highorder_key(cj, stream, steps: int = 1) -> dict:
    """Configuration 3: the 17-point 8192^2 problem (seeded smooth RHS, seed 2) to relative residual
    1e-10 by FP32 inner cycles inside double-FP64 defect correction, `steps` solves timed with CUDA
    events after one untimed plan.  The FP64 comparisons are extrapolated from 64 timed FP64 sweeps
    of this grid (a full run would take minutes) and labelled as such: one plain FP64 cycle of M
    sweeps (plain cycles stall above 1e-10 here, so this is a lower bound on their time), and the
    all-FP64 path at the sweep count of two inner cycles of its planner's length (a lower bound too:
    one cycle cannot reach 1e-10)."""
    import torch
    import workloads
    N, st = 8192, 17
    f = torch.from_numpy(workloads.smooth_random_rhs(N, N, 2)).cuda()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with cj.Plan(N, N, st, TOL, precision=cj.CJ_FP32_INNER_DD) as plan:
        info = plan.info()
        u = torch.zeros_like(f)
        res = []
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            u.zero_()
            res.append(cj.cj_solve(plan.handle, f, u, stream))
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
    sweeps = sum(r["sweeps"] for r in res)
    with cj.Plan(N, N, st, TOL) as p64:
        M = p64.info()["M"]
        g = torch.zeros_like(f)
        cj.cj_sweeps(p64.handle, f, g, 0, 4)
        torch.cuda.synchronize()
        e0.record(stream)
        cj.cj_sweeps(p64.handle, f, g, 0, 64)
        e1.record(stream)
        torch.cuda.synchronize()
        per64 = e0.elapsed_time(e1) / 64 * 1e-3
    with cj.Plan(N, N, st, TOL, precision=cj.CJ_FP64_INNER_DD) as pdd:
        M_dd = pdd.info()["M_inner"]
    r = res[-1]
    t = ms / steps * 1e-3
    return {"workload": "17-point alpha=2/3, 8192x8192, smooth random RHS (seed 2), tol 1e-10, FP32 inner "
                        "cycles in double-FP64 defect correction", "steps": steps,
            "time_to_tol_s": t, "gupdates_s": N * N * sweeps / (ms * 1e-3) / 1e9,
            "status": cj.cj_status_string(r["rc"]), "rel_res_l2": r["rel_res_l2"], "fp32_sweeps": r["sweeps"],
            "outer_steps": r["cycles"], "inner_cycle": info["M_inner"],
            "fp64_sweep_s": per64,
            "plain_fp64_one_cycle_s_extrapolated": per64 * M,
            "fp64_inner_dd_lower_bound_s_extrapolated": per64 * 2 * M_dd,
            "speedup_vs_plain_fp64_one_cycle": per64 * M / t,
            "speedup_vs_fp64_inner_dd_lower_bound": per64 * 2 * M_dd / t,
            "fp64_note": "extrapolated from 64 timed FP64 sweeps: one plain cycle of %d sweeps (plain FP64 stalls "
                         "above 1e-10 here) and two inner cycles of %d of the all-FP64 path; both are lower "
                         "bounds on the FP64 times, so the speed-ups are too" % (M, M_dd)}


def run_highorder(args):
    import torch

    import paper_1705_00103_gb300 as cj
    torch.cuda.set_device(0)
    cj.build.build()
    stream = torch.cuda.current_stream()
    d = keyed(lambda: highorder_key(cj, stream, args.steps), 0)
    out = {"metric": METRIC, "value": d["gupdates_s"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
           "warmup": 0, "ms_per_step": d["time_to_tol_s"] * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32+f64x2", "data": "synthetic",
           "config": {"workload": d["workload"], "l2_flush": "none needed: grids of 268-537 MB"}}
    out.update(d)
    print(json.dumps(out), flush=True)


def paper_solve(cj, torch, N, st, tol, stream, err_goal=None, check_every=0, method=0, precision=0):
    """One solve of the paper's test problem (Sec. 3.3) with its Dirichlet data: to the
    relative residual tol, or, with err_goal, to that real error (Sec. 3.4); method 1 is
    classical Jacobi."""
    import workloads
    f, ue, g = workloads.paper_problem(N, N)
    fd, ued, Gd = f_to(torch, f), f_to(torch, ue), f_to(torch, cj.dirichlet_ring(N, N, g))
    u = torch.zeros_like(fd)
    with cj.Plan(N, N, st, tol, bc=cj.CJ_BC_DIRICHLET, method=method, precision=precision) as p:
        cj.cj_set_boundary(p.handle, Gd, stream)
        M = p.info()["M"]
        every = max(1, M // 64) if check_every else 0
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        if err_goal is None:
            r = cj.cj_solve(p.handle, fd, u, stream)
        else:
            r = cj.cj_solve_to_error(p.handle, fd, u, ued, err_goal, every, stream)
        e1.record(stream)
        torch.cuda.synchronize()
    r["time_s"] = e0.elapsed_time(e1) * 1e-3
    r["M"] = M
    r["real_error_final"] = float((u - ued).abs().max())
    return r


def f_to(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def table1_ratios(cj, torch, stream, t3, N, tol):
    """Table 1 on this machine: classical Jacobi on the GPU (one solve per stencil, timed with
    CUDA events), and the serial times of both methods extrapolated from the single-threaded
    C oracle's time per sweep on the same grid (the two methods' sweeps cost the same there)
    times each method's sweep count.  ratios["a/b"] = time of a / time of b."""
    import workloads
    from oracle import oracle as orc
    for row in t3:
        st = row["stencil"]
        j = paper_solve(cj, torch, N, st, tol, stream, method=1)
        f, _, g = workloads.paper_problem(N, N)
        G = orc.ghost_ring(N, N, g)
        b = orc.scale_rhs(f)
        u = np.zeros_like(f)
        t0 = time.perf_counter()
        k = 0
        while k < 3 or time.perf_counter() - t0 < 1.0:
            u = orc.sweep_bc(st, u, G, b, 0.25)
            k += 1
        per = (time.perf_counter() - t0) / k
        t = {"j": j["sweeps"] * per, "j_gpu": j["time_s"], "cj": row["sweeps"] * per, "cj_gpu": row["time_s"]}
        row["jacobi_gpu"] = {"sweeps": j["sweeps"], "time_s": j["time_s"], "intervals": j["cycles"],
                             "status": cj.cj_status_string(j["rc"]), "rel_res_l2": j["rel_res_l2"],
                             "real_error": j["real_error_final"]}
        row["serial_oracle_s_per_sweep"] = per
        row["serial_note"] = "j and cj serial times = sweeps x the oracle's time per sweep (%d sweeps timed)" % k
        row["ratios"] = {"%s/%s" % (a, c): t[a] / t[c] for a, c in
                         [("j", "j_gpu"), ("j", "cj"), ("j", "cj_gpu"), ("j_gpu", "cj"), ("j_gpu", "cj_gpu"),
                          ("cj", "cj_gpu")]}


def run_paper(args):
    """The paper's own experiments on its test problem (Sec. 3.3, u = -e^{xy}) with plain FP64
    CJM: (a) the N = 1024 point of Fig. 3 / Table 1 for the 5-, 9- and 17-point stencils, tol =
    N^-2; (b) Fig. 4 right: the 17-point stencil on N = 128 and the 5-point one on N = 2048,
    each until the real error reaches 1e-8 (tested every M/64 sweeps).  A step runs all five
    solves; value = their grid-point updates per second.  After the timed steps, unless
    --no-jacobi, classical Jacobi solves the N = 1024 problems once each for the Table 1
    ratios (table1_ratios)."""
    import torch

    import paper_1705_00103_gb300 as cj
    torch.cuda.set_device(0)
    cj.build.build()
    stream = torch.cuda.current_stream()
    N3, tol3 = 1024, 1.0 / 1024 ** 2
    runs = [("table1", 5, N3, tol3, None), ("table1", 9, N3, tol3, None), ("table1", 17, N3, tol3, None),
            ("fig4", 17, 128, 1e-8, 1e-8), ("fig4", 5, 2048, 1e-8, 1e-8)]

    def step():
        return [paper_solve(cj, torch, N, st, tol, stream, goal, check_every=goal is not None)
                for _, st, N, tol, goal in runs]

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    t_dev = 0.0
    upd = 0
    for _ in range(args.steps):
        res = step()
        t_dev += sum(r["time_s"] for r in res)
        upd += sum(N * N * r["sweeps"] for (_, _, N, _, _), r in zip(runs, res))
    clk = clocks.stop()

    def brief(r, kind, st, N):
        d = {"stencil": st, "N": N, "M": r["M"], "sweeps": r["sweeps"], "cycles": r["cycles"],
             "time_s": r["time_s"], "status": cj.cj_status_string(r["rc"]), "rel_res_l2": r["rel_res_l2"],
             "real_error": r["real_error_final"]}
        if kind == "fig4":
            h = r["history"]
            pick = np.unique(np.linspace(0, len(h) - 1, min(len(h), 17)).astype(int))
            d["real_error_vs_sweeps"] = [[int(h[k, 0]), float(h[k, 1])] for k in pick]
        return d

    t3 = [brief(r, k, st, N) for (k, st, N, _, _), r in zip(runs, res) if k == "table1"]
    # the same problem by FP32 inner cycles in double-FP64 defect correction, to 1e-10
    mixed = []
    for st, N in ((5, 2048), (17, 1024), (17, 2048)):
        r = paper_solve(cj, torch, N, st, 1e-10, stream, precision=cj.CJ_FP32_INNER_DD)
        mixed.append({"stencil": st, "N": N, "fp32_sweeps": r["sweeps"], "outer_steps": r["cycles"],
                      "time_s": r["time_s"], "status": cj.cj_status_string(r["rc"]),
                      "rel_res_l2": r["rel_res_l2"], "real_error": r["real_error_final"]})
    # Fig. 4 right by the same defect correction: the real error is tested at every outer step
    mixed_f4 = []
    for st, N in ((17, 128), (5, 2048)):
        r = paper_solve(cj, torch, N, st, 1e-8, stream, 1e-8, precision=cj.CJ_FP32_INNER_DD)
        mixed_f4.append({"stencil": st, "N": N, "fp32_sweeps": r["sweeps"], "outer_steps": r["cycles"],
                         "time_s": r["time_s"], "status": cj.cj_status_string(r["rc"]),
                         "real_error": r["real_error_final"]})
    if not args.no_jacobi:
        table1_ratios(cj, torch, stream, t3, N3, tol3)
    f4 = [brief(r, k, st, N) for (k, st, N, _, _), r in zip(runs, res) if k == "fig4"]
    out = {"metric": METRIC, "value": upd / t_dev / 1e9, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": t_dev / args.steps * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "the paper's test problem (Sec. 3.3): Delta u = -(x^2+y^2) e^{xy} with the "
                                  "Dirichlet data of u = -e^{xy}; plain FP64 CJM",
                      "table1": "N = 1024, stencils 5/9/17, tol = N^-2",
                      "fig4_right": "17-point N = 128 vs 5-point N = 2048, real error goal 1e-8",
                      "l2_flush": "none: the 2048^2 arrays (34 MB) fit in L2; the timing is of whole solves"},
           "table1": t3, "fig4_right": f4, "mixed_dd_to_1e-10": mixed,
           "fig4_right_mixed_dd": mixed_f4,
           "fig4_sweep_ratio_5pt_over_17pt": f4[1]["sweeps"] / max(1, f4[0]["sweeps"]),
           "fig4_time_ratio_5pt_over_17pt": f4[1]["time_s"] / max(1e-12, f4[0]["time_s"]),
           "clocks": clk}
    print(json.dumps(out), flush=True)


def run_masks(args):
    """Coefficient-mask sweeps (Sec. 3.2) on 4096^2 grids: the polar 5-point mask (planes that
    vary with r only), the bipolar one (a constant mask times a node factor), and random
    position-dependent 9- and 25-point masks (full planes).  Per case the FP64 sweep time comes
    from two cj_sweeps calls (64 and 0 sweeps: the difference removes the import and export);
    then a polar-mask solve of a harmonic function, N = 1024, to tol 1e-10 with its real error.
    value = updates per second over all timed sweeps."""
    import torch

    import paper_1705_00103_gb300 as cj
    from workloads import masks
    torch.cuda.set_device(0)
    cj.build.build()
    stream = torch.cuda.current_stream()
    N = 4096
    cases = [("polar", 5), ("bipolar", 5), ("random", 9), ("random", 25)]
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]

    def problem(name, pat, n):
        if name == "random":
            return masks.random_dominant(pat, n, n, 5)
        return {"polar": masks.polar, "bipolar": masks.bipolar}[name](n, n)

    rows, upd, t_all = [], 0, 0.0
    clocks = ClockSampler(0)
    for name, pat in cases:
        P = problem(name, pat, N)
        coef = f_to(torch, P["coef"])
        scale = None if P["scale"] is None else f_to(torch, P["scale"])
        fd = f_to(torch, P["f"])
        u = torch.zeros_like(fd)
        K = {5: 4, 9: 8, 25: 24}[pat]
        with cj.Plan.mask(N, N, pat, coef, 1e-6, 1.999, 1e-8, scale=scale) as p:
            for _ in range(args.warmup):
                cj.cj_sweeps(p.handle, fd, u, 0, 8, stream)
            torch.cuda.synchronize()
            if not rows:
                clocks.start()
            best = None
            for _ in range(args.steps):
                ev[0].record(stream)
                cj.cj_sweeps(p.handle, fd, u, 0, 0, stream)
                ev[1].record(stream)
                cj.cj_sweeps(p.handle, fd, u, 0, 64, stream)
                ev[2].record(stream)
                torch.cuda.synchronize()
                t = (ev[1].elapsed_time(ev[2]) - ev[0].elapsed_time(ev[1])) * 1e-3 / 64
                best = t if best is None else min(best, t)
                upd += 64 * N * N
                t_all += 64 * t
        full = P["coef"].shape[-1] == N and P["coef"].shape[-2] == N
        bytes_node = 24 + (8 * K if full else 0) + (0 if P["scale"] is None else 0)
        rows.append({"mask": name, "pattern": pat, "layout": "full planes" if full else
                     ("constant planes x node factor" if P["scale"] is not None else "planes varying with x only"),
                     "sweep_us": best * 1e6, "gupd_s": N * N / best / 1e9,
                     "fp64_tops": (K + 2) * N * N / best / 1e12,
                     "fp64_frac_of_issue_peak": (K + 2) * N * N / best / 1e12 / FP64_PEAK_TOPS,
                     "hbm_gbs_algorithmic": bytes_node * N * N / best / 1e9})
        del coef, scale, fd, u
    clk = clocks.stop()
    # a polar solve with its real error
    n = 1024
    P = masks.polar(n, n, solution="harmonic")
    # kmin (n+1)^2 = 4.87, 4.88 for this polar sector at n = 15, 31 (dense eigenvalues); 5 % below
    kmin = 0.95 * 4.88 / (n + 1) ** 2
    G = f_to(torch, cj.dirichlet_ring(n, n, P["g"]))
    fd, ue = f_to(torch, P["f"]), f_to(torch, P["u_exact"])
    u = torch.zeros_like(fd)
    with cj.Plan.mask(n, n, 5, f_to(torch, P["coef"]), kmin, 2.0, 1e-10) as p:
        cj.cj_set_boundary(p.handle, G, stream)
        ev[0].record(stream)
        r = cj.cj_solve(p.handle, fd, u, stream)
        ev[1].record(stream)
        torch.cuda.synchronize()
    solve = {"N": n, "sweeps": r["sweeps"], "cycles": r["cycles"],
             "time_s": ev[0].elapsed_time(ev[1]) * 1e-3, "status": cj.cj_status_string(r["rc"]),
             "rel_res_l2": r["rel_res_l2"], "real_error": float((u - ue).abs().max()), "kmin": kmin}
    out = {"metric": METRIC, "value": upd / t_all / 1e9, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": t_all / args.steps * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "coefficient-mask FP64 sweeps, 4096x4096: polar 5-pt, bipolar 5-pt, random "
                                  "9-pt and 25-pt full planes; plus a polar solve at N = 1024",
                      "l2_flush": "none needed: 134 MB per grid array exceeds the 129 MB L2"},
           "sweeps": rows, "polar_solve": solve, "clocks": clk}
    print(json.dumps(out), flush=True)


def batch_key(cj, stream, autotune: bool = True, steps: int = 1, fp64_every: int = 16) -> dict:
    """Configuration 4: the 512-problem batch (sides log-uniform in [64, 2048], 5/9-point, tol 1e-8,
    FP32-inner / FP64-outer) through cj_solve_batch, after the engine autotuner has picked tile rows
    and depth for each (stencil, size class) on the class's median problem; one warm-up batch, then
    `steps` timed ones.  The FP64 comparison solves every fp64_every-th problem alone by the all-FP64
    path (FP64 CJM cycles in double-FP64 defect correction) and scales the sum of their times by
    fp64_every (labelled)."""
    import torch
    import workloads
    specs = workloads.batch_problems()
    fs = [torch.from_numpy(workloads.smooth_random_rhs(p["Nx"], p["Ny"], p["rhs_seed"])).cuda() for p in specs]
    us = [torch.zeros_like(f) for f in fs]
    probs = [dict(Nx=p["Nx"], Ny=p["Ny"], st=p["st"], tol=p["tol"], precision=cj.CJ_FP32_INNER, f=f, u=u)
             for p, f, u in zip(specs, fs, us)]
    tuned, t_tune = {}, 0.0
    if autotune:
        t0 = time.perf_counter()
        classes = {}
        for p in specs:
            n, c = p["Nx"] * p["Ny"], 0
            while n > 3:
                n >>= 2
                c += 1
            classes.setdefault((p["st"], c), []).append((p["Nx"] * p["Ny"], p["Nx"], p["Ny"]))
        for (st, c), members in sorted(classes.items()):
            _, nx, ny = sorted(members)[len(members) // 2]
            r = cj.cj_autotune_engine(nx, ny, st)
            tuned["%d-point class %d (%dx%d)" % (st, c, nx, ny)] = [r["tile_rows"], r["depth"]]
        t_tune = time.perf_counter() - t0
    for u in us:
        u.zero_()
    cj.cj_solve_batch(probs, stream)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    res = []
    for _ in range(steps):
        for u in us:
            u.zero_()
        res = cj.cj_solve_batch(probs, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    t_batch = ms / steps * 1e-3
    updates = sum(r["sweeps"] * p["Nx"] * p["Ny"] for r, p in zip(res, specs))
    stat = {}
    for r in res:
        k = cj.cj_status_string(r["rc"])
        stat[k] = stat.get(k, 0) + 1
    # the all-FP64 path on a sample, one problem at a time
    t64, upd64, stat64 = 0.0, 0, {}
    sample = list(range(0, len(specs), fp64_every))
    for k in sample:
        p = specs[k]
        with cj.Plan(p["Nx"], p["Ny"], p["st"], p["tol"], precision=cj.CJ_FP64_INNER_DD) as pl:
            u = torch.zeros_like(fs[k])
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = cj.cj_solve(pl.handle, fs[k], u, stream)
            t64 += time.perf_counter() - t0
        upd64 += r["sweeps"] * p["Nx"] * p["Ny"]
        nm = cj.cj_status_string(r["rc"])
        stat64[nm] = stat64.get(nm, 0) + 1
    fp64_all = t64 * fp64_every
    return {"workload": "batched: 512 Dirichlet problems, Nx, Ny log-uniform in [64, 2048], 5/9-point, tol 1e-8, "
                        "FP32-inner / FP64-outer, one engine per batch", "steps": steps,
            "points": sum(p["Nx"] * p["Ny"] for p in specs),
            "time_to_all_converged_s": t_batch, "gupdates_s": updates / t_batch / 1e9, "statuses": stat,
            "max_rel_res_l2": max(r["rel_res_l2"] for r in res),
            "autotuned_tile_rows_depth": tuned, "autotune_s": t_tune,
            "gpu_launches": res[0]["launches"] if res else 0,
            "fp64_one_at_a_time_s_extrapolated": fp64_all,
            "fp64_sample": {"problems": len(sample), "every": fp64_every, "time_s": t64, "statuses": stat64,
                            "gupdates_s": upd64 / t64 / 1e9 if t64 > 0 else None},
            "speedup_vs_fp64_one_at_a_time": fp64_all / t_batch,
            "fp64_note": "all-FP64 path (FP64 CJM cycles in double-FP64 defect correction, which reaches 1e-8 on "
                         "every size where plain FP64 cycles may stall), one problem at a time; time of every "
                         "%d-th problem (host time of cj_solve), summed and scaled by %d" % (fp64_every, fp64_every)}


def run_batch(args):
    import torch

    import paper_1705_00103_gb300 as cj
    torch.cuda.set_device(0)
    cj.build.build()
    stream = torch.cuda.current_stream()
    d = keyed(lambda: batch_key(cj, stream, autotune=not args.no_autotune, steps=args.steps), 0)
    out = {"metric": METRIC, "value": d["gupdates_s"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
           "warmup": 1, "ms_per_step": d["time_to_all_converged_s"] * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
           "config": {"workload": d["workload"], "points": d["points"]}}
    out.update(d)
    print(json.dumps(out), flush=True)


def serve_key(cj, n_requests: int, fp64_every: int = 4, fp64_max_nodes: int = 1 << 22) -> dict:
    """Configuration 5, an arrival-faithful prefix: the first n_requests requests of the seeded
    Poisson stream (lambda = 2000/s, sides log-uniform in [32, 8192], 5/9/17-point, tol 1e-6 or
    1e-10) submitted at their arrival times to one server with a 150 GB budget and 64 slots per
    lane.  Latency = submit to result ready; service time = admission to result ready.  Offered
    load = the prefix's updates / its arrival window; achieved = updates / wall time.  The FP64
    comparison solves every fp64_every-th request of at most fp64_max_nodes nodes alone, by plain
    FP64 CJM for tol 1e-6 and by the all-FP64 defect correction for 1e-10."""
    import workloads
    import torch
    reqs = workloads.request_stream()[:n_requests]
    fs = [workloads.smooth_random_rhs(r["Nx"], r["Ny"], r["rhs_seed"]) for r in reqs]
    lat, svc, upd, got = [], [], 0, {}
    with cj.Server(150 * 10 ** 9, 64) as srv:
        t0 = time.perf_counter()
        tickets = {}
        k = 0
        while k < len(reqs) or tickets:
            now = time.perf_counter() - t0
            while k < len(reqs) and reqs[k]["t_arrival"] <= now:
                tickets[srv.submit(fs[k], reqs[k]["st"], reqs[k]["tol"])] = k
                k += 1
            for t, j in list(tickets.items()):
                g = srv.poll(t, fs[j].shape)
                if g is not None:
                    got[j] = g[1]
                    lat.append(g[1]["seconds"])
                    svc.append(g[1]["sweep_seconds"])
                    upd += g[1]["sweeps"] * reqs[j]["Nx"] * reqs[j]["Ny"]
                    del tickets[t]
            time.sleep(0.0002)
        wall = time.perf_counter() - t0
        stats = srv.stats()
    window = reqs[-1]["t_arrival"]
    stat = {}
    for j in got:
        nm = cj.cj_status_string(got[j]["rc"])
        stat[nm] = stat.get(nm, 0) + 1
    # service time a request needs alone, median over the sizes: its own work
    own = []
    sample = [j for j in range(0, len(reqs), fp64_every) if reqs[j]["Nx"] * reqs[j]["Ny"] <= fp64_max_nodes]
    fp64 = []
    stream = torch.cuda.current_stream()
    for j in sample:
        r = reqs[j]
        fd = torch.from_numpy(fs[j]).cuda()
        prec = cj.CJ_FP64 if r["tol"] >= 1e-6 else cj.CJ_FP64_INNER_DD
        with cj.Plan(r["Nx"], r["Ny"], r["st"], r["tol"], precision=prec) as pl:
            u = torch.zeros_like(fd)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            rr = cj.cj_solve(pl.handle, fd, u, stream, check=False)
            dt = time.perf_counter() - t1
        fp64.append({"request": j, "Nx": r["Nx"], "Ny": r["Ny"], "st": r["st"], "tol": r["tol"],
                     "fp64_s": dt, "fp64_status": cj.cj_status_string(rr["rc"]),
                     "served_latency_s": got[j]["seconds"], "served_service_s": got[j]["sweep_seconds"]})
        own.append(dt)
    # every request of the prefix by the FP64 path, one at a time, as a lower bound: its FP64 sweep
    # time (8 timed sweeps) x the fewest sweeps an FP64 solve can take (the plain cycle length M for
    # tol 1e-6, which plain FP64 reaches; for 1e-10 the all-FP64 path's two inner cycles, or M if less)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    lower = 0.0
    for j, r in enumerate(reqs):
        fd = torch.from_numpy(fs[j]).cuda()
        with cj.Plan(r["Nx"], r["Ny"], r["st"], r["tol"], launch=cj.CJ_LAUNCH_STREAM) as pl:
            M = pl.info()["M"]
            g = torch.zeros_like(fd)
            cj.cj_sweeps(pl.handle, fd, g, 0, 2, stream)
            torch.cuda.synchronize()
            e0.record(stream)
            cj.cj_sweeps(pl.handle, fd, g, 0, 8, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            t0s = e0.elapsed_time(e1) * 1e-3
            e0.record(stream)
            cj.cj_sweeps(pl.handle, fd, g, 0, 0, stream)  # the import and export alone
            e1.record(stream)
            torch.cuda.synchronize()
            per = max(0.0, t0s - e0.elapsed_time(e1) * 1e-3) / 8
        n_min = M
        if r["tol"] < 1e-6:
            with cj.Plan(r["Nx"], r["Ny"], r["st"], r["tol"], precision=cj.CJ_FP64_INNER_DD) as pdd:
                n_min = min(M, 2 * pdd.info()["M_inner"])
        lower += per * n_min
        del fd, g
    return {"workload": "served: arrival-faithful prefix of the seeded Poisson stream (2000/s), first %d of "
                        "10,000 requests, sides log-uniform in [32, 8192], 5/9/17-point, tol 1e-6 / 1e-10, "
                        "budget 150 GB" % len(reqs),
            "requests": len(reqs), "full_stream": "10,000 requests: not run (about 80x the GPU's throughput "
                                                 "over its 5 s arrival window)",
            "latency_s": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                          "max": float(max(lat))},
            "service_s": {"p50": float(np.percentile(svc, 50)), "p99": float(np.percentile(svc, 99))},
            "statuses": stat,
            "offered_gupdates_s": upd / window / 1e9, "achieved_gupdates_s": upd / wall / 1e9,
            "arrival_window_s": window, "wall_s": wall, "server": stats,
            "fp64_one_at_a_time": {"requests": fp64, "sum_fp64_s": sum(x["fp64_s"] for x in fp64),
                                   "sum_served_service_s": sum(x["served_service_s"] for x in fp64),
                                   "median_fp64_s": float(np.median(own)) if own else None,
                                   "note": "every %d-th request of at most %d nodes, alone: plain FP64 CJM for tol "
                                           "1e-6, FP64 cycles in double-FP64 defect correction for 1e-10; for these "
                                           "small requests the FP64 path alone is faster than their service in the "
                                           "mix, whose engine spends ~2.5 launches per sweep"
                                           % (fp64_every, fp64_max_nodes)},
            "fp64_whole_prefix_lower_bound_s_extrapolated": lower,
            "speedup_vs_fp64_one_at_a_time_lower_bound": lower / wall,
            "fp64_whole_prefix_note": "every request of the prefix by the FP64 path one at a time: its FP64 sweep "
                                      "time (8 timed sweeps) x the fewest sweeps an FP64 solve can take (the plain "
                                      "cycle length for 1e-6; for 1e-10 two inner cycles of the all-FP64 path, or the "
                                      "plain cycle if shorter); a lower bound, so the speed-up is one too"}


def run_serve(args):
    import torch

    import paper_1705_00103_gb300 as cj
    torch.cuda.set_device(0)
    cj.build.build()
    d = keyed(lambda: serve_key(cj, args.serve_requests), 0)
    out = {"metric": METRIC, "value": d["achieved_gupdates_s"], "unit": UNIT, "n_gpus": 1, "steps": 1,
           "warmup": 0, "ms_per_step": d["wall_s"] * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic", "config": {"workload": d["workload"]}}
    out.update(d)
    print(json.dumps(out), flush=True)


def run_reference(args):
    """The oracle as the reference arm: each step a bounded sample (4 sweeps) of the same
    workload, on the host cores, rank 0 only."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from oracle import oracle as orc
    f = make_rhs(1)
    b = orc.scale_rhs(f)
    kmin, kmax = orc.kappa_bounds(STENCIL, N_GRID, N_GRID)
    M = orc.cycle_length(kmin, kmax, TOL)
    w = orc.sweep_coeffs(STENCIL, kmin, kmax, M)
    u = np.zeros_like(b)
    per_step = 4

    def step(k):
        nonlocal u
        for s in range(per_step):
            u = orc.sweep(STENCIL, u, b, w[(k * per_step + s) % M])

    for k in range(args.warmup):
        step(k)
    t0 = time.perf_counter()
    for k in range(args.steps):
        step(args.warmup + k)
    dt = time.perf_counter() - t0
    value = N_GRID * N_GRID * per_step * args.steps / dt / 1e9
    sample = ("%d FP64 9-point CJM sweeps of the 4096x4096 grid per step, single-threaded C oracle"
              % per_step)
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": "plain CJM FP64, 9-point alpha=2/3 stencil, 4096x4096 interior, "
                                  "homogeneous Dirichlet, tol 1e-10 (bounded sample per step)",
                      "Nx": N_GRID, "Ny": N_GRID, "stencil": STENCIL, "tol": TOL},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main(argv=None):
    args = parse_args(argv)
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "highorder":
        run_highorder(args)
    elif args.workload == "paper":
        run_paper(args)
    elif args.workload == "masks":
        run_masks(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "serve":
        run_serve(args)
    else:
        run_cj(args)


if __name__ == "__main__":
    main()
