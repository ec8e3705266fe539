"""Runs a fixed number of CJM sweeps through the C ABI, for kernel profiling (ncu).

    python -m paper_1705_00103_gb300.profile_sweeps --stencil 9 --n 4096 --precision fp64 --count 3
    python -m paper_1705_00103_gb300.profile_sweeps --stencil 9 --precision fp32 --depth 8 --count 16
    python -m paper_1705_00103_gb300.profile_sweeps --stencil 9 --n 4096 --solve fp32_inner_dd
    python -m paper_1705_00103_gb300.profile_sweeps --stencil 9 --n 4096 --precision ff --count 16
    python -m paper_1705_00103_gb300.profile_sweeps --stencil 9 --n 1024 --batch 24 --depth 4

Inputs are zero grids of the given size (the sweep's cost does not depend on the values);
three FP64 grids of 4096^2 (400 MB) exceed the 129 MB L2.
"""
from __future__ import annotations

import argparse


def main(argv=None):
    import torch

    from . import cj
    from . import build
    ap = argparse.ArgumentParser()
    ap.add_argument("--stencil", type=int, default=9)
    ap.add_argument("--n", type=int, default=4096)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32", "ff"],
                    help="ff: the FP64 sweep in float-float on the FP32 pipe (cj_sweeps_ff)")
    ap.add_argument("--count", type=int, default=3)
    ap.add_argument("--depth", type=int, default=1, help="FP32 sweeps per launch (temporal blocking)")
    ap.add_argument("--time", type=int, default=0,
                    help="also time this many sweeps with CUDA events and print us per sweep")
    ap.add_argument("--solve", default="", choices=["", "fp32_inner", "fp32_inner_dd"],
                    help="instead of sweeps, one mixed-precision solve of the smooth random RHS "
                         "(seed 2) to a relative residual of 1e-10, at the default temporal depth")
    ap.add_argument("--batch", type=int, default=0,
                    help="instead of sweeps, cj_solve_batch of this many n x n problems (smooth random "
                         "RHSs, FP32 inner, tol 1e-8) at temporal depth --depth")
    a = ap.parse_args(argv)
    build.build()
    if a.batch:
        import workloads
        probs = []
        for k in range(a.batch):
            f = torch.from_numpy(workloads.smooth_random_rhs(a.n, a.n, 50 + k)).cuda()
            probs.append(dict(Nx=a.n, Ny=a.n, st=a.stencil, tol=1e-8, precision=cj.CJ_FP32_INNER,
                              temporal_depth=a.depth, f=f, u=torch.zeros_like(f)))
        res = cj.cj_solve_batch(probs)
        torch.cuda.synchronize()
        print("batch of %d %dx%d stencil %d depth %d: %d sweeps each, %.3f s"
              % (a.batch, a.n, a.n, a.stencil, a.depth, res[0]["sweeps"], res[0]["seconds"]))
        print("ok")
        return
    if a.solve:
        import workloads
        prec = cj.CJ_FP32_INNER if a.solve == "fp32_inner" else cj.CJ_FP32_INNER_DD
        f = torch.from_numpy(workloads.smooth_random_rhs(a.n, a.n, 2)).cuda()
        with cj.Plan(a.n, a.n, a.stencil, 1e-10, precision=prec) as p:
            u = torch.zeros_like(f)
            res = cj.cj_solve(p.handle, f, u)
        torch.cuda.synchronize()
        print("%s solve %dx%d stencil %d: %d FP32 sweeps, %d outer steps, rel residual %.3e, %.3f s"
              % (a.solve, a.n, a.n, a.stencil, res["sweeps"], res["cycles"], res["rel_res_l2"], res["seconds"]))
        print("ok")
        return

    def run(fn):
        fn(a.count)
        torch.cuda.synchronize()
        if a.time > 0:
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            fn(a.time)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            e0.record()
            fn(0)
            e1.record()
            torch.cuda.synchronize()
            per = (ms - e0.elapsed_time(e1)) / a.time
            print("stencil %d %s depth %d %dx%d: %.2f us per sweep, %.1f Gupdates/s"
                  % (a.stencil, a.precision, a.depth, a.n, a.n, per * 1e3, a.n * a.n / per / 1e6))

    if a.precision in ("fp64", "ff"):
        sweeps = cj.cj_sweeps if a.precision == "fp64" else cj.cj_sweeps_ff
        with cj.Plan(a.n, a.n, a.stencil, 1e-10) as p:
            f = torch.zeros((a.n, a.n), dtype=torch.float64, device="cuda")
            u = torch.zeros_like(f)
            run(lambda c: sweeps(p.handle, f, u, 0, c))
    else:
        with cj.Plan(a.n, a.n, a.stencil, 1e-10, precision=cj.CJ_FP32_INNER, temporal_depth=a.depth) as p:
            r = torch.zeros((a.n, a.n), dtype=torch.float32, device="cuda")
            e = torch.zeros_like(r)
            run(lambda c: cj.cj_sweeps_f32(p.handle, r, e, 0, c))
    print("ok")


if __name__ == "__main__":
    main()
