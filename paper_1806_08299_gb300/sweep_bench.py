"""Time the compiled sweep variants on a synthetic workload.

    python -m paper_1806_08299_gb300.sweep_bench --n 512 --so 8            # every variant
    python -m paper_1806_08299_gb300.sweep_bench --n 256 --so 8 --time-tile 1 --tile-y 8 --vec 4
    python -m paper_1806_08299_gb300.sweep_bench --grad --n 256 --nt 32 --ckpt-every 8 --time-tile 2

The workload is the two-layer model of `inputs.c2` on an n^3 grid with a
fixed number of steps.  For each variant it runs `--reps` forward calls and
reports the best milliseconds per time step of the sweep launches (CUDA
events the library records on the launch stream) and the resulting GPts/s.
This is also the small case that the ncu summaries under profiles/ capture.
With --grad it times wave_grad instead: the FWI gradient of the c4 model
family (sphere-free initial model, one source, 256 receivers) on an n^3 grid,
after a forward call with checkpoints, and prints the shapes its recompute and
adjoint sweeps ran.
It is a measurement driver for profiling, not part of the library's API.
"""
import argparse
import json

import torch

from . import inputs, wave


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--so", type=int, default=8)
    ap.add_argument("--nt", type=int, default=8)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--time-tile", type=int, default=0, help="0 = every compiled variant")
    ap.add_argument("--tile-y", type=int, default=0)
    ap.add_argument("--vec", type=int, default=0)
    ap.add_argument("--tile-z", type=int, default=0)
    ap.add_argument("--tile-x", type=int, default=0, help="x-chunk (0 = default)")
    ap.add_argument("--kernel", type=int, default=0, help="1 shared-warp, 2 stage-specialised (0 = any)")
    ap.add_argument("--rows", type=int, default=0, help="rows per thread (0 = any)")
    ap.add_argument("--grad", action="store_true", help="time wave_grad on the c4 model family")
    ap.add_argument("--ckpt-every", type=int, default=8)
    args = ap.parse_args()
    if args.grad:
        return grad_main(args)
    p = inputs.c2(nt=args.nt, n=(args.n,) * 3)
    grid = wave.Grid(p.n, p.h, p.dt, p.nt, args.so)
    tm, td, tq = (torch.from_numpy(a).cuda() for a in (p.m, p.damp, p.src_q))
    if args.time_tile:
        cands = [dict(time_tile=args.time_tile, tile_y=args.tile_y, vec=args.vec, tile_z=args.tile_z,
                      kernel=args.kernel, rows=args.rows)]
    else:
        cands = [v for v in wave.list_variants(args.so) if args.kernel in (0, v["kernel"])]
    for v in cands:
        tune = wave.Tuning(time_tile=v["time_tile"], tile_y=v["tile_y"], vec=v["vec"],
                           tile_x=args.tile_x, flags=wave.WAVE_TIME_SWEEPS, tile_z=v.get("tile_z", 0),
                           kernel=v.get("kernel", 0), rows=v.get("rows", 0))
        best = float("inf")
        for _ in range(args.reps):
            _, _, _, ws = wave.fwd(grid, tm, td, p.src_xyz, tq, p.rec_xyz, tuning=tune)
            ms, launches, steps = wave.sweep_stats()
            best = min(best, ms / steps)
        status = wave.status(ws)
        plan = wave.describe_plan(grid, tune)
        print(json.dumps(dict(plan, n=args.n, so=args.so, ms_per_step=best,
                              gpts=args.n ** 3 / (best / 1e3) / 1e9, status=status)), flush=True)


def grad_main(args):
    p = inputs.c4(nt=args.nt, n=(args.n,) * 3, true_model=False)
    grid = wave.Grid(p.n, p.h, p.dt, p.nt, args.so)
    tm, td, tq = (torch.from_numpy(a).cuda() for a in (p.m, p.damp, p.src_q))
    k = args.ckpt_every
    tune = wave.Tuning(time_tile=args.time_tile, flags=wave.WAVE_TIME_SWEEPS, kernel=args.kernel)
    d, _, ckpt, _ = wave.fwd(grid, tm, td, p.src_xyz, tq, p.rec_xyz, tuning=tune, ckpt_every=k)
    best = float("inf")
    for _ in range(args.reps):
        _, ws = wave.grad(grid, tm, td, p.src_xyz, tq, p.rec_xyz, d, ckpt, k, tuning=tune)
        ms, launches, steps = wave.sweep_stats()
        best = min(best, ms)
    status = wave.status(ws)
    plans = wave.describe_grad_plan(grid, len(p.src_xyz), len(p.rec_xyz), k, tuning=tune)
    print(json.dumps(dict(n=args.n, so=args.so, nt=args.nt, ckpt_every=k, sweep_ms=best,
                          ms_per_step=best / args.nt, plans=plans, status=status)), flush=True)


if __name__ == "__main__":
    main()
