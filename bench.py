"""Benchmark: time-tiled acoustic forward sweep (and its untiled baseline) on GB300.

Default workload (one "step" = one wave_fwd call = the whole forward path):
512^3 grid, space order 8, two-layer velocity with +-2% noise, 40-point
damping layer, 1000 time steps, one Ricker source and 512 receivers, fused
injection and interpolation.  Metric: grid-point updates per second (GPts/s)
= nx*ny*nz*nt / seconds, device-timed with inputs resident in HBM; each field
(512 MiB) is larger than L2, so no flush is needed between steps.

Also reported: the untiled sweep on the same workload, the end-to-end rate
through the C ABI with host buffers (pinned H2D copies of m, damp and the
source trace, D2H of the receiver traces, inside the timed region), the
roofline of the sweep kernel from CUDA events the library records around its
launches, the FWI gradient time per shot (256^3, so 8, 2000 steps,
checkpoints every 50 steps), SM clocks sampled during the timed region, and
the FP64 CPU oracle timed on a bounded sample of the workload.

`--impl reference` times the oracle itself (the CPU reference of this
method) on the same workload and metric.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "acoustic stencil GPts/s tiled vs untiled, % roofline; FWI gradient s/shot"
HBM_FALLBACK_GBS = 6800.0


# DRAM traffic of one launch of the bench's sweep at full size
# (dram__bytes_read.sum + dram__bytes_write.sum from one single-pass ncu capture;
# profiles/traffic_tsweep_t2_so8_512.md), valid only for the kernel sources it was
# taken on: the SHA-256 of csrc/sweep.cuh, csrc/tsweep.cuh and the radius-4
# variant lists must match, else the bench reports null.
TRAFFIC_SRC_SHA256 = "de67d7eb9a0fcf2381682edcccbbaf4a084634580ad2a99bc76c93eeb874d1a0"
TRAFFIC_BYTES = {  # ("family R T V rows BZ BY P", chunk, n) -> bytes per launch
    ("staged R4 T2 V4 rows2 BZ64 BY24 P1", 103, (512, 512, 512)): 2334687744 + 1043836672,
}


def _kernel_sha256():
    """SHA-256 of what the bench kernel is built from: csrc/sweep.cuh (its
    PTX helpers), csrc/tsweep.cuh and the radius-4 variant lists of
    csrc/variants.h (other radii do not change it)."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1806_08299_gb300", "csrc")
    for f in ("sweep.cuh", "tsweep.cuh"):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    with open(os.path.join(csrc, "variants.h"), "r") as fh:
        text = fh.read()
    for key in ("#define WAVE_SWEEP_VARIANTS_R4(", "#define WAVE_TSWEEP_VARIANTS_R4("):
        a = text.index(key)
        b = text.index("#define", a + 1)
        h.update(text[a:b].encode())
    return h.hexdigest()


def _traffic(space_order, plan, n):
    if TRAFFIC_SRC_SHA256 is None or _kernel_sha256() != TRAFFIC_SRC_SHA256:
        return None
    fam = "staged" if plan.get("kernel") == 2 else "shared"
    key = ("%s R%d T%d V%d rows%d BZ%d BY%d P%d" % (fam, space_order // 2, plan["time_tile"], plan["vec"],
                                                   plan["rows"], plan["tile_z"], plan["tile_y"],
                                                   plan["prefetch"]),
           plan["tile_x"], tuple(n))
    return TRAFFIC_BYTES.get(key)


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = max(smax, float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x, dist=None, device=None):
    """Largest x over the ranks of the default process group (x itself when
    there is none): the job is as slow as its slowest replica."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gradient_bytes_per_point_step(t_forward, t_recompute, t_adjoint):
    """Compulsory HBM bytes per grid point and time step of one FWI gradient
    shot at the depths its three passes ran.  Forward: u^n, u^{n-1}, B, C read
    and u^{n+1} written, 20 B untiled; a depth-2 launch reads the four once
    and writes two levels, 24 B per two steps.  Recompute storing D: E read
    and D written besides, 28 B untiled, 36 B per two steps at depth 2 (two
    levels and two D rows written).  Adjoint with the imaging condition: D
    and G read and G written besides, 32 B untiled, 40 B per two steps at
    depth 2 (two D rows read, G read and written once)."""
    fwd = 24.0 / 2 if t_forward >= 2 else 20.0
    rec = 36.0 / 2 if t_recompute >= 2 else 28.0
    adj = 40.0 / 2 if t_adjoint >= 2 else 32.0
    return fwd + rec + adj


def whole_job_rate(pts_per_rank, steps, ms, world):
    """GPts/s of `world` replicas that each update pts_per_rank points per
    step for `steps` steps, over the slowest rank's `ms` milliseconds."""
    return world * pts_per_rank * steps / (ms / 1e3) / 1e9


def _workload(args):
    from paper_1806_08299_gb300 import inputs
    if args.workload == "c1":
        p = inputs.c1(nt=args.nt or 100)
        desc = "c1: 64^3 so4 constant 1.5 km/s, no damping, %d steps, Ricker 10 Hz, 32 receivers" % p.nt
    else:
        n = (args.size,) * 3
        p = inputs.c2(nt=args.nt or 1000, n=n)
        desc = ("c2: %d^3 so8 two-layer 1.5/2.5 km/s +-2%% noise, 40-pt damping, %d steps, "
                "1 Ricker 15 Hz source, %d receivers, fused inject/interp" % (n[0], p.nt, len(p.rec_xyz)))
    return p, desc


def _cpu_sample(p, target_s=15.0, max_steps=64):
    """Time the FP64 oracle on the top z-slab of the workload (the part that
    holds the source and receivers), sized to ~target_s seconds of host work."""
    import oracle
    ncores = os.cpu_count() or 1
    oracle.set_threads(ncores)
    nzs = min(p.n[2], 64)
    m = np.ascontiguousarray(p.m[:, :, :nzs], dtype=np.float64)
    damp = np.ascontiguousarray(p.damp[:, :, :nzs], dtype=np.float64)
    h = [float(np.float32(v)) for v in p.h]
    dt = float(np.float32(p.dt))
    q = p.src_q.astype(np.float64)

    def run(steps):
        t0 = time.perf_counter()
        oracle.forward(m, damp, h, dt, steps, p.space_order, p.src_xyz.astype(np.float64),
                       q[:steps], p.rec_xyz.astype(np.float64))
        return time.perf_counter() - t0

    t2 = run(2)
    steps = int(max(2, min(max_steps, target_s / max(t2 / 2, 1e-6))))
    dt_run = run(steps)
    pts = m.size * steps
    # the paper's skewed time-tiled loop nest (time tile 4, 8 x 8 space tiles), and the untiled
    # loop on one core, each on 8 steps of the same slab
    t0 = time.perf_counter()
    oracle.forward_tiled(m, damp, h, dt, 8, p.space_order, p.src_xyz.astype(np.float64), q[:8],
                         p.rec_xyz.astype(np.float64), tt=4, bx=8, by=8)
    t_tiled = time.perf_counter() - t0
    oracle.set_threads(1)
    t_one = run(2)
    oracle.set_threads(ncores)
    return {"value": pts / dt_run / 1e9, "unit": "GPts/s", "cores": oracle.max_threads(),
            "kind": "oracle", "seconds": dt_run,
            "tiled_value": m.size * 8 / t_tiled / 1e9,
            "single_core_value": m.size * 2 / t_one / 1e9,
            "sample": "FP64 oracle forward (untiled loop, OpenMP) on the top %d-plane z-slab "
                      "%dx%dx%d of the workload for %d steps; tiled_value: the paper's skewed "
                      "time-tiled loop (tt 4, 8x8 tiles) on 8 steps; single_core_value: the untiled "
                      "loop on one core, 2 steps" % (nzs, p.n[0], p.n[1], nzs, steps)}


def run_reference(args):
    rank, world, _ = _dist()
    if rank != 0:
        return
    p, desc = _workload(args)
    import oracle
    ncores = os.cpu_count() or 1
    oracle.set_threads(ncores)
    nzs = min(p.n[2], 32)
    m = np.ascontiguousarray(p.m[:, :, :nzs], dtype=np.float64)
    damp = np.ascontiguousarray(p.damp[:, :, :nzs], dtype=np.float64)
    h = [float(np.float32(v)) for v in p.h]
    dt = float(np.float32(p.dt))
    q = p.src_q.astype(np.float64)
    steps = 2

    def one():
        t0 = time.perf_counter()
        oracle.forward(m, damp, h, dt, steps, p.space_order, p.src_xyz.astype(np.float64),
                       q[:steps], p.rec_xyz.astype(np.float64))
        return time.perf_counter() - t0

    for _ in range(args.warmup):
        one()
    times = [one() for _ in range(args.steps)]
    tot = sum(times)
    val = m.size * steps * args.steps / tot / 1e9
    sample = ("FP64 oracle forward (untiled, OpenMP) on the top %d-plane z-slab %dx%dx%d for %d "
              "steps per bench step" % (nzs, p.n[0], p.n[1], nzs, steps))
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": "GPts/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": desc, "sample": sample},
        "cpu_baseline": {"value": val, "unit": "GPts/s", "cores": oracle.max_threads(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": val, "unit": "GPts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def _timed(fn, steps, stream):
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    extra = [fn() for _ in range(steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), extra


def _model_line(space_order, plan):
    """Traffic model of the plan's shape: DRAM and L2 -> shared-memory bytes
    per point-update (paper_1806_08299_gb300.traffic_model)."""
    from paper_1806_08299_gb300 import traffic_model as tm
    shape = tm.Shape(R=space_order // 2, T=plan["time_tile"], V=plan["vec"], BZ=plan["tile_z"],
                     BY=plan["tile_y"], kernel=plan["kernel"])
    return {"dram_bytes_per_point": tm.dram_bytes_per_update(plan["time_tile"]),
            "l2_bytes_per_point": tm.l2_bytes_per_update(shape),
            "stage_points_per_update": shape.stage_points_per_update()}


def _per_call(fn, n, stream):
    """Device time of each of n consecutive calls (CUDA events on the stream
    between calls): the spread behind the timed mean."""
    import torch
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(n + 1)]
    torch.cuda.synchronize()
    ev[0].record(stream)
    for i in range(n):
        fn()
        ev[i + 1].record(stream)
    torch.cuda.synchronize()
    return [ev[i].elapsed_time(ev[i + 1]) for i in range(n)]


def _spread(ms_list, pts):
    ms_sorted = sorted(ms_list)
    med = float(np.median(ms_sorted))
    return {"runs": len(ms_list), "min_ms": ms_sorted[0], "median_ms": med,
            "max_gpts": pts / (ms_sorted[0] / 1e3) / 1e9, "median_gpts": pts / (med / 1e3) / 1e9}


def run_section_only(args):
    """One section alone (one GPU), for profiling its kernels."""
    import torch
    from paper_1806_08299_gb300 import inputs, wave
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    if args.only_survey:
        print(json.dumps({"fwi_survey": _fwi_survey(dev, inputs, wave, args)}))
    if args.only_fwi:
        print(json.dumps({"fwi_gradient": _fwi_gradient(dev, inputs, wave, args)}))
    if args.only_laplace:
        print(json.dumps({"laplace": _laplace_sweep(dev, inputs, wave, args)}))


def run_ours(args):
    import torch
    from paper_1806_08299_gb300 import inputs, wave
    rank, world, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    p, desc = _workload(args)
    grid = wave.Grid(p.n, p.h, p.dt, p.nt, p.space_order)
    tm = torch.from_numpy(p.m).to(dev)
    td = torch.from_numpy(p.damp).to(dev)
    tq = torch.from_numpy(p.src_q).to(dev)
    stream = torch.cuda.current_stream()
    nsrc, nrec = len(p.src_xyz), len(p.rec_xyz)
    ws = torch.empty(wave.workspace_bytes(grid, wave.WAVE_OP_FWD, nsrc, nrec), dtype=torch.uint8,
                     device=dev)
    pts = float(np.prod(p.n)) * p.nt

    def fwd(tune):
        d, _, _, _ = wave.fwd(grid, tm, td, p.src_xyz, tq, p.rec_xyz, tuning=tune, workspace=ws)
        return wave.sweep_stats() if tune.flags & wave.WAVE_TIME_SWEEPS else None

    def barrier():
        if dist is not None:
            dist.barrier()

    def slowest(x):
        return max_over_ranks(x, dist, dev)

    # autotune once (outside any timed region), then fix the plans: the
    # product plan (every depth, shape and kernel family), the fastest untiled
    # sweep (every T = 1 shape of both families) and the fastest time-tiled
    # sweep (every T >= 2 shape of both families)
    def tuned(tune):
        fwd(tune)
        pl = wave.describe_plan(grid, tune)
        return wave.Tuning(time_tile=pl["time_tile"], tile_y=pl["tile_y"], tile_x=pl["tile_x"],
                           vec=pl["vec"], tile_z=pl["tile_z"], kernel=pl["kernel"], rows=pl["rows"])

    def timing(t):
        return wave.Tuning(t.time_tile, t.tile_y, t.tile_x, wave.WAVE_TIME_SWEEPS, t.vec, t.tile_z,
                           t.kernel, t.rows)
    if args.time_tile:
        tiled = tuned(wave.Tuning(time_tile=args.time_tile, flags=wave.WAVE_AUTOTUNE_SHAPE))
    else:
        tiled = tuned(wave.Tuning(time_tile=0))
    try:  # candidates the autotuner considered and those its runtime bound pruned
        tune_stats = dict(zip(("candidates", "pruned"), wave.autotune_stats()))
    except wave.WaveError:  # plan read from the plan cache: no autotuner ran
        tune_stats = None
    untiled = tuned(wave.Tuning(time_tile=1, flags=wave.WAVE_AUTOTUNE_SHAPE))
    depths = sorted({v["time_tile"] for v in wave.list_variants(p.space_order) if v["time_tile"] >= 2})
    deep_plans = [tuned(wave.Tuning(time_tile=T, flags=wave.WAVE_AUTOTUNE_SHAPE)) for T in depths]
    plan = wave.describe_plan(grid, tiled)
    uplan = wave.describe_plan(grid, untiled)
    prof = timing(tiled)

    # --- device-timed, inputs resident: the product plan (headline) --------
    for _ in range(args.warmup):
        fwd(prof)
    sampler = ClockSampler(local)
    sampler.start()
    barrier()
    ms, stats = _timed(lambda: fwd(prof), args.steps, stream)
    barrier()
    clocks = sampler.stop()
    ms = slowest(ms)
    value = whole_job_rate(pts, args.steps, ms, world)
    sweep_ms = sum(s[0] for s in stats)
    launches = sum(s[1] for s in stats)

    def side(t):
        """The same workload on a fixed plan: whole-call rate and the mean
        duration of its sweep launches."""
        tt = timing(t)
        fwd(tt)
        barrier()
        ms_s, st = _timed(lambda: fwd(tt), args.steps, stream)
        ms_s = slowest(ms_s)
        pl = wave.describe_plan(grid, t)
        sw = sum(x[0] for x in st)
        nl = sum(x[1] for x in st)
        return {"gpts": whole_job_rate(pts, args.steps, ms_s, world), "plan": pl,
                "avg_launch_ms": sw / max(nl, 1), "launches_per_call": nl // max(args.steps, 1)}

    # --- the fastest untiled and time-tiled plans, same workload ------------
    untiled_line = side(untiled)
    untiled_gpts = untiled_line["gpts"]
    deep_lines = [side(t) for t in deep_plans]
    deep_line = max(deep_lines, key=lambda r: r["gpts"]) if deep_lines else None

    # --- spread over single calls (after the timed region) -----------------
    spread = None
    if args.spread_runs > 0:
        spread = {"product": _spread(_per_call(lambda: fwd(tiled), args.spread_runs, stream), pts),
                  "untiled": _spread(_per_call(lambda: fwd(untiled), args.spread_runs, stream), pts)}

    # --- end to end through the C ABI with host buffers --------------------
    hm = torch.from_numpy(p.m).pin_memory()
    hd = torch.from_numpy(p.damp).pin_memory()
    hq = torch.from_numpy(p.src_q).pin_memory()
    hrec = torch.empty((p.nt, nrec), dtype=torch.float32).pin_memory()
    dm, dd, dq = torch.empty_like(tm), torch.empty_like(td), torch.empty_like(tq)

    def e2e_step():
        dm.copy_(hm, non_blocking=True)
        dd.copy_(hd, non_blocking=True)
        dq.copy_(hq, non_blocking=True)
        d, _, _, _ = wave.fwd(grid, dm, dd, p.src_xyz, dq, p.rec_xyz, tuning=tiled, workspace=ws)
        hrec.copy_(d, non_blocking=True)

    e2e_step()
    barrier()
    ms_e, _ = _timed(e2e_step, args.steps, stream)
    ms_e = slowest(ms_e)
    h2d = (hm.numel() + hd.numel() + hq.numel()) * 4
    d2h = hrec.numel() * 4

    # --- FWI gradient per shot (256^3 so 8, 2000 steps, k = 50) -------------
    fwi = None
    if args.fwi and world == 1:
        fwi = _fwi_gradient(dev, inputs, wave, args)
    survey = None
    if args.survey and world == 1:
        survey = _fwi_survey(dev, inputs, wave, args)
    orders = None
    if args.orders and world == 1:
        orders = _orders_sweep(dev, inputs, wave, args)
    laplace = None
    if args.laplace and world == 1:
        laplace = _laplace_sweep(dev, inputs, wave, args)

    # --- roofline of the sweep kernels ---------------------------------------
    hbm, peak_kind = _peaks()
    fp32_tflops, smem_tbs = wave.measure_peaks()
    flops_per_pt = 7 * (p.space_order // 2) + 10  # per radius 6 adds + 1 FMA; centre and update

    def roof(pl, avg_ms, traffic=None):
        """Algorithmic HBM bytes of one launch (24 B per point for a time tile
        -- read u^n, u^{n-1}, B, C, write two levels -- 20 B untiled) over its
        mean duration, against the measured copy bandwidth; and the same
        launch's point-updates against the FP32 FMA roof at F(r) flops each."""
        T = pl["time_tile"]
        bpp = 24 if T >= 2 else 20
        alg = float(np.prod(p.n)) * bpp
        ach = alg / (avg_ms / 1e3) / 1e9
        gpts = float(np.prod(p.n)) * T / (avg_ms / 1e3) / 1e9
        alu_roof = fp32_tflops * 1e3 / flops_per_pt
        fam = "tsweep_kernel" if pl["kernel"] == wave.WAVE_KERNEL_STAGED else "sweep_kernel"
        return {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                "traffic": traffic, "peak_kind": peak_kind,
                "kernel": "%s<R=%d,T=%d>" % (fam, p.space_order // 2, T),
                "algorithmic_bytes_per_launch": alg, "avg_launch_ms": avg_ms,
                "hbm_roof_gpts": hbm / (bpp / T), "sweep_gpts": gpts,
                "alu": {"fp32_tflops_measured": fp32_tflops, "flops_per_point": flops_per_pt,
                        "roof_gpts": alu_roof, "frac": gpts / alu_roof},
                "smem_tbs_measured": smem_tbs,
                # the launch's point-updates at the untiled sweep's 20 B each: above
                # the measured HBM bandwidth (frac > 1) a time tile delivers more
                # updates than any untiled sweep could at that bandwidth
                "untiled_equivalent": {"bytes_per_point": 20, "gbs": gpts * 20.0,
                                       "frac": gpts * 20.0 / hbm},
                "model": _model_line(p.space_order, pl)}

    T = plan["time_tile"]
    avg_launch_ms = sweep_ms / max(launches, 1)
    roofline = roof(plan, avg_launch_ms,
                    args.traffic if args.traffic is not None else _traffic(p.space_order, plan, p.n))
    untiled_line["roofline"] = roof(uplan, untiled_line["avg_launch_ms"])
    if deep_line is not None:
        deep_line["roofline"] = roof(deep_line["plan"], deep_line["avg_launch_ms"])
        deep_line["tiled_over_untiled"] = deep_line["gpts"] / untiled_gpts
        deep_line["all_depths"] = [{"time_tile": r["plan"]["time_tile"], "gpts": r["gpts"]}
                                   for r in deep_lines]

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = _cpu_sample(p)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GPts/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": desc, "l2": "inputs larger than L2 (512 MiB per field)",
                       "plan": plan, "per_call_spread": spread, "autotune": tune_stats,
                       "parallelism": "replicas" if world > 1 else "single"},
            "untiled": untiled_line,
            "time_tiled": deep_line,
            "tiled_over_untiled": deep_line["tiled_over_untiled"] if deep_line else None,
            "e2e": {"value": whole_job_rate(pts, args.steps, ms_e, world), "unit": "GPts/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "roofline": roofline,
            "gpu_launches": args.steps * (launches // max(args.steps, 1) + 2),
            "clocks": clocks,
        }
        if fwi is not None:
            line["fwi_gradient"] = fwi
        if survey is not None:
            line["fwi_survey"] = survey
        if orders is not None:
            line["orders_c3"] = orders
        if laplace is not None:
            line["laplace"] = laplace
        if cpu is not None:
            line["cpu_baseline"] = cpu
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


def _fwi_gradient(dev, inputs, wave, args):
    """Forward with checkpoints + recompute + adjoint + imaging condition for
    one 256^3 so-8 shot of 2000 steps, k = 50 (s per shot); the same gradient
    by binomial checkpointing with 40 and 10 stored states (wave_grad_revolve:
    s per shot, forward steps, device bytes); Born modelling of the shot along
    the sphere the initial model lacks (wave_born: both fields in one fused
    sweep per step, 40 B per point-update; and the two-sweep form, a
    background sweep storing D and a perturbation sweep, 28 + 28 B)."""
    import torch
    p = inputs.c4(nt=args.fwi_nt, true_model=False)
    grid = wave.Grid(p.n, p.h, p.dt, p.nt, p.space_order)
    tm = torch.from_numpy(p.m).to(dev)
    td = torch.from_numpy(p.damp).to(dev)
    tq = torch.from_numpy(p.src_q).to(dev)
    k = 50
    tune = wave.Tuning(time_tile=0)

    def shot():
        d, _, ckpt, _ = wave.fwd(grid, tm, td, p.src_xyz, tq, p.rec_xyz, tuning=tune, ckpt_every=k)
        g, _ = wave.grad(grid, tm, td, p.src_xyz, tq, p.rec_xyz, d, ckpt, k, tuning=tune)
        return g

    shot()
    torch.cuda.synchronize()
    ms, _ = _timed(shot, 1, torch.cuda.current_stream())
    plan = wave.describe_plan(grid, tune)
    pts = float(np.prod(p.n))
    nrec = len(p.rec_xyz)
    out = {"s_per_shot": ms / 1e3, "workload": "c4: 256^3 so8, %d steps, checkpoints every %d, "
           "forward + recompute + adjoint + imaging condition" % (p.nt, k),
           "time_tile": plan["time_tile"],
           "gpts_equiv": 3 * pts * p.nt / (ms / 1e3) / 1e9,
           "device_bytes": wave.ckpt_bytes(grid, k) + wave.workspace_bytes(grid, wave.WAVE_OP_GRAD, 1, nrec, k)}
    # HBM roof of the shot at the depths its three passes ran (checkpoint
    # copies not counted)
    gp = wave.describe_grad_plan(grid, len(p.src_xyz), nrec, k, tuning=tune)
    tf, tr, ta = plan["time_tile"], gp["recompute"]["time_tile"], gp["adjoint"]["time_tile"]
    bps = gradient_bytes_per_point_step(tf, tr, ta)
    roof_s = pts * p.nt * bps / (_peaks()[0] * 1e9)
    out["roofline"] = {"bound": "hbm", "bytes_per_point_step": bps, "roof_s_per_shot": roof_s,
                       "frac": roof_s / (ms / 1e3), "peak_gbs": _peaks()[0],
                       "depths": {"forward": tf, "recompute": tr, "adjoint": ta}}
    out["gradient_plans"] = gp

    # the same gradient by binomial checkpointing, no forward call first
    d, _, _, _ = wave.fwd(grid, tm, td, p.src_xyz, tq, p.rec_xyz, tuning=tune)
    rev = []
    for ns in (40, 10):
        ws_r = torch.empty(wave.workspace_bytes(grid, wave.WAVE_OP_REVOLVE, 1, nrec, ns), dtype=torch.uint8,
                           device=dev)

        def shot_rev():
            return wave.grad_revolve(grid, tm, td, p.src_xyz, tq, p.rec_xyz, d, ns, tuning=tune, workspace=ws_r)

        shot_rev()
        torch.cuda.synchronize()
        ms_r, _ = _timed(shot_rev, 1, torch.cuda.current_stream())
        rev.append({"slots": ns, "s_per_shot": ms_r / 1e3, "forward_steps": wave.revolve_forward_steps(p.nt, ns),
                    "device_bytes": ws_r.numel()})
        del ws_r
    out["revolve"] = rev
    out["uniform_forward_steps"] = 2 * p.nt

    # Born modelling on the same shot: dm = the sphere the initial model lacks
    pt = inputs.c4(nt=args.fwi_nt, true_model=True)
    tdm = torch.from_numpy((pt.m - p.m).astype(np.float32)).to(dev)
    del pt

    def born():
        return wave.born(grid, tm, td, tdm, p.src_xyz, tq, p.rec_xyz, tuning=tune)

    born()
    torch.cuda.synchronize()
    ms_b, _ = _timed(born, 1, torch.cuda.current_stream())
    gpts_b = pts * p.nt / (ms_b / 1e3) / 1e9
    out["born"] = {"s_per_shot": ms_b / 1e3, "gpts": gpts_b, "kernel": "fused (one sweep per step)",
                   "dram_bytes_per_point": 40.0, "hbm_roof_gpts": _peaks()[0] / 40.0,
                   "frac_hbm": gpts_b * 40.0 / _peaks()[0]}

    def born2():
        return wave.born(grid, tm, td, tdm, p.src_xyz, tq, p.rec_xyz,
                         tuning=wave.Tuning(time_tile=0, flags=wave.WAVE_BORN_TWO_SWEEPS))

    born2()
    torch.cuda.synchronize()
    ms_b2, _ = _timed(born2, 1, torch.cuda.current_stream())
    gpts_b2 = pts * p.nt / (ms_b2 / 1e3) / 1e9
    out["born_two_sweeps"] = {"s_per_shot": ms_b2 / 1e3, "gpts": gpts_b2, "dram_bytes_per_point": 56.0,
                              "frac_hbm": gpts_b2 * 56.0 / _peaks()[0]}
    torch.cuda.empty_cache()
    return out


def _fwi_survey(dev, inputs, wave, args):
    """One FWI gradient step over the first shots of the c5 survey (windows of
    one 512 x 512 x 256 model, so 8, 1500 steps, k = 50): the batched forward
    for the predicted traces, then the batched gradient (forward with
    checkpoints, recompute, adjoint and imaging condition) with the predicted
    traces as residual (an all-zero observed-data stand-in).  s per shot."""
    import torch
    sv = inputs.c5(nshots=args.survey_shots, nt=args.survey_nt, true_model=False)
    grid = wave.Grid(sv.n, sv.h, sv.dt, sv.nt, sv.space_order)
    tm = torch.from_numpy(sv.m).to(dev)
    td = torch.from_numpy(sv.damp).to(dev)
    shots = [wave.Shot(origin=x["origin"], n=x["n"], src_xyz=x["src_xyz"], rec_xyz=x["rec_xyz"])
             for x in sv.shots]
    q = [torch.from_numpy(x).to(dev) for x in sv.src_q]
    k = 50
    conc = min(len(shots), 8)  # shots per lockstep group (8 groups of 8 for the whole survey)
    tune = wave.Tuning()  # each group times its forward kernel (once per group shape, cached)
    ws_f = torch.empty(wave.batch_workspace_bytes(grid, shots, 0, conc), dtype=torch.uint8, device=dev)
    ws_g = torch.empty(wave.batch_workspace_bytes(grid, shots, k, conc), dtype=torch.uint8, device=dev)

    def step():
        d, _ = wave.fwd_batched(grid, shots, tm, td, q, concurrency=conc, tuning=tune, workspace=ws_f)
        g, _ = wave.grad_batched(grid, shots, tm, td, q, d, k, concurrency=conc, tuning=tune,
                                 workspace=ws_g)
        return g

    step()
    torch.cuda.synchronize()
    ms, _ = _timed(step, 1, torch.cuda.current_stream())
    pts = sum(int(np.prod(x["n"])) for x in sv.shots)
    plan_f = wave.describe_batch_plan(grid, shots, 0, conc, tune)
    plan_g = wave.describe_batch_plan(grid, shots, k, conc, tune)

    def kname(p):
        if p is None:
            return "per shot"
        return "%s T=%d %dx%d rows %d" % ("staged" if p["kernel"] == wave.WAVE_KERNEL_STAGED else "shared-warp",
                                          p["time_tile"], p["tile_z"], p["tile_y"], p["rows"])
    return {"s_per_shot": ms / 1e3 / len(shots),
            "workload": "c5: %d of 64 shots (windows of a 512x512x256 layered model), so8, "
                        "%d steps, k = %d, %d shots per lockstep group (one launch per step or per T steps, "
                        "CUDA graph); batched forward + batched gradient"
                        % (len(shots), sv.nt, k, conc),
            "forward_kernel": kname(plan_f),
            "gradient_forward_kernel": kname(plan_g),
            "gradient_recompute_adjoint_kernel": (
                "per shot" if plan_g is None else "%s T=%d" % (
                    "staged" if plan_g["grad_kernel"] == wave.WAVE_KERNEL_STAGED else "shared-warp",
                    plan_g["grad_time_tile"])),
            "status": wave.status(ws_g),
            "gpts_equiv": 4 * pts * sv.nt / (ms / 1e3) / 1e9}


def _orders_sweep(dev, inputs, wave, args):
    """c3: 768 x 768 x 512, smooth random velocity 1.5-4.5 km/s, 40-point
    damping, one source.  Per space order 4/8/12/16: the fastest untiled plan
    and the fastest time-tiled plan (every compiled depth T >= 2, shapes
    autotuned), each timed over args.orders_nt steps with the inputs resident,
    as GPts/s and as a fraction of the HBM roof at the plan's algorithmic
    bytes per point-update (20 untiled, 24/T time-tiled)."""
    import torch
    p0 = inputs.c3(space_order=4, nt=args.orders_nt)
    tm = torch.from_numpy(p0.m).to(dev)
    td = torch.from_numpy(p0.damp).to(dev)
    hbm, _ = _peaks()
    pts = float(np.prod(p0.n)) * p0.nt
    stream = torch.cuda.current_stream()
    out = {"workload": "c3: 768x768x512, smooth random velocity 1.5-4.5 km/s, 40-pt damping, "
                       "1 Ricker 15 Hz source, %d steps per timing" % p0.nt}
    for so in (4, 8, 12, 16):
        dt = inputs.DT[("c3", so)]
        grid = wave.Grid(p0.n, p0.h, dt, p0.nt, so)
        q = np.ascontiguousarray(inputs.ricker(15.0, dt, p0.nt)[:, None], dtype=np.float32)
        tq = torch.from_numpy(q).to(dev)
        ws = torch.empty(wave.workspace_bytes(grid, wave.WAVE_OP_FWD, 1, 0), dtype=torch.uint8,
                         device=dev)

        def fwd(tune):
            wave.fwd(grid, tm, td, p0.src_xyz, tq, None, tuning=tune, workspace=ws)

        def best_at(T):
            t = wave.Tuning(time_tile=T, flags=wave.WAVE_AUTOTUNE_SHAPE)
            fwd(t)
            try:
                st = dict(zip(("candidates", "pruned"), wave.autotune_stats()))
            except wave.WaveError:
                st = None
            pl = wave.describe_plan(grid, t)
            fixed = wave.Tuning(time_tile=pl["time_tile"], tile_y=pl["tile_y"], tile_x=pl["tile_x"],
                                vec=pl["vec"], tile_z=pl["tile_z"], kernel=pl["kernel"], rows=pl["rows"])
            fwd(fixed)
            ms, _ = _timed(lambda: fwd(fixed), 1, stream)
            g = pts / (ms / 1e3) / 1e9
            bpp = 20.0 if T == 1 else 24.0 / T
            return {"gpts": g, "frac_hbm": g * bpp / hbm, "bytes_per_point": bpp, "plan": pl,
                    "autotune": st}

        row = {"untiled": best_at(1)}
        depths = sorted({v["time_tile"] for v in wave.list_variants(so) if v["time_tile"] >= 2})
        tiled = [best_at(T) for T in depths]
        row["time_tiled"] = max(tiled, key=lambda r: r["gpts"]) if tiled else None
        row["tiled_over_untiled"] = (row["time_tiled"]["gpts"] / row["untiled"]["gpts"]
                                     if tiled else None)
        if not tiled:
            row["note"] = "no time-tiled shape of this order fits the shared-memory and register budget"
        out["so%d" % so] = row
        del ws
        torch.cuda.empty_cache()
    return out


def _laplace_sweep(dev, inputs, wave, args):
    """The Laplace (heat) operator of Sec. 5.7 on its 600^3 grid, 16 steps:
    explicit Euler for u_t = lap u from a smooth seeded field, per space
    order 2/4/8/16 the fastest untiled plan and the fastest time-tiled plan
    (every compiled depth T >= 2, shapes autotuned), GPts/s of the sweeps
    (best of three calls; call_gpts: whole calls, set-up included).  The sweep
    is the wave sweep with B = 0, so it still reads level n-1 and B (20 B per
    point-update where the operator needs 12).  adams_bashforth2: the same
    operator by the two-step Adams-Bashforth scheme (a time dependence of two
    levels, Sec. 6), untiled (20 B per point-update) and at depth 2 (10 B),
    sweep time of the call's launches (its first step is an untiled Euler
    step)."""
    import torch
    n = (args.laplace_n,) * 3
    nt = 16
    h = (inputs.H,) * 3
    rng = np.random.default_rng(7)
    idx = [np.arange(k, dtype=np.float32) / k for k in n]
    u0 = (np.sin(2 * np.pi * idx[0])[:, None, None] * np.cos(4 * np.pi * idx[1])[None, :, None]
          * np.sin(6 * np.pi * idx[2])[None, None, :]).astype(np.float32)
    u0 += np.float32(0.01) * rng.standard_normal(n).astype(np.float32)
    tu = torch.from_numpy(u0).to(dev)
    del u0
    pts = float(np.prod(n)) * nt
    stream = torch.cuda.current_stream()
    out = {"workload": "Laplace operator (Sec. 5.7): %dx%dx%d, %d steps, explicit Euler, "
                       "smooth seeded field" % (n + (nt,))}
    for so in (2, 4, 8, 16):
        c = wave.fd_coefficients(so)  # |symbol| at the Nyquist corner bounds explicit Euler
        sig = abs(c[0] + 2 * sum(c[k] * (-1) ** k for k in range(1, len(c))))
        lam = sum(sig / (hh * hh) for hh in h)
        grid = wave.Grid(n, h, float(np.float32(0.4 * 2.0 / lam)), nt, so)
        ws = torch.empty(wave.workspace_bytes(grid, wave.WAVE_OP_FWD, 0, 0), dtype=torch.uint8,
                         device=dev)

        def run(tune):
            wave.heat(grid, tu, None, None, None, None, tuning=tune, workspace=ws)

        def best_at(T):
            t = wave.Tuning(time_tile=T, flags=wave.WAVE_AUTOTUNE_SHAPE)
            run(t)
            pl = wave.describe_plan(grid, t)
            fixed = wave.Tuning(time_tile=pl["time_tile"], tile_y=pl["tile_y"], tile_x=pl["tile_x"],
                                vec=pl["vec"], flags=wave.WAVE_TIME_SWEEPS, tile_z=pl["tile_z"],
                                kernel=pl["kernel"], rows=pl["rows"])
            run(fixed)
            best = float("inf")
            for _ in range(3):  # the sweeps alone (16 steps leave per-call set-up visible)
                run(fixed)
                best = min(best, wave.sweep_stats()[0])
            ms, _ = _timed(lambda: run(fixed), 3, stream)
            return {"gpts": pts / (best / 1e3) / 1e9, "call_gpts": 3 * pts / (ms / 1e3) / 1e9, "plan": pl}

        row = {"untiled": best_at(1)}
        depths = sorted({v["time_tile"] for v in wave.list_variants(so) if v["time_tile"] >= 2})
        tiled = [best_at(T) for T in depths]
        row["time_tiled"] = max(tiled, key=lambda r: r["gpts"]) if tiled else None
        row["tiled_over_untiled"] = (row["time_tiled"]["gpts"] / row["untiled"]["gpts"]
                                     if tiled else None)

        # the two-step Adams-Bashforth form (time dependence 2): untiled and
        # depth 2 (where compiled), dt within its limit dt |L| <= 1
        grid2 = wave.Grid(n, h, float(np.float32(0.4 / lam)), nt, so)

        def ab2_at(T):
            t = wave.Tuning(time_tile=T, flags=wave.WAVE_TIME_SWEEPS)
            wave.heat_ab2(grid2, tu, None, None, None, None, tuning=t, workspace=ws)
            best, launches = float("inf"), 0
            for _ in range(3):
                wave.heat_ab2(grid2, tu, None, None, None, None, tuning=t, workspace=ws)
                st = wave.sweep_stats()
                best, launches = min(best, st[0]), st[1]
            gpts = pts / (best / 1e3) / 1e9
            bpp = 20.0 if T == 1 else 10.0
            return {"gpts": gpts, "launches_per_call": launches, "dram_bytes_per_point": bpp,
                    "frac_hbm": gpts * bpp / _peaks()[0]}

        ab1 = ab2_at(1)
        ab = {"untiled": ab1}
        if so in (2, 4, 8):
            ab["time_tiled"] = ab2_at(2)
            ab["tiled_over_untiled"] = ab["time_tiled"]["gpts"] / ab1["gpts"]
        row["adams_bashforth2"] = ab
        out["so%d" % so] = row
        del ws
        torch.cuda.empty_cache()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c2", choices=["c1", "c2"])
    ap.add_argument("--size", type=int, default=512)
    ap.add_argument("--nt", type=int, default=0)
    ap.add_argument("--time-tile", type=int, default=0)
    ap.add_argument("--no-fwi", dest="fwi", action="store_false")
    ap.add_argument("--no-survey", dest="survey", action="store_false")
    ap.add_argument("--survey-shots", type=int, default=64)
    ap.add_argument("--survey-nt", type=int, default=1500)
    ap.add_argument("--no-orders", dest="orders", action="store_false")
    ap.add_argument("--no-laplace", dest="laplace", action="store_false")
    ap.add_argument("--laplace-n", type=int, default=600)
    ap.add_argument("--spread-runs", type=int, default=10,
                    help="single calls timed one by one after the timed region (min / median)")
    ap.add_argument("--orders-nt", type=int, default=500)
    ap.add_argument("--fwi-nt", type=int, default=2000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--traffic", type=float, default=None,
                    help="ncu dram bytes per sweep launch, when captured for this kernel")
    ap.add_argument("--only-survey", action="store_true",
                    help="run only the batched survey (FWI gradient step over c5 shots) and print its entry")
    ap.add_argument("--only-fwi", action="store_true",
                    help="run only the c4 gradient, revolve and Born entry and print it")
    ap.add_argument("--only-laplace", action="store_true",
                    help="run only the Laplace operator entry (leapfrog-form and Adams-Bashforth sweeps)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.only_survey or args.only_fwi or args.only_laplace:
        run_section_only(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
