#!/usr/bin/env python
"""Throughput of the arbitrary-shape-surface Fresnel transform on GB300.

Metric: source samples per second of the forward transform (Eq. 8) on the
2048 x 2048 smooth-random-surface workload (4 um pitch, 633 nm, z0 = 0.1 m,
oversampling 2, ES kernel width 7), with the relative L2 error against the
FP64 direct-sum oracle on sampled destination points.

One step = one pass of the whole hot path over one synthetic input: the
per-sample prefactor + tiled spread, the row FFT, and the column FFT with
deconvolution and destination chirp, on inputs already resident in HBM.  L2
is flushed (a 512 MiB write) between timed steps, outside the timed region.
Each rank of a multi-GPU run processes its own copy of the workload (the path
shards by independent surfaces; no collective on the data path).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "source samples/sec at 2048^2 (forward transform, rel-L2 vs FP64 oracle)"
UNIT = "samples/s"
WORKLOAD = "smooth_random2048"
FALLBACK_HBM_GBS = 6800.0
# seconds of untimed back-to-back steps under clock sampling before the timed region
CLOCK_LOAD_S = 0.5
# extra lines after the headline (each on the same single GPU)
EXTRAS = ("peaks", "deterministic", "es_widths", "learned", "direct_sum", "line", "multi", "adjoint",
          "batch", "fft_reference")


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--width", type=int, default=7)
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--cpu-seconds", type=float, default=10.0,
                    help="target CPU time of the oracle baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the width sweep, learned kernel, adjoint and batch lines")
    ap.add_argument("--extras", default="all",
                    help="comma-separated subset of the extra lines: " + ", ".join(EXTRAS))
    args = ap.parse_args()
    args.extras = set(EXTRAS) if args.extras == "all" else set(args.extras.split(","))
    unknown = args.extras - set(EXTRAS)
    if unknown:
        ap.error(f"unknown extras: {sorted(unknown)}")
    return args


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(x: float, device, world: int) -> float:
    """Maximum of a per-rank time over the process group (identity at N = 1)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """Units processed by all ranks (each rank runs its own replica of the
    workload) per second of the slowest rank."""
    return world * units_per_rank / seconds


def workload_config(name, width):
    return {"workload": f"{name}: 2048x2048 source at 4 um, smooth random surface (sigma 40 "
                        "samples, 0-50 um), amplitude U[0,1], phase U[0,2pi), 633 nm, z0 0.1 m, "
                        "2048x2048 destination at 4 um" if name == WORKLOAD else name,
            "method": "type-1 NUFFT, ES kernel", "kernel_width": width, "sigma": 2,
            "precision": "FP32 spread/FFT/deconvolution, FP64-built phase tables",
            "l2": "flushed between timed steps (512 MiB write)"}


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, interval_ms: int = 50):
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", str(interval_ms)],
                stdout=self.file, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None

    def wait_first_sample(self, timeout_s: float = 5.0):
        """Block until nvidia-smi has written a line (it needs ~0.1-1 s to start)."""
        t = time.perf_counter()
        while self.proc is not None and time.perf_counter() - t < timeout_s:
            self.file.flush()
            if os.path.getsize(self.file.name) > 0:
                return
            time.sleep(0.02)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [r.split(",") for r in self.file.read().strip().splitlines() if r.strip()]
        os.unlink(self.file.name)
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for name, val in zip(names, r[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm),
                "window": f"warm-up, {CLOCK_LOAD_S} s of the same steps back to back, timed region"}


def keep_busy(step, flush, seconds, synchronize, batch=16):
    """Runs flush.zero_() and step() back to back, untimed, for about `seconds`,
    synchronising every `batch` steps; returns the number of steps run."""
    n = 0
    end = time.perf_counter() + seconds
    while time.perf_counter() < end:
        for _ in range(batch):
            flush.zero_()
            step()
            n += 1
        synchronize()
    return n


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "MEASURED_PEAKS.json hbm_gbs (of measured)"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "profiling-recipe fallback 6.8 TB/s (of fallback)"


def stage_bytes(info, g):
    """Algorithmic HBM bytes per launch of each stage: the spread reads u1 and
    q (12 B per sample) plus the axis tables and writes the band of the fine
    grid once; the row pass reads the band and writes band rows x m2x; the
    column pass reads those and writes u2 plus the destination tables."""
    n = g["n1x"] * g["n1y"]
    band_rows = info["band_y1"] - info["band_y0"]
    band_cols = info["band_x1"] - info["band_x0"]
    tables = 2 * (g["n1x"] + g["n1y"]) * 24
    spread = n * (8 + 4) + band_rows * band_cols * 8 + tables
    rows = band_rows * band_cols * 8 + band_rows * g["m2x"] * 8
    cols = band_rows * g["m2x"] * 8 + g["m2x"] * g["m2y"] * 8 + (g["m2x"] + g["m2y"]) * 8
    return [spread, rows, cols]


STAGE_KERNELS = ["spread", "fft_rows_kernel", "fft_cols_kernel"]
SPREAD_KERNEL = {0: "spread_es_colored_kernel", 1: "spread_es_atomic_kernel",
                 2: "spread_es_window_kernel", 3: "spread_es_dense_kernel",
                 4: "spread_item_kernel"}
# bytes per source sample of the whole forward step in the unpruned model:
# u1 + d1 (12) + fine-grid write (4 M^2 8 / N^2 = 32) + row read (32) + row write
# (16) + column read (16) + u2 write (8), sigma = 2 and N = M
STEP_BYTES_PER_SAMPLE = 116
# DRAM bytes (read + write) per launch of the dominant kernel from one ncu
# capture, with the SHA-1 of the kernel's code (the files that define it and
# the per-sample arithmetic it inlines) and its launch grid at the time of the
# capture: the traffic is reported only while both are unchanged (a kernel
# changed since its capture, or without one, reports null)
SPREAD_SOURCES = ("paper_1203_3583_gb300/csrc/spread.cuh", "paper_1203_3583_gb300/csrc/sample.cuh")
NCU_TRAFFIC = {("spread_es_dense_kernel<7>", "smooth_random2048"): {
    "bytes": 86.784000e6 + 1.624832e6,
    "grid": 912,
    "capture": "profiles/spread_es_dense_w7_smooth_random2048.md",
    "sources_sha1": "025f3964b6ff962a8ece156c70b2c7dcb768ebdb"}}


def sources_sha1(paths) -> str:
    import hashlib
    h = hashlib.sha1()
    for rel in paths:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def captured_traffic(kernel: str, workload: str, grid: int):
    """(DRAM bytes per launch or None, provenance note)."""
    rec = NCU_TRAFFIC.get((kernel, workload))
    if rec is None:
        return None, "no ncu capture of this kernel and workload"
    if sources_sha1(SPREAD_SOURCES) != rec["sources_sha1"]:
        return None, f"kernel sources changed since the capture in {rec['capture']}"
    if grid != rec["grid"]:
        return None, f"launch grid {grid} differs from the capture's {rec['grid']}"
    return rec["bytes"], (f"ncu capture in {rec['capture']} (sources sha1 "
                          f"{rec['sources_sha1'][:12]}, grid {grid})")


def oracle_sample(g, u1, d1, seconds, seed=7):
    """Time the FP64 oracle on a bounded sample of destination points.
    Returns (samples_per_s, cores, n_points, elapsed, points, values)."""
    import oracle
    from paper_1203_3583_gb300 import workloads as W
    n = g["n1x"] * g["n1y"]
    m = g["m2x"] * g["m2y"]
    probe = W.sample_points(g, 8, seed=seed + 1)
    t = time.perf_counter()
    oracle.eq7(g, u1, d1, points=probe)
    dt = max(time.perf_counter() - t, 1e-6)
    npts = int(max(8, min(m, round(8 * seconds / dt))))
    pts = W.sample_points(g, npts, seed=seed)
    t = time.perf_counter()
    vals = oracle.eq7(g, u1, d1, points=pts)
    el = time.perf_counter() - t
    samples_per_s = n * npts / (el * m)
    return samples_per_s, oracle.max_threads(), npts, el, pts, vals


def run_reference(args):
    """The reference arm: the FP64 oracle as it stands, on the host cores."""
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    import numpy as np  # noqa: F401
    import oracle
    from paper_1203_3583_gb300 import workloads as W
    g, u1, d1 = W.make(args.workload)
    n = g["n1x"] * g["n1y"]
    m = g["m2x"] * g["m2y"]
    npts = 16
    times = []
    for i in range(args.warmup + args.steps):
        pts = W.sample_points(g, npts, seed=1000 + i)
        t = time.perf_counter()
        oracle.eq7(g, u1, d1, points=pts)
        if i >= args.warmup:
            times.append(time.perf_counter() - t)
    t_step = statistics.mean(times)
    value = n * npts / (t_step * m)
    cores = oracle.max_threads()
    sample = (f"{npts} seeded destination points per step of the {g['m2x']}x{g['m2y']} grid, "
              f"each a direct FP64 sum over all {n} source samples; value = source samples / "
              "(step time x destination points / sampled points)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t_step * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args.workload, args.width),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1203_3583_gb300 import capi, workloads as W
    from paper_1203_3583_gb300.fresnel import FresnelPlan

    world, rank, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    capi.load()
    dev = torch.device("cuda", local)

    g, u1, d1 = W.make(args.workload)
    n_src = g["n1x"] * g["n1y"]
    t0 = time.perf_counter()
    plan = FresnelPlan(g, d1, kernel_width=args.width)
    torch.cuda.synchronize()
    plan_ms = (time.perf_counter() - t0) * 1e3
    # re-planning for a new height map, as an optimisation loop does each
    # step (asfd_plan_update_d1 from a device-resident d1; wall clock)
    d1_dev = [torch.as_tensor(d1, device=dev), torch.as_tensor(d1 * 0.99, device=dev)]
    upd = []
    for k in range(6):
        torch.cuda.synchronize()
        t = time.perf_counter()
        plan.update_d1(d1_dev[k % 2])
        torch.cuda.synchronize()
        upd.append((time.perf_counter() - t) * 1e3)
    plan.update_d1(d1_dev[0])
    update_d1_ms = statistics.median(upd[1:])
    del d1_dev
    info = plan.info()
    u1_d = torch.as_tensor(u1, device=dev)
    u2_d = torch.empty(plan.shape2, dtype=torch.complex64, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step(ev):
        ev[0].record(stream)
        plan.execute_stage(0, u1=u1_d)
        ev[1].record(stream)
        plan.execute_stage(1)
        ev[2].record(stream)
        plan.execute_stage(2, out=u2_d)
        ev[3].record(stream)

    # clocks are sampled from the start of the warm-up to the end of the timed
    # region; the timed region alone is shorter than one sample period, so the
    # same steps also run back to back (untimed) for about half a second just
    # before it, and the samples see the GPU under this workload's load
    clocks = ClockSampler(local) if rank == 0 else None
    if clocks:
        clocks.wait_first_sample()
    for _ in range(args.warmup):
        flush.zero_()
        step([torch.cuda.Event(enable_timing=True) for _ in range(4)])
    torch.cuda.synchronize()
    if clocks:
        load_evs = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        keep_busy(lambda: step(load_evs), flush, CLOCK_LOAD_S, torch.cuda.synchronize)
    plan.check_device_status()

    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.zero_()
        step(evs[i])
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if world > 1:
        dist.barrier()
    clk = clocks.stop() if clocks else None
    plan.check_device_status()

    step_ms = [e[0].elapsed_time(e[3]) for e in evs]
    stage_ms = [[e[s].elapsed_time(e[s + 1]) for e in evs] for s in range(3)]
    ms = max_over_ranks(statistics.mean(step_ms), dev, world)
    value = whole_job_rate(n_src, world, ms * 1e-3)

    # roofline of the dominant kernel (algorithmic bytes / event-timed duration)
    sb = stage_bytes(info, g)
    mean_stage = [statistics.mean(s) for s in stage_ms]
    dom = int(np.argmax(mean_stage))
    peak, peak_src = measured_peaks()
    achieved = sb[dom] / (mean_stage[dom] * 1e-3) / 1e9
    names = [f"{SPREAD_KERNEL[info['spread_kind']]}<{args.width}>"] + STAGE_KERNELS[1:]
    # launch grid of the dense spread: warp items of 32 columns x run_rows rows, 4 per block
    n_items = -(-g["n1x"] // 32) * -(-g["n1y"] // max(1, info["run_rows"]))
    traffic, traffic_src = captured_traffic(names[dom], args.workload, -(-n_items // 4))
    roofline = {"bound": "hbm", "kernel": names[dom], "achieved": achieved, "peak": peak,
                "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "traffic_source": traffic_src,
                "algorithmic_bytes_per_launch": sb[dom], "peak_source": peak_src,
                "stage_ms": {k: v for k, v in zip(names, mean_stage)},
                "stage_frac": {k: b / (t * 1e-3) / 1e9 / peak
                               for k, b, t in zip(names, sb, mean_stage)}}
    # the whole step against the memory traffic it must make: the pruned bytes
    # of its three kernels (only the band of the fine grid that footprints
    # reach is written and transformed), and beside it the unpruned
    # spread+FFT model of 116 B per source sample
    t_step = statistics.mean(step_ms) * 1e-3
    pruned = sum(sb)
    step_bytes = STEP_BYTES_PER_SAMPLE * n_src
    step_roofline = {"bound": "hbm", "model": "pruned bytes of the three kernels",
                     "bytes_per_step": pruned, "achieved": pruned / t_step / 1e9,
                     "peak": peak, "unit": "GB/s", "frac": pruned / t_step / 1e9 / peak,
                     "unpruned_bytes_per_sample": STEP_BYTES_PER_SAMPLE,
                     "unpruned_bytes_per_step": step_bytes,
                     "unpruned_frac": step_bytes / t_step / 1e9 / peak}

    # end to end through the C ABI with pinned host buffers
    hu1 = torch.as_tensor(u1).pin_memory()
    hu2 = torch.empty(plan.shape2, dtype=torch.complex64).pin_memory()
    for _ in range(max(1, args.warmup)):
        plan.execute_host(hu1, hu2)
    e2e_t = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t = time.perf_counter()
        plan.execute_host(hu1, hu2)
        e2e_t.append(time.perf_counter() - t)
    e2e_s = max_over_ranks(statistics.mean(e2e_t), dev, world)
    serial_value = whole_job_rate(n_src, world, e2e_s)
    # a stream of transforms: E2E_PLANS plans on as many streams take turns,
    # each step queued with asfd_execute_host_async, so that one step's
    # copies of u2 to the host overlap the next steps' uploads and kernels
    pipe_s = max_over_ranks(e2e_pipelined(g, d1, args, plan, hu1, hu2), dev, world)
    pipe_value = whole_job_rate(n_src, world, pipe_s)
    e2e = {"value": pipe_value, "unit": UNIT,
           "h2d_bytes_per_step": hu1.numel() * 8,
           "d2h_bytes_per_step": hu2.numel() * 8,
           "path": f"page-locked host buffers, steps queued with asfd_execute_host_async "
                   f"on {E2E_PLANS} plans and streams in turn, one synchronisation after the "
                   "last: u1 uploaded by a copy, u2 copied to the host in four column "
                   "blocks, each while the column pass transforms the next (each plan's "
                   "work buffers, 268 MB, exceed L2 between its steps)",
           "serial_value": serial_value,
           "serial_path": "one asfd_execute_host call at a time (synchronous, u1 read by the "
                          "spread in place over the host link), L2 flushed before each"}
    # context: pageable host buffers, staged through device copies by the library
    pu1 = torch.as_tensor(u1).clone()
    pu2 = torch.empty(plan.shape2, dtype=torch.complex64)
    plan.execute_host(pu1, pu2)
    st_t = []
    for _ in range(min(args.steps, 5)):
        flush.zero_()
        torch.cuda.synchronize()
        t = time.perf_counter()
        plan.execute_host(pu1, pu2)
        st_t.append(time.perf_counter() - t)
    e2e["pageable_staged_value"] = whole_job_rate(n_src, world, statistics.mean(st_t))

    line = None
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic", "config": workload_config(args.workload, args.width),
                "roofline": roofline, "step_roofline": step_roofline, "e2e": e2e, "clocks": clk,
                "spread_kind": info["spread_kind"],
                "gpu_launches": 3 * args.steps, "plan_ms": plan_ms,
                "update_d1_ms": update_d1_ms,
                "wall_s_timed_region": wall,
                "plan": {k: info[k] for k in ("nfx", "nfy", "band_x0", "band_x1", "band_y0",
                                              "band_y1", "spread_tiles", "tile_pairs")}}
        if world == 1 and not args.no_cpu_baseline:
            sps, cores, npts, el, pts, ref = oracle_sample(g, u1, d1, args.cpu_seconds)
            got = u2_d.cpu().numpy()[pts[1], pts[0]].astype(np.complex128)
            line["rel_l2_vs_oracle"] = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
            line["rel_l2_points"] = npts
            line["cpu_baseline"] = {
                "value": sps, "unit": UNIT, "cores": cores, "kind": "oracle",
                "sample": f"{npts} seeded destination points of the {g['m2x']}x{g['m2y']} grid "
                          f"({el:.1f} s), each a direct FP64 sum over all {n_src} source samples; "
                          "scaled to source samples/s of the full transform"}
        if world == 1 and not args.no_extras:
            pts_x, ref_x = (pts, ref) if "cpu_baseline" in line else (None, None)
            line.update(extra_measurements(args, g, u1, d1, pts_x, ref_x, flush, stream))
            if "measured_peaks" in line and info["spread_kind"] == 3:
                line["resource_frac"] = resource_fractions(
                    info, g, args.width, mean_stage, line["measured_peaks"])
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


# transforms in flight in the pipelined end-to-end measurement: at 2048^2
# two leave the host link idle between steps, three keep it busy (four
# measure the same)
E2E_PLANS = 3


def e2e_pipelined(g, d1, args, plan, hu1, hu2):
    """Seconds per step of `args.steps` host-buffer transforms queued back to
    back, step k on plan k mod E2E_PLANS and its own stream (after
    `args.warmup` untimed ones)."""
    import torch
    from paper_1203_3583_gb300.fresnel import FresnelPlan
    plans = [plan] + [FresnelPlan(g, d1, kernel_width=args.width) for _ in range(E2E_PLANS - 1)]
    streams = [torch.cuda.Stream() for _ in plans]
    hin = [hu1] + [hu1.clone().pin_memory() for _ in plans[1:]]
    hout = [hu2] + [torch.empty_like(hu2).pin_memory() for _ in plans[1:]]

    def run(n):
        for k in range(n):
            j = k % len(plans)
            plans[j].execute_host(hin[j], hout[j], stream=streams[j], sync=False)
        torch.cuda.synchronize()

    try:
        run(max(len(plans), args.warmup))
        t = time.perf_counter()
        run(args.steps)
        return (time.perf_counter() - t) / args.steps
    finally:
        for p in plans[1:]:
            p.close()


def time_device_ms(fn, steps, warmup, flush, stream):
    """Mean CUDA-event time (ms) of fn() on `stream`, L2 flushed before each call
    outside the timed interval."""
    import torch
    for _ in range(warmup):
        flush.zero_()
        fn()
    torch.cuda.synchronize()
    evs = []
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize()
    return statistics.mean(a.elapsed_time(b) for a, b in evs)


def width4_floor():
    """The width-4 floor (2D relative L2) stored by tests/golden/make_learned_floor.py."""
    path = os.path.join(ROOT, "tests", "golden", "learned_floor_sigma2.txt")
    try:
        for line in open(path):
            f = line.split()
            if f and not line.startswith("#") and f[0] == "4":
                return float(f[2])
    except OSError:
        pass
    return None


def probe_peaks(stream, repeats=5):
    """Measured peaks of the on-chip resources (include/asfd_peaks.h probes),
    best of `repeats` CUDA-event timed launches after one warm-up each."""
    import torch

    from paper_1203_3583_gb300 import capi
    sink = torch.zeros(1 << 16, dtype=torch.float32, device="cuda")
    red = torch.zeros(32 << 20, dtype=torch.uint8, device="cuda")  # 32 MiB, L2-resident
    cases = {"smem_load": (sink, 4096, "GB/s"), "smem_store": (sink, 4096, "GB/s"),
             "l2_red_v2f32": (red, 256, "GB/s"), "ffma2": (sink, 16384, "TFLOP/s"),
             "mufu_ex2": (sink, 8192, "Gop/s")}
    out = {}
    for kind, (buf, iters, unit) in cases.items():
        capi.asfd_probe_launch(kind, iters, buf, stream)
        best = None
        for _ in range(repeats):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            work = capi.asfd_probe_launch(kind, iters, buf, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            rate = work / (e0.elapsed_time(e1) * 1e-3)
            best = rate if best is None else max(best, rate)
        scale = 1e12 if unit == "TFLOP/s" else 1e9
        out[kind] = {"value": best / scale, "unit": unit}
    return out


def resource_fractions(info, g, width, stage_ms, peaks):
    """Each stage of the step against the on-chip resources that bound it
    (measured peaks), beside its HBM fraction: the spread's packed FP32 FMA
    (4 W^2 flops per sample), MUFU (4 W evaluations per sample: an exp2 and a
    reciprocal square root per tap and axis) and L2 float2 reductions (window
    rows flushed: per source column alpha_y n1y + W rows per run, W cells
    each); the FFT passes' shared-memory exchanges ((passes - 1) stores and
    loads of every line)."""
    import math
    n = g["n1x"] * g["n1y"]
    nfx, nfy = info["nfx"], info["nfy"]
    alpha_y = g["p1y"] * g["p2y"] * nfy / (g["lam"] * g["z0"])
    runs = max(1, math.ceil(g["n1y"] / max(1, info["run_rows"] or g["n1y"])))
    flushed = g["n1x"] * (alpha_y * g["n1y"] + runs * width) * width * 8.0
    t_sp, t_r, t_c = (ms * 1e-3 for ms in stage_ms)

    def smem_bytes(L, lines):
        passes = (int(math.log2(L)) + 3) // 4
        return (passes - 1) * 8.0 * L * lines  # each of stores and loads
    rows = (info["band_y1"] - info["band_y0"])
    sm_r, sm_c = smem_bytes(nfx, rows), smem_bytes(nfy, g["m2x"])
    ld, st = peaks["smem_load"]["value"] * 1e9, peaks["smem_store"]["value"] * 1e9
    return {
        "spread": {"ffma2": 4.0 * width * width * n / t_sp / (peaks["ffma2"]["value"] * 1e12),
                   "mufu": 4.0 * width * n / t_sp / (peaks["mufu_ex2"]["value"] * 1e9),
                   "l2_red": flushed / t_sp / (peaks["l2_red_v2f32"]["value"] * 1e9)},
        "fft_rows": {"smem": (sm_r / st + sm_r / ld) / t_r},
        "fft_cols": {"smem": (sm_c / st + sm_c / ld) / t_c},
    }


def extra_measurements(args, g, u1, d1, pts, ref_pts, flush, stream):
    """Single-GPU context lines: the ES width sweep and the learned kernel at the
    same workload (accuracy against the ES width-12 field and the oracle
    points), the adjoint on the 4096^2 workload and the 24-surface batch."""
    import numpy as np
    import torch

    from paper_1203_3583_gb300 import learned as L, workloads as W
    from paper_1203_3583_gb300.fresnel import FresnelBatch, FresnelPlan

    steps = max(5, min(args.steps, 20))
    n_src = g["n1x"] * g["n1y"]
    u1_d = torch.as_tensor(u1, device="cuda")
    ref12 = L.reference_fields([(g, u1, d1)])[0]

    def accuracy(out):
        full = float(torch.linalg.vector_norm(out - ref12) / torch.linalg.vector_norm(ref12))
        if ref_pts is None:  # no oracle points in this run
            return full, None
        got = out.cpu().numpy()[pts[1], pts[0]].astype(np.complex128)
        return full, float(np.linalg.norm(got - ref_pts) / np.linalg.norm(ref_pts))

    res = {}
    widths = {}
    peak, _ = measured_peaks()
    if "peaks" in args.extras:
        res["measured_peaks"] = probe_peaks(stream)

    def step_frac(ms):
        # the step against the spread+FFT memory model (STEP_BYTES_PER_SAMPLE)
        return STEP_BYTES_PER_SAMPLE * n_src / (ms * 1e-3) / 1e9 / peak
    if "deterministic" in args.extras:
        # the atomic-free (bit-reproducible) spreading path on the same workload
        with FresnelPlan(g, d1, kernel_width=args.width, deterministic=True) as p:
            out = torch.empty(p.shape2, dtype=torch.complex64, device="cuda")
            ms = time_device_ms(lambda: p.execute(u1_d, out=out), steps, 3, flush, stream)
            sp = time_device_ms(lambda: p.execute_stage(0, u1=u1_d), steps, 3, flush, stream)
            full, orc = accuracy(out)
            kind = p.info()["spread_kind"]
        res["deterministic"] = {"spread_kernel": SPREAD_KERNEL[kind], "samples_per_s": n_src / (ms * 1e-3),
                                "ms": ms, "spread_ms": sp, "rel_l2_vs_oracle": orc}

    if "es_widths" in args.extras:
        for w in (4, 5, 6, 7, 8):
            with FresnelPlan(g, d1, kernel_width=w) as p:
                out = torch.empty(p.shape2, dtype=torch.complex64, device="cuda")
                ms = time_device_ms(lambda: p.execute(u1_d, out=out), steps, 3, flush, stream)
                full, orc = accuracy(out)
            widths[str(w)] = {"samples_per_s": n_src / (ms * 1e-3), "ms": ms,
                              "rel_l2_vs_es12": full, "rel_l2_vs_oracle": orc,
                              "unpruned_step_frac": step_frac(ms)}
        res["es_widths"] = widths

    if "learned" in args.extras:
        t0 = time.perf_counter()
        pairs = L.train_set()
        model, losses = L.train_model(pairs)
        torch.cuda.synchronize()
        train_s = time.perf_counter() - t0
        with FresnelPlan(g, d1, kind="learned") as p:
            model.apply_to(p)
            out = torch.empty(p.shape2, dtype=torch.complex64, device="cuda")
            ms = time_device_ms(lambda: p.execute(u1_d, out=out), steps, 3, flush, stream)
            full, orc = accuracy(out)
        match = [w for w in sorted(widths, key=int) if widths[w]["rel_l2_vs_es12"] <= full]
        floor = width4_floor()
        res["learned"] = {
            "kernel_width": 4, "samples_per_s": n_src / (ms * 1e-3), "ms": ms,
            "unpruned_step_frac": step_frac(ms),
            "rel_l2_vs_es12": full, "rel_l2_vs_oracle": orc,
            "target_rel_l2": 1e-4, "meets_target": (orc if orc is not None else full) <= 1e-4,
            "width4_floor_rel_l2": floor,
            "above_floor": (orc if orc is not None else full) / floor if floor else None,
            "floor_source": "tests/golden/learned_floor_sigma2.txt (no width-4 gridding reaches "
                            "below it at sigma 2 on random-phase samples)",
            "gain_vs_es4_error": widths["4"]["rel_l2_vs_es12"] / full if "4" in widths else None,
            "es_width_at_same_accuracy": int(match[0]) if match else None,
            "speedup_vs_es_at_same_accuracy": (widths[match[0]]["ms"] / ms) if match else None,
            "training": {"steps": model.meta["steps"], "seconds_incl_references": train_s,
                         "pairs": len(pairs),
                         "geometry": "smooth_random2048 recipe at 2048^2, surface seeds 100-101",
                         "final_train_rel_l2": float(np.sqrt(losses[-1]))}}

    if "direct_sum" in args.extras:
        # direct sums of Eq. 7, Eq. 5 and Eq. 2 on sampled points: what the
        # approximations of Eqs. 4 and 6 cost at this size, and the GPU pair rate
        from paper_1203_3583_gb300.fresnel import direct_sum
        pts_d = W.sample_points(g, 512, seed=11)
        vals, dms = {}, {}
        for form in (7, 5, 2):
            direct_sum(g, d1, u1_d, form, pts_d)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            v = direct_sum(g, d1, u1_d, form, pts_d)
            e1.record(stream)
            torch.cuda.synchronize()
            dms[form] = e0.elapsed_time(e1)
            vals[form] = v.cpu().numpy().astype(np.complex128)
        with FresnelPlan(g, d1, kernel_width=args.width) as p:
            nu = p.execute(u1_d).cpu().numpy()[pts_d[1], pts_d[0]].astype(np.complex128)

        def rl(a, b):
            return float(np.linalg.norm(a - b) / np.linalg.norm(b))
        npairs = n_src * len(pts_d[0])
        res["direct_sum"] = {
            "points": len(pts_d[0]),
            "ms": {f"eq{f}": dms[f] for f in dms},
            "pairs_per_s": {f"eq{f}": npairs / (dms[f] * 1e-3) for f in dms},
            "rel_l2": {"nufft_vs_eq7": rl(nu, vals[7]), "eq7_vs_eq5 (Eq. 6)": rl(vals[7], vals[5]),
                       "eq5_vs_eq2 (Eq. 4, r^2 ~ z0^2)": rl(vals[5], vals[2]),
                       "nufft_vs_eq2": rl(nu, vals[2])}}

    if "line" in args.extras:
        # the paper's 1D experiments (Sec. 3; layout readings in workloads.line_*):
        # the line NUFFT against the 1D oracle, and the paper's comparison of the
        # method (Eq. 7) with the Huygens sum (Eq. 2) as the largest difference of
        # the intensities normalised to the Eq. 2 peak
        from oracle import line as oline
        from paper_1203_3583_gb300.fresnel import LinePlan
        lines = {}
        for shape, (lx, ld, lw) in (("facets", W.line_facets()), ("quadratic", W.line_quadratic())):
            lg = W.line_geometry()
            lu = np.ones(lx.size, np.complex128)
            with LinePlan(lg, lx, ld, lw) as lp:
                lu_d = torch.as_tensor(lu.astype(np.complex64), device="cuda")
                out_l = torch.empty(lg["m2"], dtype=torch.complex64, device="cuda")
                lms = time_device_ms(lambda: lp.execute(lu_d, out=out_l), steps, 3, flush, stream)
                got = out_l.cpu().numpy().astype(np.complex128)
            r7 = oline.line(lg, lx, ld, lw, lu, 7)
            r2 = oline.line(lg, lx, ld, lw, lu, 2)
            i2 = np.abs(r2) ** 2
            lines[shape] = {"samples": int(lx.size), "ms": lms,
                            "rel_l2_vs_oracle_eq7": float(np.linalg.norm(got - r7) / np.linalg.norm(r7)),
                            "max_intensity_diff_vs_eq2": float(np.max(np.abs(np.abs(got) ** 2 - i2))
                                                               / np.max(i2))}
        res["line"] = {"geometry": "1024 samples at 10 um along the surface, 1024 x 10 um "
                                   "destination, 633 nm, z0 1 m", **lines}

    if "multi" in args.extras:
        # several surfaces summed at one destination: one shared grid and FFT
        # against the surfaces' own transforms one after another
        from paper_1203_3583_gb300.fresnel import multi_execute
        mitems = W.make_multi()
        mplans = [FresnelPlan(gm, dm) for gm, _, dm in mitems]
        try:
            mu = [torch.as_tensor(um, device="cuda") for _, um, _ in mitems]
            mout = torch.empty(mplans[0].shape2, dtype=torch.complex64, device="cuda")
            souts = [torch.empty(p.shape2, dtype=torch.complex64, device="cuda") for p in mplans]
            ms_multi = time_device_ms(lambda: multi_execute(mplans, mu, out=mout), steps, 3, flush,
                                      stream)
            ms_each = time_device_ms(lambda: [p.execute(u, out=o) for p, u, o in zip(mplans, mu, souts)],
                                     steps, 3, flush, stream)
        finally:
            for p in mplans:
                p.close()
        nsm = sum(gm["n1x"] * gm["n1y"] for gm, _, _ in mitems)
        res["multi"] = {"workload": "3 surfaces (384^2, 256^2, 512^2 at 8 um, offset) -> 1024^2",
                        "source_samples": nsm, "ms_shared_grid": ms_multi,
                        "ms_separate_transforms": ms_each,
                        "samples_per_s": nsm / (ms_multi * 1e-3)}

    if "adjoint" in args.extras:
        ga, ua, da = W.make("tilt_bump4096")
        with FresnelPlan(ga, da) as p:
            ua_d = torch.as_tensor(ua, device="cuda")
            u2a = p.execute(ua_d)
            inten = (u2a.abs() ** 2)
            target = torch.rand(inten.shape, generator=torch.Generator().manual_seed(5)).to("cuda") \
                * 2 * inten.mean()
            gu2 = (4 * (inten - target) * u2a).to(torch.complex64)
            gu1 = torch.empty_like(ua_d)
            gd1 = torch.empty(p.shape1, dtype=torch.float32, device="cuda")
            ms = time_device_ms(lambda: p.adjoint(ua_d, gu2, gu1, gd1), steps, 3, flush, stream)
        res["adjoint"] = {"workload": "tilt_bump4096 (4096^2 at 3.74 um, 532 nm, z0 0.15 m)",
                          "samples_per_s": ga["n1x"] * ga["n1y"] / (ms * 1e-3), "ms": ms,
                          "outputs": "dL/du1 (complex) and dL/dd1"}

    if "fft_reference" in args.extras:
        # cuFFT (through torch.fft) as a timing reference for the two FFT stages:
        # the full 2D transform of the fine grid, and the same pruning as the
        # hand-written passes (band rows only, then the kept columns only); the
        # hand-written column pass also applies the deconvolution, the crop and
        # the destination chirp, which the cuFFT lines leave out
        with FresnelPlan(g, d1, kernel_width=args.width) as p:
            info = p.info()
            out = torch.empty(p.shape2, dtype=torch.complex64, device="cuda")
            p.execute_stage(0, u1=u1_d)
            ours = time_device_ms(lambda: (p.execute_stage(1), p.execute_stage(2, out=out)),
                                  steps, 3, flush, stream)
        nfx, nfy, m2x = info["nfx"], info["nfy"], g["m2x"]
        y0, y1 = info["band_y0"], info["band_y1"]
        x0, x1 = info["band_x0"], info["band_x1"]
        gen = torch.Generator(device="cuda").manual_seed(3)
        grid = torch.zeros((nfy, nfx), dtype=torch.complex64, device="cuda")
        grid[y0:y1, x0:x1] = torch.randn((y1 - y0, x1 - x0), dtype=torch.complex64, device="cuda",
                                         generator=gen)
        full = time_device_ms(lambda: torch.fft.fft2(grid), steps, 3, flush, stream)
        kept = torch.cat([torch.arange(nfx - m2x // 2, nfx), torch.arange(0, m2x // 2)]).to("cuda")
        cols = torch.zeros((nfy, m2x), dtype=torch.complex64, device="cuda")

        def pruned():
            cols[y0:y1] = torch.fft.fft(grid[y0:y1], dim=1).index_select(1, kept)
            return torch.fft.fft(cols, dim=0)
        pr = time_device_ms(pruned, steps, 3, flush, stream)
        res["fft_reference"] = {
            "library": "cuFFT through torch.fft, timing reference only",
            "fine_grid": [nfy, nfx], "band_rows": y1 - y0, "kept_columns": m2x,
            "ms_rows_cols_ours": ours, "ms_cufft_fft2_full_grid": full,
            "ms_cufft_band_rows_then_kept_columns": pr}

    if "batch" in args.extras:
        items = W.make_batch()
        with FresnelBatch([(gb, db) for gb, _, db in items]) as b:
            u1s = [torch.as_tensor(ub, device="cuda") for _, ub, _ in items]
            outs = [torch.empty((gb["m2y"], gb["m2x"]), dtype=torch.complex64, device="cuda")
                    for gb, _, _ in items]
            ms = time_device_ms(lambda: b.execute(u1s, out=outs), steps, 3, flush, stream)
            info = b.info()
            b.set_schedule("persistent")
            pms = time_device_ms(lambda: b.execute(u1s, out=outs), steps, 3, flush, stream)
            pinfo = b.info()
        res["batch"] = {"workload": "rgb_batch24 (24 surfaces, 256^2..2048^2, 450/532/633 nm)",
                        "samples_per_s": info["source_samples"] / (ms * 1e-3), "ms": ms,
                        "schedule": f"streams ({info['streams']} streams of the batch, CUDA graph)",
                        "source_samples": info["source_samples"],
                        "cuda_graph": bool(info["graph"]),
                        "persistent": {"ms": pms,
                                       "samples_per_s": info["source_samples"] / (pms * 1e-3),
                                       "blocks": pinfo["blocks"],
                                       "cuda_graph": bool(pinfo["graph"])}}

    return res


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
