"""Benchmark of the SV-MPR hot path on GB300 (one JSON line on rank 0).

A step is one pass of the whole method over one synthetic field: create
(Sec. 2.1 transform, Eq. 2 per block), per-block temperature calibration,
R local-equilibrium realizations with per-block stop, and the back-transformed
mean. Default workload: a 1024 x 1024 non-stationary Gaussian random field
(correlation length 4 -> 32 cells left to right, N(0, 0.1^2) nugget), 50 %
gaps at random, 16 x 16 temperature blocks, 100 realizations, FP32.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Metric: gap-site updates/s (Metropolis + over-relaxation site updates of the
calibration and of the realizations, per second of step time); the line also
carries gap-filled Mpix/s. Under torchrun every rank fills its own field
(independent slices, no collective on the data path): weak scaling; with
--shard realizations the ranks share one field's realizations instead and
add their per-site sums with one all-reduce (strong scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
STORAGE = {"f32": 0, "bf16": 1, "f16": 2}
sys.path.insert(0, ROOT)

METRIC = "gap-site updates/s"
L2_FLUSH_BYTES = 256 << 20   # > 129 MB L2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="field1024")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--storage", default="f32", choices=["f32", "bf16", "f16"],
                    help="element type of the realizations' angles (arithmetic stays FP32)")
    ap.add_argument("--cal-mode", type=int, default=0, choices=[0, 1, 2, 3],
                    help="calibration launch form (3: every kernel from the host, for profilers)")
    ap.add_argument("--cal-points", type=int, default=2, choices=[1, 2],
                    help="calibration temperatures per block and iteration (1 bisection, "
                         "2 trisection, the default: the two temperatures run on the two "
                         "lanes of a realization pair); --cal-iters sets the iterations")
    ap.add_argument("--cal-iters", type=int, default=None,
                    help="calibration iterations (default 24 for bisection, 16 for trisection)")
    ap.add_argument("--plain-sample", type=int, default=0,
                    help="batch workloads: also time the plain form (one FP32 context per "
                         "field) on this many fields")
    ap.add_argument("--calibration", default="bisection", choices=["bisection", "newton"],
                    help="per-block temperature fit: bisection (the plain form) or safeguarded "
                         "Newton steps from the fluctuation identity")
    ap.add_argument("--pipeline", type=int, default=3,
                    help="also time the fields with this many in flight (one CUDA stream and "
                         "host thread each; 0 or 1: skip), reported as 'pipelined'")
    ap.add_argument("--shard", default="fields", choices=["fields", "realizations"],
                    help="fields: every rank its own field (weak scaling, no collective); "
                         "realizations: ranks share one field's realizations (strong scaling, "
                         "one all-reduce of the per-site sums)")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def cal_iters(args) -> int:
    """Calibration iterations: 24 bisection steps, or 16 trisection steps (a
    narrower final bracket: 2 / 3^16 < 2 / 2^24)."""
    if args.cal_iters is not None:
        return args.cal_iters
    return 16 if args.cal_points == 2 else 24


def bytes_per_gap_update(s_bytes: float, p: float) -> float:
    """Algorithmic HBM bytes per gap-site update of one field: per sweep the
    two half-steps read the other colour once (s*HW), read and write the
    gap sites (2*s*p*HW) and read the gap mask (HW/8 bytes); divided by the
    p*HW updates of the sweep."""
    return (s_bytes * (1.0 + 2.0 * p) + 0.125) / p


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4)
                          if r[5 + k].lower() in ("active", "1")})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


# ------------------------------------------------------------ reference --
def run_reference(args, world, rank):
    """The oracle (FP64 C, all host cores) on a bounded sample of the workload."""
    if rank != 0:
        return
    import oracle
    from paper_2212_01317_gb300 import synth
    oracle.build()
    if args.workload in synth.BATCH_WORKLOADS:
        # A batch's fields are independent problems: the oracle's rate is taken
        # on its first field.
        bw = synth.batch_workload(args.workload)
        wl = synth.Workload(bw.name + "_field0", bw.truths[0], bw.masks[0], bw.block,
                            bw.realizations)
    else:
        wl = synth.workload(args.workload)
    lb = wl.block
    cores = len(os.sched_getaffinity(0))
    if wl.truth.ndim == 3:                         # the 3-D extension
        D, H, W = wl.shape
        o = oracle.Oracle3(D, H, W, lb, seed=2024)
        o.m.threads = cores
        phi, _, _, _ = oracle.Oracle.transform(wl.truth.reshape(D * H, W),
                                               wl.mask.reshape(D * H, W))
        phi = phi.reshape(D, H, W)
    else:
        H, W = wl.shape
        o = oracle.Oracle(H, W, lb, seed=2024, threads=cores)
        phi, _, _, _ = o.transform(wl.truth, wl.mask)
    st = o.block_stats(phi, wl.mask)
    phi0 = o.init_block_mean(phi, wl.mask, st)
    T = np.full(o.nblk, 0.1)

    def step(r):
        t0 = time.perf_counter()
        stop = o.simulate_one(phi0, wl.mask, T, st, 200, r)[1]
        dt = time.perf_counter() - t0
        return int(np.sum(stop.astype(np.int64) * st.n_gap)), dt

    for r in range(args.warmup):
        step(r)
    ups, secs = 0, 0.0
    for r in range(args.steps):
        u, dt = step(args.warmup + r)
        ups += u
        secs += dt
    val = ups / secs
    sample = (f"oracle simulate of one realization per step on {wl.name} at uniform T=0.1 "
              f"(calibration not run), {cores} threads")
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "updates/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl.name, "shape": list(wl.shape), "block": lb,
                       "realizations": wl.realizations},
            "cpu_baseline": {"value": val, "unit": "updates/s", "cores": cores,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": "updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------- our arm --
def cpu_baseline(wl, T_gpu, seconds):
    import oracle
    oracle.build()
    H, W = wl.shape
    cores = len(os.sched_getaffinity(0))
    o = oracle.Oracle(H, W, wl.block, seed=2024, threads=cores)
    phi, *_ = o.transform(wl.truth, wl.mask)
    st = o.block_stats(phi, wl.mask)
    phi0 = o.init_block_mean(phi, wl.mask, st)
    T = np.asarray(T_gpu, dtype=np.float64)
    ups, secs, r = 0, 0.0, 0
    while secs < seconds or r == 0:
        t0 = time.perf_counter()
        _, stop, _, _ = o.simulate_one(phi0, wl.mask, T, st, 200, r)
        secs += time.perf_counter() - t0
        ups += int(np.sum(stop.astype(np.int64) * st.n_gap))
        r += 1
    return {"value": ups / secs, "unit": "updates/s", "cores": cores, "kind": "oracle",
            "sample": f"{r} realization(s) of {wl.name} at the GPU-calibrated block T, "
                      f"simulate only, {secs:.1f} s on {cores} threads"}


def run_ours(args, world, rank, local):
    import torch
    from paper_2212_01317_gb300 import mpr, replicas, synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    mpr.load()
    wl = synth.workload(args.workload, seed=0)
    H, W = wl.shape
    n = H * W
    P = wl.n_gap
    p = P / n
    R = wl.realizations
    stream = torch.cuda.current_stream(dev)
    vals_h = np.where(wl.mask != 0, np.nan, wl.truth).astype(np.float32)
    values_d = torch.from_numpy(vals_h).to(dev)
    mask_d = torch.from_numpy(wl.mask).to(dev)
    out_d = torch.empty((H, W), dtype=torch.float32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    shard = args.shard if world > 1 else "fields"
    seed, slice_id = replicas.rank_seed(2024, rank, shard)
    acc_d = torch.empty((H, W), dtype=torch.float64, device=dev)
    T_d = None

    def options(profile):
        return mpr.mpr_default_options(seed=seed, slice_id=slice_id, profile=profile,
                                       storage=STORAGE[args.storage], cal_mode=args.cal_mode,
                                       cal_method=1 if args.calibration == "newton" else 0,
                                       cal_points=args.cal_points, n_bisect=cal_iters(args),
                                       cuda_stream=stream.cuda_stream)

    def step(values, mask, out, profile=1):
        nonlocal T_d
        ctx = mpr.mpr_create(H, W, wl.block, mask, values, options(profile))
        try:
            if shard == "fields":
                mpr.mpr_calibrate(ctx, None)
                mpr.mpr_simulate(ctx, R)
            else:
                if T_d is None:
                    T_d = torch.empty(mpr.mpr_get_info(ctx).nblk, dtype=torch.float32, device=dev)
                replicas.fill_shared_field(ctx, R, world, rank, acc_d, T_d)
            mpr.mpr_predict(ctx, out)
            info = mpr.mpr_get_info(ctx)
            prof = mpr.mpr_get_profile(ctx)
        finally:
            mpr.mpr_destroy(ctx)
        return info, prof

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    for _ in range(args.warmup):
        step(values_d, mask_d, out_d)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    step_ms, updates, cal_updates, launches = [], 0, 0, 0
    sim_ms = cal_ms = tail_ms = 0.0
    sim_launch = cal_launch = sim_updates = tail_updates = tail_launch = 0
    for k in range(args.steps):
        flush.zero_()                              # L2 flush between timed steps
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        info, prof = step(values_d, mask_d, out_d)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        updates += info.gap_updates + info.cal_gap_updates
        sim_updates += info.gap_updates
        cal_updates += info.cal_gap_updates
        launches += prof.kernel_launches
        sim_ms += prof.sim_halfstep_ms
        cal_ms += prof.cal_halfstep_ms
        sim_launch += prof.sim_halfstep_launches
        cal_launch += prof.cal_halfstep_launches
        tail_ms += prof.sim_tail_ms
        tail_updates += prof.sim_tail_updates
        tail_launch += prof.sim_tail_launches
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()
    total_ms = float(np.sum(step_ms))
    total_ms = replicas.max_over_ranks(total_ms, dev)
    updates_all = replicas.sum_over_ranks(updates, dev)
    value = updates_all / (total_ms / 1e3)
    fields = world if shard == "fields" else 1          # distinct fields filled per step
    mpix = fields * P * args.steps / (total_ms / 1e3) / 1e6

    # End to end through the C-ABI with pinned host buffers: the H2D copy of
    # the step's inputs and the D2H copy of its predictions are timed.
    e2e = None
    if not args.no_e2e:
        vals_pin = torch.from_numpy(vals_h).pin_memory()
        mask_pin = torch.from_numpy(wl.mask).pin_memory()
        out_pin = torch.empty((H, W), dtype=torch.float32).pin_memory()
        step(vals_pin, mask_pin, out_pin, profile=0)
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        ups = 0
        for k in range(args.steps):
            info, _ = step(vals_pin, mask_pin, out_pin, profile=0)
            ups += info.gap_updates + info.cal_gap_updates
        torch.cuda.synchronize()
        dt = replicas.max_over_ranks(time.perf_counter() - t0, dev)
        ups = replicas.sum_over_ranks(ups, dev)
        e2e = {"value": ups / dt, "unit": "updates/s",
               "h2d_bytes_per_step": int(vals_h.nbytes + wl.mask.nbytes),
               "d2h_bytes_per_step": int(out_pin.numel() * 4),
               "gap_filled_mpix_s": fields * P * args.steps / dt / 1e6}

    # Fields in flight: the same per-field work (calibrate, R realizations,
    # predict, each field its own context) with `pipeline` fields at a time,
    # one CUDA stream and host thread each, so that one field's latency-bound
    # phases (calibration, the stop tail) overlap another's. Device time over
    # all K fields, between events that every stream waits on / joins.
    pipelined = None
    if args.pipeline > 1 and shard == "fields":
        import threading
        npipe = args.pipeline
        pstreams = [torch.cuda.Stream(dev) for _ in range(npipe)]
        pouts = [torch.empty((H, W), dtype=torch.float32, device=dev) for _ in range(npipe)]
        pups = [0] * npipe

        def pworker(w, ks):
            for _ in ks:
                o = options(0)
                o.cuda_stream = pstreams[w].cuda_stream
                ctx = mpr.mpr_create(H, W, wl.block, mask_d, values_d, o)
                try:
                    mpr.mpr_calibrate(ctx, None)
                    mpr.mpr_simulate(ctx, R)
                    mpr.mpr_predict(ctx, pouts[w])
                    inf = mpr.mpr_get_info(ctx)
                    pups[w] += inf.gap_updates + inf.cal_gap_updates
                finally:
                    mpr.mpr_destroy(ctx)

        def prun(k_total):
            for w in range(npipe):
                pups[w] = 0
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for ps in pstreams:
                ps.wait_event(e0)
            th = [threading.Thread(target=pworker, args=(w, range(w, k_total, npipe)))
                  for w in range(npipe)]
            for t in th:
                t.start()
            for t in th:
                t.join()
            for ps in pstreams:
                ev = torch.cuda.Event()
                ev.record(ps)
                stream.wait_event(ev)
            e1.record(stream)
            e1.synchronize()
            return e0.elapsed_time(e1), sum(pups)

        prun(npipe)                                   # warm-up: one field per stream
        barrier()
        p_ms, p_ups = prun(args.steps)
        p_ms = replicas.max_over_ranks(p_ms, dev)
        p_ups = replicas.sum_over_ranks(p_ups, dev)
        pipelined = {"fields_in_flight": npipe, "value": p_ups / (p_ms / 1e3),
                     "unit": "updates/s", "ms_per_field": p_ms / args.steps,
                     "gap_filled_mpix_s": world * P * args.steps / (p_ms / 1e3) / 1e6,
                     "fields": args.steps,
                     "form": "each field its own context, calibrate + simulate + predict; "
                             f"{npipe} fields at a time on {npipe} CUDA streams"}

    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return

    peak, peak_kind = measured_peaks()
    bpu = bytes_per_gap_update(4.0 if args.storage == "f32" else 2.0, p)
    # The realizations' per-launch half-steps (k_sweep) ran every update but
    # those of the stop-tail launch, which is timed and counted apart.
    sweep_updates = sim_updates - tail_updates
    sim_gbs = sweep_updates * bpu / (sim_ms / 1e3) / 1e9 if sim_ms > 0 else None
    cal_gbs = cal_updates * bpu / (cal_ms / 1e3) / 1e9 if cal_ms > 0 else None
    # Dominant kernel by summed device time.
    dom = "sim" if sim_ms >= cal_ms else "cal"
    achieved = sim_gbs if dom == "sim" else cal_gbs
    # DRAM bytes per launch of the dominant kernel: the ncu-measured bytes per
    # gap-site update (profiles/traffic.json, taken on this workload) times the
    # average updates per launch of this run.
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tpath) and dom == "sim" and args.storage == "f32" and sim_launch:
        with open(tpath) as f:
            rec = json.load(f).get(f"sim_{wl.name}")
        if rec:
            traffic = rec["bytes_per_update"] * sweep_updates / sim_launch
    roofline = {
        "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
        "frac": (achieved / peak) if achieved else None, "traffic": traffic,
        "kernel": ("k_sweep_half / k_sweep (realizations' per-launch half-steps)" if dom == "sim"
                   else ("k_sweep_flat (calibration)" if args.cal_mode == 3
                         else "calibration graph (k_sweep_flat + bookkeeping)")),
        "peak_kind": peak_kind,
        "bytes_per_gap_update": bpu,
        "avg_launch_us": 1e3 * (sim_ms / sim_launch if dom == "sim" else cal_ms / max(cal_launch, 1)),
        "sim_halfstep": {"ms": sim_ms / args.steps, "launches": sim_launch // args.steps,
                         "gbs": sim_gbs,
                         "updates_per_s": sweep_updates / (sim_ms / 1e3) if sim_ms else None},
        "stop_tail": {"kernel": "k_pair_tail (one CTA per realization pair; its time includes "
                                "the stop tests of its sweeps)",
                      "ms": tail_ms / args.steps, "launches": tail_launch // args.steps,
                      "updates": tail_updates // args.steps,
                      "updates_per_s": tail_updates / (tail_ms / 1e3) if tail_ms else None},
        "cal_halfstep": {"ms": cal_ms / args.steps, "launches": cal_launch // args.steps,
                         "gbs": cal_gbs,
                         "updates_per_s": cal_updates / (cal_ms / 1e3) if cal_ms else None},
    }
    line = {
        "metric": METRIC, "value": value, "unit": "updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak" if shard == "fields" else "strong",
        "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": wl.name, "H": H, "W": W, "block": wl.block, "gap_fraction": p,
                   "realizations": R, "storage": args.storage, "cal_mode": args.cal_mode,
                   "calibration": args.calibration if args.calibration == "newton" else
                   ("bisection" if args.cal_points == 1 else "trisection") + f" x{cal_iters(args)}",
                   "l2": "flushed between timed steps",
                   "parallelism": (f"replicas{world}" if shard == "fields"
                                   else f"realizations{world}")},
        "gap_filled_mpix_s": mpix,
        "updates_per_step": {"calibration": cal_updates // args.steps,
                             "realizations": sim_updates // args.steps},
        "gpu_launches": int(launches),
        "roofline": roofline,
        "clocks": clk,
        "e2e": e2e,
        "pipelined": pipelined,
    }
    if world == 1 and not args.no_cpu:
        ctx = mpr.mpr_create(H, W, wl.block, mask_d, values_d, options(0))
        T = np.zeros(mpr.mpr_get_info(ctx).nblk, np.float32)
        mpr.mpr_calibrate(ctx, T)
        mpr.mpr_destroy(ctx)
        line["cpu_baseline"] = cpu_baseline(wl, T, args.cpu_seconds)
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_ours_batch(args, world, rank, local):
    """Batched form: all fields of a batch workload in one context (one launch
    per half-step for all of them), against the plain form (one FP32 context
    per field, one after another) on a sample of the fields."""
    import torch
    from paper_2212_01317_gb300 import mpr, replicas, synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    mpr.load()
    bw = synth.batch_workload(args.workload, seed=rank)
    R = bw.realizations
    stream = torch.cuda.current_stream(dev)
    vals_h = [np.where(m != 0, np.nan, z).astype(np.float32) for z, m in zip(bw.truths, bw.masks)]
    vals_d = [torch.from_numpy(v).to(dev) for v in vals_h]
    masks_d = [torch.from_numpy(m).to(dev) for m in bw.masks]
    outs_d = [torch.empty(m.shape, dtype=torch.float32, device=dev) for m in bw.masks]
    grids = [(m.shape[0], m.shape[1], bw.block) for m in bw.masks]
    storage = args.storage
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def options(profile, st=storage, slice_id=0):
        return mpr.mpr_default_options(seed=2024 + 7919 * rank, slice_id=slice_id, profile=profile,
                                       storage=STORAGE[st], cal_mode=args.cal_mode,
                                       cal_method=1 if args.calibration == "newton" else 0,
                                       cal_points=args.cal_points, n_bisect=cal_iters(args),
                                       sim_graph=0, cuda_stream=stream.cuda_stream)

    def step(values, masks, outs, profile=1):
        ctx = mpr.mpr_create_batch(grids, masks, values, options(profile))
        try:
            mpr.mpr_calibrate(ctx, None)
            mpr.mpr_simulate(ctx, R)
            mpr.mpr_predict_batch(ctx, outs)
            info = mpr.mpr_get_info(ctx)
            prof = mpr.mpr_get_profile(ctx)
        finally:
            mpr.mpr_destroy(ctx)
        return info, prof

    for _ in range(args.warmup):
        step(vals_d, masks_d, outs_d)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    step_ms, updates, sim_updates, launches, sim_ms, sim_launch = [], 0, 0, 0, 0.0, 0
    tail_updates = 0
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        info, prof = step(vals_d, masks_d, outs_d)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        updates += info.gap_updates + info.cal_gap_updates
        sim_updates += info.gap_updates
        launches += prof.kernel_launches
        sim_ms += prof.sim_halfstep_ms
        sim_launch += prof.sim_halfstep_launches
        tail_updates += prof.sim_tail_updates
    torch.cuda.synchronize()
    clk = clocks.stop()
    total_ms = replicas.max_over_ranks(float(np.sum(step_ms)), dev)
    updates_all = replicas.sum_over_ranks(updates, dev)
    P = bw.n_gap
    value = updates_all / (total_ms / 1e3)
    mpix = world * P * args.steps / (total_ms / 1e3) / 1e6
    # Accuracy of the timed form: AAE over all gap sites of the last step.
    err = sum(float(np.abs(o.cpu().numpy() - z)[m != 0].sum())
              for o, z, m in zip(outs_d, bw.truths, bw.masks))
    aae = err / P

    # The plain form on a sample of fields: one FP32 context per field, in turn.
    plain = None
    if args.plain_sample > 0 and rank == 0:
        k = min(args.plain_sample, len(bw.masks))
        ups, t_plain, gaps, err_p = 0, 0.0, 0, 0.0
        for j in range(k):
            H, W = bw.masks[j].shape
            o1 = torch.empty((H, W), dtype=torch.float32, device=dev)
            for rep in range(2):                 # first pass warms the allocator and caches
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ctx = mpr.mpr_create(H, W, bw.block, masks_d[j], vals_d[j],
                                     options(0, "f32", slice_id=j))
                mpr.mpr_calibrate(ctx, None)
                mpr.mpr_simulate(ctx, R)
                mpr.mpr_predict(ctx, o1)
                inf = mpr.mpr_get_info(ctx)
                mpr.mpr_destroy(ctx)
                e1.record(stream)
                e1.synchronize()
            ups += inf.gap_updates + inf.cal_gap_updates
            t_plain += e0.elapsed_time(e1)
            gaps += int(np.count_nonzero(bw.masks[j]))
            err_p += float(np.abs(o1.cpu().numpy() - bw.truths[j])[bw.masks[j] != 0].sum())
        err_b = sum(float(np.abs(outs_d[j].cpu().numpy() - bw.truths[j])[bw.masks[j] != 0].sum())
                    for j in range(k))
        plain = {"value": ups / (t_plain / 1e3), "unit": "updates/s",
                 "gap_filled_mpix_s": gaps / (t_plain / 1e3) / 1e6, "aae": err_p / gaps,
                 "aae_batched_same_fields": err_b / gaps,
                 "sample": f"fields 0..{k - 1} of {len(bw.masks)}, one FP32 context each, "
                           "calibrate + simulate + predict, one after another"}
    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return
    peak, peak_kind = measured_peaks()
    p_mean = P / bw.n_sites
    bpu = bytes_per_gap_update(4.0 if storage == "f32" else 2.0, p_mean)
    # (the stop-tail launch's updates are timed and counted apart)
    achieved = (sim_updates - tail_updates) * bpu / (sim_ms / 1e3) / 1e9 if sim_ms > 0 else None
    line = {
        "metric": METRIC, "value": value, "unit": "updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": bw.name, "fields": len(bw.masks), "sites": bw.n_sites,
                   "gap_sites": P, "block": bw.block, "realizations": R, "storage": storage,
                   "form": "batched: every field in one context",
                   "calibration": args.calibration if args.calibration == "newton" else
                   ("bisection" if args.cal_points == 1 else "trisection") + f" x{cal_iters(args)}",
                   "l2": "inputs larger than L2; flushed between timed steps",
                   "parallelism": f"replicas{world}"},
        "gap_filled_mpix_s": mpix, "aae": aae,
        "gpu_launches": int(launches),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": (achieved / peak) if achieved else None, "traffic": None,
                     "kernel": "k_sweep_half / k_sweep (realizations)", "peak_kind": peak_kind,
                     "bytes_per_gap_update": bpu,
                     "avg_launch_us": 1e3 * sim_ms / sim_launch if sim_launch else None},
        "clocks": clk, "e2e": None, "plain_form": plain,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_ours_3d(args, world, rank, local):
    """The 3-D extension (mpr3_*): calibrate, simulate, predict one D x H x W
    field per step, inputs resident on the device; the roofline of its
    half-step kernel (k3_sweep) from CUDA events around each sweep."""
    import ctypes as C
    import torch
    from paper_2212_01317_gb300 import mpr, replicas, synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    lib = mpr.load()
    wl = synth.workload(args.workload, seed=rank)
    D, H, W = wl.shape
    n = D * H * W
    P = wl.n_gap
    p = P / n
    R = wl.realizations
    stream = torch.cuda.current_stream(dev)
    vals_d = torch.from_numpy(np.where(wl.mask != 0, np.nan, wl.truth).astype(np.float32)).to(dev)
    mask_d = torch.from_numpy(wl.mask).to(dev)
    out_d = torch.empty((D, H, W), dtype=torch.float32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def check(ctx, st):
        if st != mpr.MPR_OK:
            raise mpr.MprError(st, lib.mpr3_last_error(ctx).decode() if ctx else "")

    def step(profile=1):
        o = mpr.mpr_default_options(seed=2024 + 7919 * rank, slice_id=rank, profile=profile,
                                    n_bisect=cal_iters(args) if args.cal_points == 1 else 24,
                                    cuda_stream=stream.cuda_stream)
        ctx = C.c_void_p()
        g = mpr.mpr_grid3(D, H, W, wl.block)
        check(None, lib.mpr3_create(C.byref(g), mpr._ptr(mask_d), mpr._ptr(vals_d), C.byref(o),
                                    C.byref(ctx)))
        try:
            check(ctx, lib.mpr3_calibrate(ctx, None))
            check(ctx, lib.mpr3_simulate(ctx, R))
            check(ctx, lib.mpr3_predict(ctx, mpr._ptr(out_d), None, None))
            info = mpr.mpr3_info()
            check(ctx, lib.mpr3_get_info(ctx, C.byref(info)))
            prof = mpr.mpr_profile()
            check(ctx, lib.mpr3_get_profile(ctx, C.byref(prof)))
        finally:
            lib.mpr3_destroy(ctx)
        return info, prof

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    step_ms, ups, sim_ups, launches, sim_ms, sim_launch, cal_ms = [], 0, 0, 0, 0.0, 0, 0.0
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        info, prof = step()
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        ups += info.gap_updates + info.cal_gap_updates
        sim_ups += info.gap_updates
        launches += prof.kernel_launches
        sim_ms += prof.sim_halfstep_ms
        sim_launch += prof.sim_halfstep_launches
        cal_ms += prof.cal_halfstep_ms
    torch.cuda.synchronize()
    clk = clocks.stop()
    total_ms = replicas.max_over_ranks(float(np.sum(step_ms)), dev)
    ups_all = replicas.sum_over_ranks(ups, dev)
    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return
    peak, peak_kind = measured_peaks()
    bpu = bytes_per_gap_update(4.0, p)
    achieved = sim_ups * bpu / (sim_ms / 1e3) / 1e9 if sim_ms > 0 else None
    # DRAM bytes per launch: the ncu-measured bytes per update of this
    # workload's half-step (profiles/traffic.json) times the updates per launch.
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tpath) and sim_launch:
        with open(tpath) as f:
            rec = json.load(f).get(f"sim_{wl.name}")
        if rec:
            traffic = rec["bytes_per_update"] * sim_ups / sim_launch
    line = {
        "metric": METRIC, "value": ups_all / (total_ms / 1e3), "unit": "updates/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": wl.name, "D": D, "H": H, "W": W, "block": wl.block,
                   "gap_fraction": p, "realizations": R, "storage": "f32",
                   "calibration": "bisection x24",
                   "l2": "inputs larger than L2; flushed between timed steps",
                   "parallelism": f"replicas{world}"},
        "gap_filled_mpix_s": world * P * args.steps / (total_ms / 1e3) / 1e6,
        "gpu_launches": int(launches),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                     "kernel": "k3_sweep (realizations)", "peak_kind": peak_kind,
                     "bytes_per_gap_update": bpu,
                     "avg_launch_us": 1e3 * sim_ms / max(sim_launch, 1),
                     "sim_halfstep": {"ms": sim_ms / args.steps,
                                      "launches": sim_launch // args.steps,
                                      "updates_per_s": sim_ups / (sim_ms / 1e3) if sim_ms else None},
                     "calibration_ms": cal_ms / args.steps},
        "clocks": clk,
        "e2e": None,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    args = parse()
    world, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    from paper_2212_01317_gb300 import synth
    if args.workload in synth.BATCH_WORKLOADS:
        run_ours_batch(args, world, rank, local)
        return
    if args.workload.startswith("cube"):
        run_ours_3d(args, world, rank, local)
        return
    run_ours(args, world, rank, local)


if __name__ == "__main__":
    main()
