#!/usr/bin/env python
"""Benchmark: segments/s of nested-geometry particle tracking on GB300.

Workload: the three-level nested rectilinear core (15x15 assemblies of 17x17
pins inside a vacuum cylinder r=170 cm, h=366 cm, 4 materials, absorption
0.25), 1e7 particles per GPU per step, synthetic inputs from the seeded
generator.  One step = source_init + run_histories (BVH-CSG tracker, FP64,
history kernel) over the whole batch: every step of the hot path.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  N>1 runs under torchrun: each rank tracks
its own particle-id range (weak scaling, no collective in the timed region).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)

METRIC = "segments/s on 1 GB300: BVH-CSG vs rect tracker; batched FP32-local vs plain FP64"
UNIT = "segments/s"
WORKLOAD = "core_15x15_assemblies_17x17_pins_r170_h366_4mat_pabs0.25"
PARTICLES = 10_000_000
P_ABSORB = 0.25
SEED = 1
CPU_SAMPLE = 1_000_000


def _env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# CPU oracle baseline (bounded sample)
# ---------------------------------------------------------------------------
def cpu_baseline(desc_json: str, n: int, first_id: int = 0) -> dict:
    import oracle as O
    g = O.Geometry(desc_json, O.MODE_CSG)
    cores = host_cores()
    t0 = time.perf_counter()
    r = g.run(n, SEED, P_ABSORB, first_id=first_id, threads=cores, records=False)
    dt = time.perf_counter() - t0
    seg = int(r["counters"][O.K_SEGMENTS])
    return {"value": seg / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n} particles (ids {first_id}..{first_id + n - 1}) of the same workload, CSG-mode "
                      f"oracle, {seg} segments in {dt:.2f} s"}


def flops_per_segment(desc_json: str) -> dict:
    """Algorithmic FP64 operations per segment: the counting build of the
    oracle in rect-tracker mode (the fewest operations the method needs) on
    a sample of the workload; add/sub, mul, div and sqrt each count one."""
    import oracle as O
    g = O.Geometry(desc_json, O.MODE_RECT, counting=True)
    g.flop_counts(reset=True)
    r = g.run(2000, SEED, P_ABSORB, threads=1, records=False)
    fc = g.flop_counts()
    seg = float(r["counters"][O.K_SEGMENTS])
    ops = fc["add"] + fc["mul"] + fc["div"] + fc["sqrt"]
    return {"per_segment": ops / seg, "counts_per_segment": {k: v / seg for k, v in fc.items()}}


# ---------------------------------------------------------------------------
# reference arm: the CPU oracle as it stands
# ---------------------------------------------------------------------------
def run_reference(args, rank: int, world: int) -> None:
    if rank != 0:
        return
    from paper_2406_13849_gb300 import inputs as I
    import oracle as O
    desc = I.to_json(I.config2())
    g = O.Geometry(desc, O.MODE_CSG)
    cores = host_cores()
    per_step = 200_000
    for w in range(args.warmup):
        g.run(per_step // 10, SEED, P_ABSORB, first_id=w * per_step, threads=cores, records=False)
    seg = 0
    t0 = time.perf_counter()
    for k in range(args.steps):
        r = g.run(per_step, SEED, P_ABSORB, first_id=k * per_step, threads=cores, records=False)
        seg += int(r["counters"][O.K_SEGMENTS])
    dt = time.perf_counter() - t0
    v = seg / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "particles_per_step": per_step, "tracker": "csg (linear scan)",
                       "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} particles per step of the same workload"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--particles", type=int, default=PARTICLES)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    rank, world, local = _env_int("RANK", 0), _env_int("WORLD_SIZE", 1), _env_int("LOCAL_RANK", 0)
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")

    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2406_13849_gb300 import inputs as I
    from paper_2406_13849_gb300 import native as N

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    desc = I.to_json(I.config2())
    n = args.particles
    first_id = rank * n
    g = N.Geometry(desc, device=dev)
    stream = torch.cuda.current_stream()
    parts = torch.empty(g.particle_bytes(n), dtype=torch.uint8, device=dev)
    tally = torch.zeros(g.n_inst, dtype=torch.int64, device=dev)
    cnt = torch.zeros(N.NCOUNTERS, dtype=torch.int64, device=dev)

    def make_opts(tracker, mode=N.MODE_HISTORY):
        return N.default_opts(tracker=tracker, mode=mode, precision=N.FP64, seed=SEED,
                              first_id=first_id, p_absorb=P_ABSORB)

    work_cache = {}

    def timed(tracker, steps, warmup, sampler=None, mode=N.MODE_HISTORY):
        opts = make_opts(tracker, mode)
        wb = g.work_bytes(n, opts)
        work = None
        if wb:
            if wb not in work_cache:
                work_cache[wb] = torch.empty(wb + 256, dtype=torch.uint8, device=dev)
            work = work_cache[wb]
        for _ in range(warmup):
            g.source_init(n, seed=SEED, first_id=first_id, out=parts)
            g.run_histories(parts, n, tally=tally, counters=cnt, opts=opts, work=work)
        tally.zero_()
        cnt.zero_()
        barrier()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
               torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        if sampler:
            sampler.start()
        barrier()
        t0 = time.perf_counter()
        for a, b, c in ev:
            a.record(stream)
            g.source_init(n, seed=SEED, first_id=first_id, out=parts)
            b.record(stream)
            g.run_histories(parts, n, tally=tally, counters=cnt, opts=opts, work=work)
            c.record(stream)
        barrier()
        wall = time.perf_counter() - t0
        clocks = sampler.stop() if sampler else None
        step_ms = [a.elapsed_time(c) for a, b, c in ev]
        hist_ms = [b.elapsed_time(c) for a, b, c in ev]
        c_host = cnt.cpu().numpy().view(np.uint64)
        return {"ms": sum(step_ms), "hist_ms": hist_ms, "segments": int(c_host[0]), "wall": wall,
                "counters": c_host.copy(), "clocks": clocks}

    # main line: BVH-CSG tracker
    main_run = timed(N.TRACKER_CSG, args.steps, args.warmup, ClockSampler(local))
    # companion measurements (same workload): rect tracker, event-based kernel
    rect_run = timed(N.TRACKER_RECT, max(2, args.steps // 2), 3)
    ev_csg = timed(N.TRACKER_CSG, max(2, args.steps // 2), 3, mode=N.MODE_EVENT)
    ev_rect = timed(N.TRACKER_RECT, max(2, args.steps // 2), 3, mode=N.MODE_EVENT)

    # max over ranks
    t_local = torch.tensor([main_run["ms"], float(main_run["segments"])], dtype=torch.float64, device=dev)
    if world > 1:
        tmax = t_local.clone()
        dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
        tsum = t_local.clone()
        dist.all_reduce(tsum, op=dist.ReduceOp.SUM)
        total_ms, total_seg = float(tmax[0]), float(tsum[1])
    else:
        total_ms, total_seg = main_run["ms"], float(main_run["segments"])
    value = total_seg / (total_ms / 1e3)

    # end to end through the C-ABI with host buffers: births from pinned host
    # memory, tally and counters read back, every step
    host_parts = torch.empty(parts.numel(), dtype=torch.uint8, pin_memory=True)
    g.source_init(n, seed=SEED, first_id=first_id, out=parts)
    host_parts.copy_(parts)
    host_tally = np.zeros(g.n_inst)
    e2e_steps = max(2, args.steps // 2)
    opts = make_opts(N.TRACKER_CSG)
    cnt.zero_()
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(e2e_steps):
        parts.copy_(host_parts, non_blocking=True)
        tally.zero_()
        g.run_histories(parts, n, tally=tally, counters=cnt, opts=opts)
        host_tally = g.tally_read(tally, cnt)          # synchronises the stream
    e1.record(stream)
    barrier()
    e2e_ms = e0.elapsed_time(e1)
    e2e_seg = int(cnt.cpu().numpy().view(np.uint64)[0])
    e2e = {"value": world * e2e_seg / (e2e_ms / 1e3), "unit": UNIT,
           "h2d_bytes_per_step": int(parts.numel()), "d2h_bytes_per_step": int(g.n_inst * 8 + 8)}

    # roofline of the dominant kernel (the history kernel)
    fps = flops_per_segment(desc)
    hist_ms = statistics.mean(main_run["hist_ms"])
    seg_per_launch = main_run["segments"] / args.steps
    achieved = fps["per_segment"] * seg_per_launch / (hist_ms / 1e3) / 1e12
    scratch = torch.empty(1 << 16, dtype=torch.uint8, device=dev)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    pk_best = 0.0
    for _ in range(3):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ops = N.peak_kernel(0, sms * 8, 4096, 0, scratch)
        b.record(stream)
        torch.cuda.synchronize()
        pk_best = max(pk_best, ops / (a.elapsed_time(b) / 1e3) / 1e12)
    roofline = {"bound": "alu", "achieved": achieved, "peak": pk_best, "unit": "TFLOP/s",
                "frac": achieved / pk_best if pk_best else None, "traffic": None,
                "kernel": "k_history<CSG> (FP64)",
                "peak_source": "measured FP64 FMA issue rate (trk_peak_kernel, same run)",
                "flops_per_segment": fps["per_segment"]}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(desc, CPU_SAMPLE)

    rect_value = rect_run["segments"] / (rect_run["ms"] / 1e3)
    csg_value = main_run["segments"] / (main_run["ms"] / 1e3)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "particles_per_gpu": n, "tracker": "csg_bvh",
                       "mode": "history", "precision": "fp64", "build": "fast",
                       "l2": "inputs larger than L2 (particle buffer %d MB per step)" % (parts.numel() >> 20),
                       "step": "source_init + run_histories"},
            "particles_per_s": world * n * args.steps / (total_ms / 1e3),
            "clocks": main_run["clocks"],
            "e2e": e2e,
            "gpu_launches": 2 * args.steps,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "variants": {
                "csg_bvh_fp64_history_segments_per_s": csg_value,
                "rect_fp64_history_segments_per_s": rect_value,
                "csg_over_rect": csg_value / rect_value,
                "csg_bvh_fp64_event_segments_per_s": ev_csg["segments"] / (ev_csg["ms"] / 1e3),
                "rect_fp64_event_segments_per_s": ev_rect["segments"] / (ev_rect["ms"] / 1e3),
                "history_kernel_ms": hist_ms,
                "segments_per_particle": main_run["segments"] / (n * args.steps),
            },
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
