#!/usr/bin/env python
"""Benchmark: segments/s of nested-geometry particle tracking on GB300.

Workload: the three-level nested rectilinear core (15x15 assemblies of 17x17
pins inside a vacuum cylinder r=170 cm, h=366 cm, 4 materials, absorption
0.25), 1e7 particles per GPU per step, synthetic inputs from the seeded
generator.  One step = source_init + run_histories (BVH-CSG tracker, FP64,
event-based kernel) over the whole batch: every step of the hot path.
Companion lines: the rect tracker and the history kernel on the same
workload, FP32-local precision, and the 64-geometry batched workload
(FP32-local persistent launch replayed from a CUDA graph vs the plain FP64
history kernel launched once per geometry).

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
CPU_SAMPLE = 4_000_000
CPU_SAMPLE_ONE_CORE = 200_000
EVENT_SLOTS = 512
# near-surface comparison of the benchmarked launch with the oracle
NEAR_RULE_SAMPLE = 300
TRACE_CAP = 96
# DRAM bytes (read + write) per segment of the dominant kernel, from one ncu
# capture of the same kernel on the same geometry with 3e6 particles
# (16.55 GB over 82,931,315 segments); scaled to a full launch by its
# segments.  None whenever the kernel has changed since that capture.
TRAFFIC_BYTES_PER_SEGMENT = (6.667772928e9 + 9.878520576e9) / 82931315
# the same for the other rooflines' kernels, from small-case captures:
# k_event<CSG,FP32-local> on the same 3e6-particle case; the one
# k_batched_ev<CSG,FP32-local> launch of a 64-geometry pass (chunk 512,
# queue depth 512); k_transmission_bwd on 2^18 rays of the transmission
# workload (traffic scales with rays)
TRAFFIC_BYTES_PER_SEGMENT_FP32 = (14.747693e9 + 16.041718e9) / 82931442
TRAFFIC_BYTES_PER_SEGMENT_BATCH = (58.925292e9 + 54.138522e9) / 301969347
TRAFFIC_BYTES_PER_RAY_BWD = (15.207424e6 + 4.624384e6) / 262144
# Algorithmic FP64 operations per unit of work, the rooflines' numerators,
# from `python -m oracle.flop_counts` (the oracle's counting build in
# array-tracker mode; add/sub, mul, div and sqrt count one each): per
# segment of the main workload; per segment of the 64-geometry batch (its
# array-lattice members' figure, which undercounts the hex members); per ray
# of the transmission workload (the segment arithmetic the backward kernel
# recomputes; its derivative terms are not counted).
OPS_PER_SEGMENT = 100.74230573512504
OPS_PER_SEGMENT_BATCH = 70.55553343953962
OPS_PER_RAY_TRANSMISSION = 41880.890625


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
def cpu_baseline(desc_json: str, n: int, n_one: int, first_id: int = 0, traced=None) -> dict:
    """The oracle on all host cores (n particles) and on one core (n_one).

    traced: optional (particle ids, instance rows, length rows, cap) from the
    benchmarked event kernel's segment log; after the timing, those particles
    are compared one by one with the oracle under the near-surface rule
    (oracle.compare) and the counts are returned under "near_surface_rule"."""
    import oracle as O
    g = O.Geometry(desc_json, O.MODE_CSG)
    cores = host_cores()
    t0 = time.perf_counter()
    r = g.run(n, SEED, P_ABSORB, first_id=first_id, threads=cores, records=False)
    dt = time.perf_counter() - t0
    seg = int(r["counters"][O.K_SEGMENTS])
    t0 = time.perf_counter()
    r1 = g.run(n_one, SEED, P_ABSORB, first_id=first_id, threads=1, records=False)
    dt1 = time.perf_counter() - t0
    seg1 = int(r1["counters"][O.K_SEGMENTS])
    out = {"value": seg / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
           "one_core": seg1 / dt1,
           "sample": f"{n} particles (ids {first_id}..{first_id + n - 1}) of the same workload, CSG-mode "
                     f"oracle, {seg} segments in {dt:.2f} s on {cores} threads; one core: {n_one} particles, "
                     f"{seg1} segments in {dt1:.2f} s"}
    if traced is not None:
        from oracle import compare as C
        ids, rows_i, rows_l, cap = traced
        res = C.compare_traces(g, ids, rows_i, rows_l, SEED, P_ABSORB, cap)
        out["near_surface_rule"] = {
            "compared": res["compared"], "matched": res["matched"], "near_surface": len(res["near_surface"]),
            "drift": len(res["drift"]), "failed": len(res["failed"]),
            "segments_matched": res["segments_compared"], "max_rel_matched": res["max_rel_matched"],
            "findings": (res["near_surface"] + res["drift"] + res["failed"])[:10]}
    return out


def tally_error(t32, t64, c32=None, c64=None) -> dict:
    """Error of an FP32-local result against the FP64 result for the same
    particles (same ids, seed and options).  t32, t64: lists of int64 tally
    arrays (fixed point, 2^-32 cm) or single arrays; c32, c64: their counter
    arrays.  The FP64 path is the oracle's arithmetic: bit-equal to it in the
    exact build, within 1e-12 relative per distance in the fast build."""
    import numpy as np
    if not isinstance(t32, (list, tuple)):
        t32, t64 = [t32], [t64]
    a = np.concatenate([t.detach().cpu().numpy().view(np.uint64).astype(np.float64) for t in t32])
    b = np.concatenate([t.detach().cpu().numpy().view(np.uint64).astype(np.float64) for t in t64])
    d = np.abs(a - b)
    hit = b > 0
    rel = d[hit] / b[hit]
    out = {"tally_l1_rel": float(d.sum() / b.sum()) if b.sum() > 0 else None,
           "tally_linf_rel": float(rel.max()) if rel.size else None,
           "tally_p99_rel": float(np.quantile(rel, 0.99)) if rel.size else None,
           "tally_median_rel": float(np.median(rel)) if rel.size else None,
           "bins": int(b.size), "bins_only_fp32": int(np.count_nonzero((a > 0) & ~hit))}
    if c32 is not None and c64 is not None:
        s32 = float(np.asarray(c32, dtype=np.float64)[0])
        s64 = float(np.asarray(c64, dtype=np.float64)[0])
        out["segments_rel_diff"] = (s32 - s64) / s64 if s64 else None
        out["close_call_fraction"] = float(np.asarray(c32, dtype=np.float64)[10]) / max(1.0, s32)
    out["against"] = "FP64 event kernel, same particles and seeds (per-bin relative error over bins the FP64 run hit)"
    return out


def _guarded(fn):
    """Runs an auxiliary report; a Python-level failure becomes an error entry
    instead of ending the benchmark line."""
    try:
        return fn()
    except Exception as e:  # noqa: BLE001 - reported in the JSON line
        return {"error": f"{type(e).__name__}: {e}"}


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
    work_cache = {}

    def make_opts(tracker, mode, prec=N.FP64):
        return N.default_opts(tracker=tracker, mode=mode, precision=prec, seed=SEED, first_id=first_id,
                              p_absorb=P_ABSORB, queue_depth=EVENT_SLOTS)

    def work_for(opts):
        wb = g.work_bytes(n, opts)
        if not wb:
            return None
        if wb not in work_cache:
            work_cache[wb] = torch.empty(wb + 256, dtype=torch.uint8, device=dev)
        return work_cache[wb]

    def timed(tracker, mode, steps, warmup, prec=N.FP64, sampler=None):
        """K steps of source_init + run_histories; CUDA events on the stream."""
        opts = make_opts(tracker, mode, prec)
        work = work_for(opts)
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
        for a, b, c in ev:
            a.record(stream)
            g.source_init(n, seed=SEED, first_id=first_id, out=parts)
            b.record(stream)
            g.run_histories(parts, n, tally=tally, counters=cnt, opts=opts, work=work)
            c.record(stream)
        barrier()
        clocks = sampler.stop() if sampler else None
        c_host = cnt.cpu().numpy().view(np.uint64)
        return {"ms": sum(a.elapsed_time(c) for a, b, c in ev), "kernel_ms": [b.elapsed_time(c) for a, b, c in ev],
                "segments": int(c_host[0]), "counters": c_host.copy(), "clocks": clocks}

    def rate(r):
        return r["segments"] / (r["ms"] / 1e3)

    # ---- main line: BVH-CSG tracker, FP64, event-based kernel ---------------
    main_run = timed(N.TRACKER_CSG, N.MODE_EVENT, args.steps, args.warmup, sampler=ClockSampler(local))
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

    # ---- the exchange a sharded run needs: the integer tallies and counters
    # of every rank merged into one (outside the timed region).  Rank 0
    # checks the merge on a sample: every rank tracks the first ids of its
    # range, and rank 0 tracks all of them alone.
    exchange = None
    if world > 1:
        from paper_2406_13849_gb300 import sharding as SH
        m_t, m_c = tally.clone(), cnt.clone()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        e0.record(stream)
        SH.merge_tallies(m_t, m_c)
        e1.record(stream)
        barrier()
        n_s = 20_000
        opts_s = make_opts(N.TRACKER_CSG, N.MODE_EVENT)
        sp = g.source_init(n_s, seed=SEED, first_id=first_id)
        st_t, st_c, _ = g.run_histories(sp, n_s, opts=opts_s, work=work_for(opts_s))
        SH.merge_tallies(st_t, st_c)
        ok = None
        if rank == 0:
            ref_t = torch.zeros_like(st_t)
            ref_c = torch.zeros_like(st_c)
            for r in range(world):
                o_r = N.default_opts(tracker=N.TRACKER_CSG, mode=N.MODE_EVENT, seed=SEED, first_id=r * n,
                                     p_absorb=P_ABSORB, queue_depth=EVENT_SLOTS)
                rp = g.source_init(n_s, seed=SEED, first_id=r * n)
                g.run_histories(rp, n_s, tally=ref_t, counters=ref_c, opts=o_r, work=work_for(o_r))
            torch.cuda.synchronize()
            ok = bool(torch.equal(ref_t, st_t) and torch.equal(ref_c, st_c))
        exchange = {"what": "all-reduce of the uint64 cell tally (SUM) and counters (SUM; status MIN)",
                    "bytes_per_rank": int(m_t.numel() * 8 + m_c.numel() * 8), "ms": e0.elapsed_time(e1),
                    "merged_segments": int(m_c[0]),
                    "check": ("a %d-particle sample per rank merged equals rank 0 tracking all of them: %s"
                              % (n_s, ok)) if rank == 0 else None}

    # ---- companions on the same workload ----------------------------------
    k2 = max(2, args.steps // 2)
    rect_ev = timed(N.TRACKER_RECT, N.MODE_EVENT, k2, 3)
    csg_hist = timed(N.TRACKER_CSG, N.MODE_HISTORY, k2, 3)
    rect_hist = timed(N.TRACKER_RECT, N.MODE_HISTORY, k2, 3)
    # the paper's DP method: the array tracker's work behind virtual calls per level
    dp_hist = timed(N.TRACKER_DP, N.MODE_HISTORY, k2, 3)
    csg_ev32 = timed(N.TRACKER_CSG, N.MODE_EVENT, k2, 3, prec=N.FP32_LOCAL)
    # the same workload with the bounding interval hierarchy (Sec. 4.3) as the CSG search
    g_bvh = g
    g = N.Geometry(I.to_json(dict(I.config2(), accel="bih")), device=dev)
    csg_ev_bih = timed(N.TRACKER_CSG, N.MODE_EVENT, k2, 3)
    g = g_bvh

    # ---- FP32-local error against FP64 on the same particles (untimed) -----
    def fp32_error_main():
        t64, t32 = torch.zeros_like(tally), torch.zeros_like(tally)
        c64, c32 = torch.zeros_like(cnt), torch.zeros_like(cnt)
        g.source_init(n, seed=SEED, first_id=first_id, out=parts)
        for prec, t, c in ((N.FP64, t64, c64), (N.FP32_LOCAL, t32, c32)):
            o = make_opts(N.TRACKER_CSG, N.MODE_EVENT, prec)
            g.run_histories(parts, n, tally=t, counters=c, opts=o, work=work_for(o))
        torch.cuda.synchronize()
        return tally_error(t32, t64, c32.cpu().numpy().view(np.uint64), c64.cpu().numpy().view(np.uint64))
    fp32_err = _guarded(fp32_error_main)

    # ---- end to end through the C-ABI with host buffers ---------------------
    host_parts = torch.empty(parts.numel(), dtype=torch.uint8, pin_memory=True)
    g.source_init(n, seed=SEED, first_id=first_id, out=parts)
    host_parts.copy_(parts)
    opts = make_opts(N.TRACKER_CSG, N.MODE_EVENT)
    work = work_for(opts)
    # one untimed end-to-end step first (the copy path and the buffers warm)
    parts.copy_(host_parts, non_blocking=True)
    g.run_histories(parts, n, tally=tally, counters=cnt, opts=opts, work=work)
    g.tally_read(tally, cnt)
    cnt.zero_()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(k2):
        parts.copy_(host_parts, non_blocking=True)
        tally.zero_()
        g.run_histories(parts, n, tally=tally, counters=cnt, opts=opts, work=work)
        g.tally_read(tally, cnt)          # device -> host, synchronises the stream
    e1.record(stream)
    barrier()
    e2e_seg = float(cnt.cpu().numpy().view(np.uint64)[0])
    e2e_ms = e0.elapsed_time(e1)
    if world > 1:
        # as for the main value: the slowest rank's time, the segments of all ranks
        t_local = torch.tensor([e2e_ms, e2e_seg], dtype=torch.float64, device=dev)
        tmax, tsum = t_local.clone(), t_local.clone()
        dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
        dist.all_reduce(tsum, op=dist.ReduceOp.SUM)
        e2e_ms, e2e_seg = float(tmax[0]), float(tsum[1])
    e2e = {"value": e2e_seg / (e2e_ms / 1e3), "unit": UNIT,
           "h2d_bytes_per_step": int(parts.numel()), "d2h_bytes_per_step": int(g.n_inst * 8 + 8)}

    # ---- batched: 64 geometries, FP32-local graph replay vs FP64 launch loop
    batch = run_config4(N, I, dev, stream, barrier, rank, k2, world)

    # ---- roofline of the dominant kernel (the event kernel, CSG, FP64) ------
    kern_ms = statistics.mean(main_run["kernel_ms"])
    seg_per_launch = main_run["segments"] / args.steps
    achieved = OPS_PER_SEGMENT * seg_per_launch / (kern_ms / 1e3) / 1e12
    scratch = torch.empty(1 << 16, dtype=torch.uint8, device=dev)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    pk = 0.0
    for _ in range(3):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ops = N.peak_kernel(0, sms * 8, 4096, 0, scratch)
        b.record(stream)
        torch.cuda.synchronize()
        pk = max(pk, ops / (a.elapsed_time(b) / 1e3) / 1e12)
    # the other ceilings of the tracking kernels: FP32 FMA and u64 atomic adds
    # into L2, spread over a tally-sized array and contended on 1024 bins
    big = torch.empty(max(1 << 16, 8 * g.n_inst), dtype=torch.uint8, device=dev)

    def peak_of(kind, blocks, iters, nbins, buf):
        best = 0.0
        for _ in range(3):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ops = N.peak_kernel(kind, blocks, iters, nbins, buf)
            b.record(stream)
            torch.cuda.synchronize()
            best = max(best, ops / (a.elapsed_time(b) / 1e3))
        return best
    fp32_tf = peak_of(1, sms * 8, 4096, 0, scratch) / 1e12
    atom_spread = peak_of(2, sms * 8, 256, g.n_inst, big)
    atom_hot = peak_of(2, sms * 8, 64, 1024, big)
    seg_rate_kernel = seg_per_launch / (kern_ms / 1e3)
    traffic_launch = TRAFFIC_BYTES_PER_SEGMENT * seg_per_launch if TRAFFIC_BYTES_PER_SEGMENT else None
    hbm_peak = None
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            hbm_peak = float(json.load(f)["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        hbm_peak = 6800.0
    util = {"fp64_pipe": achieved / pk if pk else None,
            "l2_atomic": seg_rate_kernel / atom_spread if atom_spread else None,
            "hbm": (traffic_launch / (kern_ms / 1e3) / 1e9 / hbm_peak) if traffic_launch else None}
    util["max"] = max(v for v in util.values() if v is not None)
    peaks = {"fp64_fma_tflops": pk, "fp32_fma_tflops": fp32_tf,
             "u64_atomic_per_s_spread": atom_spread, "u64_atomic_per_s_1024_bins": atom_hot,
             "hbm_gbs": hbm_peak, "source": "trk_peak_kernel in this run (CUDA events, best of 3); HBM from "
                                             "the measured copy bandwidth"}
    roofline = {"bound": "alu", "achieved": achieved, "peak": pk, "unit": "TFLOP/s",
                "frac": achieved / pk if pk else None,
                "traffic": TRAFFIC_BYTES_PER_SEGMENT * seg_per_launch if TRAFFIC_BYTES_PER_SEGMENT else None,
                "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch with 3e6 "
                                  "particles, scaled by segments per launch",
                "kernel": "k_event<CSG,FP64> (run_histories, event mode)",
                "peak_source": "measured FP64 FMA rate (trk_peak_kernel, same run; of measured)",
                "flops_per_segment": OPS_PER_SEGMENT,
                "flops_definition": "FP64 add/sub, mul, div, sqrt per segment counted by the oracle's counting "
                                    "build in rect-tracker mode on this workload (python -m oracle.flop_counts)",
                "utilisation": util,
                "utilisation_definition": "fp64_pipe: frac; l2_atomic: tally atomics (one per segment) per second "
                                          "over the spread u64 atomic rate; hbm: traffic per launch over the "
                                          "launch time, over the measured copy bandwidth",
                "peaks": peaks}

    # ---- configuration 1 size sweep and the transmission workload ----------
    sweep = run_config1_sweep(N, I, dev, stream, barrier)
    hexcore = run_config3(N, I, dev, stream, barrier, k2)
    meshline = run_mesh_tally(N, I, dev, stream, barrier, k2, rate(main_run), rate(rect_ev))
    trans = run_config5(N, I, dev, stream, barrier, k2)
    power = run_power(N, I, dev, stream, barrier, 2, n * args.steps / (main_run["ms"] / 1e3))

    cpu = None
    near_rule = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the benchmarked launch (fast build, event kernel, CSG, queue depth
        # 512, all particles) with its segment log on: a sample of particles
        # is compared with the oracle under the near-surface rule
        def traced_sample():
            import numpy as np
            g.source_init(n, seed=SEED, first_id=first_id, out=parts)
            inst, ln, _, _ = g.trace(parts, n, TRACE_CAP, opts=make_opts(N.TRACKER_CSG, N.MODE_EVENT),
                                     work=work_for(make_opts(N.TRACKER_CSG, N.MODE_EVENT)))
            ids = np.sort(np.random.default_rng(23).choice(n, NEAR_RULE_SAMPLE, replace=False))
            r = torch.from_numpy(ids).to(dev)
            rows = (inst[r].cpu().numpy(), ln[r].cpu().numpy())
            del inst, ln
            torch.cuda.empty_cache()
            return (ids + first_id, rows[0], rows[1], TRACE_CAP)
        traced = _guarded(traced_sample)
        cpu = cpu_baseline(desc, CPU_SAMPLE, CPU_SAMPLE_ONE_CORE,
                           traced=traced if isinstance(traced, tuple) else None)
        cpu["gpu_core_equivalents"] = value / cpu["one_core"]
        near_rule = cpu.pop("near_surface_rule", traced if isinstance(traced, dict) else None)
        if isinstance(near_rule, dict) and "compared" in near_rule:
            near_rule["sample"] = (f"{NEAR_RULE_SAMPLE} particles drawn from the benchmarked launch ({n} particles, "
                                   f"fast build, event kernel, BVH-CSG, queue depth {EVENT_SLOTS}) traced to "
                                   f"{TRACE_CAP} segments each, compared one by one with the oracle")
            near_rule["rule"] = ("instances equal and lengths within 1e-12 relative or the propagated rounding "
                                 "bound; else the first mismatch within 1e-9 cm of the deciding surface")

    # ---- rooflines of the other kernels (same definitions; FP64 FMA peak) ---
    def alu_roofline(kernel, ops_per_unit, units, seconds, traffic, traffic_source, unit_name, time_source):
        ach = ops_per_unit * units / seconds / 1e12
        return {"bound": "alu", "achieved": ach, "peak": pk, "unit": "TFLOP/s", "frac": ach / pk if pk else None,
                "traffic": traffic, "traffic_source": traffic_source, "kernel": kernel,
                "flops_per_unit": ops_per_unit, "work_unit": unit_name, "units_per_launch": units,
                "time_source": time_source,
                "peak_source": "measured FP64 FMA rate (trk_peak_kernel, same run; of measured)"}
    seg32 = csg_ev32["segments"] / k2
    rooflines = {
        "fp32local_event": alu_roofline(
            "k_event<CSG,FP32-local> (run_histories, event mode, main workload)", OPS_PER_SEGMENT, seg32,
            statistics.mean(csg_ev32["kernel_ms"]) / 1e3, TRAFFIC_BYTES_PER_SEGMENT_FP32 * seg32,
            "ncu dram bytes of one 3e6-particle launch, scaled by segments", "segment",
            "CUDA events around run_histories"),
    }
    if batch and batch.get("batched_fp32local_graph_segments_per_s"):
        seg_b = batch["segments_per_particle"] * batch["particles"]
        rooflines["batched_event_fp32local"] = alu_roofline(
            "k_batched_ev<CSG,FP32-local> (one 64-geometry pass)",
            OPS_PER_SEGMENT_BATCH, seg_b, seg_b / batch["batched_fp32local_graph_segments_per_s"],
            TRAFFIC_BYTES_PER_SEGMENT_BATCH * seg_b,
            "ncu dram bytes of one pass (chunk 512), scaled by segments", "segment",
            "CUDA events around the graph replay")
    if trans:
        rooflines["transmission_bwd"] = alu_roofline(
            "k_transmission_bwd (2^20 rays)", OPS_PER_RAY_TRANSMISSION, trans["rays"], trans["bwd_ms"] / 1e3,
            TRAFFIC_BYTES_PER_RAY_BWD * trans["rays"], "ncu dram bytes of one 2^18-ray launch, scaled by rays",
            "ray", "CUDA events around transmission_bwd")
        rooflines["transmission_fwd"] = alu_roofline(
            "k_transmission (2^20 rays)", OPS_PER_RAY_TRANSMISSION, trans["rays"], trans["fwd_ms"] / 1e3,
            None, "no capture", "ray", "CUDA events around transmission_fwd")

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "particles_per_gpu": n, "tracker": "csg_bvh", "mode": "event",
                       "precision": "fp64", "build": "fast", "queue_depth": EVENT_SLOTS,
                       "l2": "inputs larger than L2 (particle buffer %d MB rewritten every step)" % (parts.numel() >> 20),
                       "step": "source_init + run_histories"},
            "particles_per_s": world * n * args.steps / (total_ms / 1e3),
            "clocks": main_run["clocks"],
            "e2e": e2e,
            "gpu_launches": 2 * args.steps,
            "roofline": roofline,
            "rooflines": rooflines,
            "cpu_baseline": cpu,
            "fast_build_near_surface_mismatches": near_rule,
            "exchange": exchange,
            "variants": {
                "csg_fp64_event": rate(main_run),
                "rect_fp64_event": rate(rect_ev),
                "csg_over_rect_event": rate(main_run) / rate(rect_ev),
                "csg_fp64_history": rate(csg_hist),
                "rect_fp64_history": rate(rect_hist),
                "csg_over_rect_history": rate(csg_hist) / rate(rect_hist),
                "dp_fp64_history": rate(dp_hist),
                "dp_over_rect_history": rate(dp_hist) / rate(rect_hist),
                "csg_fp32local_event": rate(csg_ev32),
                "csg_fp32local_error_vs_fp64": fp32_err,
                "csg_fp64_event_bih": rate(csg_ev_bih),
                "bih_over_bvh_event": rate(csg_ev_bih) / rate(main_run),
                "fp32local_close_call_fraction": float(csg_ev32["counters"][10]) / max(1, csg_ev32["segments"]),
                "segments_per_particle": main_run["segments"] / (n * args.steps),
                "event_kernel_ms": kern_ms,
            },
            "batched": batch,
            "config1_sweep": sweep,
            "config3": hexcore,
            "mesh_tally": meshline,
            "transmission": trans,
            "power_iteration": power,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_config4(N, I, dev, stream, barrier, rank, steps, world=1):
    """64 geometries (3x3..17x17 rect/hex, 2-3 levels, 1e4..1e6 particles):
    the batched event kernel (warp queues over chunks of one geometry at a
    time), FP32-local, autotuned and replayed from a CUDA graph, against the
    plain FP64 history kernel launched once per geometry.  With several
    ranks the geometries are split between them (whole problems per rank,
    balanced by particle count) and each rank reports its share."""
    import numpy as np
    import torch
    members = I.config4()
    if world > 1:
        from paper_2406_13849_gb300 import sharding as SH
        mine = SH.shard_geometries([c for _, c in members], world)[rank]
        members = [members[k] for k in mine]
    geoms = [N.Geometry(I.to_json(d), device=dev) for d, _ in members]
    counts = [c for _, c in members]
    parts = [g.source_init(c, seed=SEED) for g, c in zip(geoms, counts)]
    b = N.Batch(geoms, parts, counts)

    def graph_rate(opts):
        s = torch.cuda.Stream(device=dev)
        s.wait_stream(torch.cuda.current_stream())
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=s):
            b.run(opts)
        graph.replay()
        torch.cuda.synchronize()
        b.zero()
        barrier()
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            graph.replay()
        e.record(stream)
        barrier()
        seg = int(b.counters.cpu().numpy().view(np.uint64).reshape(-1, 16)[:, 0].sum())
        return seg / (a.elapsed_time(e) / 1e3)

    ev32 = N.default_opts(seed=SEED, p_absorb=P_ABSORB, precision=N.FP32_LOCAL, mode=N.MODE_EVENT)
    ev32, chunk_ev, _ = b.autotune(ev32, reps=2)
    r_ev32 = graph_rate(ev32)
    snap32 = ([t.clone() for t in b.tallies], b.counters.clone())
    ev64 = N.default_opts(seed=SEED, p_absorb=P_ABSORB, precision=N.FP64, mode=N.MODE_EVENT,
                          queue_depth=ev32.queue_depth, sort_interval=ev32.sort_interval)
    r_ev64 = graph_rate(ev64)
    snap64 = ([t.clone() for t in b.tallies], b.counters.clone())

    def batch_error():
        c32 = snap32[1].cpu().numpy().view(np.uint64).reshape(-1, 16).sum(axis=0)
        c64 = snap64[1].cpu().numpy().view(np.uint64).reshape(-1, 16).sum(axis=0)
        err = tally_error(snap32[0], snap64[0], c32, c64)
        per = [tally_error(t32, t64)["tally_l1_rel"] for t32, t64 in zip(snap32[0], snap64[0])]
        per = [v for v in per if v is not None]
        err["tally_l1_rel_worst_geometry"] = max(per) if per else None
        err["against"] = "batched FP64 event kernel, same particles, seeds and queue depth"
        return err
    ev_err = _guarded(batch_error)
    hi32 = N.default_opts(seed=SEED, p_absorb=P_ABSORB, precision=N.FP32_LOCAL)
    hi32, chunk_hi, _ = b.autotune(hi32, reps=2)
    r_hi32 = graph_rate(hi32)
    # per-geometry loop, plain FP64 history kernel
    tallies = [torch.zeros(gg.n_inst, dtype=torch.int64, device=dev) for gg in geoms]
    cnt = torch.zeros(16, dtype=torch.int64, device=dev)
    a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def loop_rate(opts, reps):
        wb = geoms[0].work_bytes(counts[0], opts)
        work = torch.empty(wb + 256, dtype=torch.uint8, device=dev) if wb else None
        for gg, pp, cc, tt in zip(geoms, parts, counts, tallies):
            gg.run_histories(pp, cc, tally=tt, counters=cnt, opts=opts, work=work)
        cnt.zero_()
        barrier()
        a.record(stream)
        for _ in range(reps):
            for gg, pp, cc, tt in zip(geoms, parts, counts, tallies):
                gg.run_histories(pp, cc, tally=tt, counters=cnt, opts=opts, work=work)
        e.record(stream)
        barrier()
        return int(cnt.cpu().numpy().view(np.uint64)[0]) / (a.elapsed_time(e) / 1e3)

    r_l = loop_rate(N.default_opts(seed=SEED, p_absorb=P_ABSORB, precision=N.FP64, mode=N.MODE_HISTORY), steps)
    r_l32 = loop_rate(N.default_opts(seed=SEED, p_absorb=P_ABSORB, precision=N.FP32_LOCAL, mode=N.MODE_HISTORY), 1)
    # the same event kernel launched once per geometry (what the batch saves
    # over a loop of the single-geometry event kernel)
    r_le32 = loop_rate(N.default_opts(seed=SEED, p_absorb=P_ABSORB, precision=N.FP32_LOCAL, mode=N.MODE_EVENT,
                                      queue_depth=ev32.queue_depth, sort_interval=ev32.sort_interval), 1)
    seg_per_particle = float(snap32[1].cpu().numpy().view(np.uint64).reshape(-1, 16)[:, 0].sum()) / max(1, sum(counts))
    return {"workload": "64 geometries: 3x3..17x17 rect/hex lattices, 2-3 levels, 1e4..1e6 particles "
                        "(log-uniform), %d particles" % sum(counts),
            "batched_fp32local_graph_segments_per_s": r_ev32,
            "batched_fp32local_error_vs_fp64": ev_err,
            "loop_fp64_history_segments_per_s": r_l,
            "batched_over_loop": r_ev32 / r_l,
            "batched_fp64_event_graph_segments_per_s": r_ev64,
            "batched_fp32local_history_graph_segments_per_s": r_hi32,
            "loop_fp32local_history_segments_per_s": r_l32,
            "loop_fp32local_event_segments_per_s": r_le32,
            "batched_over_event_loop": r_ev32 / r_le32,
            "segments_per_particle": seg_per_particle,
            "particles": sum(counts),
            "autotuned": {"event": {"queue_depth": ev32.queue_depth, "chunk": chunk_ev,
                                    "sort_interval": ev32.sort_interval},
                          "history": {"block": hi32.block, "chunk": chunk_hi}},
            "launches_per_pass": {"batched_event": 1, "batched_history": 1, "loop": len(geoms)},
            "geometries_on_this_rank": len(geoms)}


def run_config1_sweep(N, I, dev, stream, barrier):
    """One 17x17 pin lattice in a reflecting box (absorption 0.3): segments/s
    of the rect and BVH-CSG trackers (event kernel) from 1e4 to 1e8 particles,
    and the history kernel at the small sizes, where the event kernel's
    persistent grid is mostly idle."""
    import numpy as np
    import torch
    g = N.Geometry(I.to_json(I.config1()), device=dev)
    rows = []
    for n in (10_000, 100_000, 1_000_000, 10_000_000, 100_000_000):
        parts = torch.empty(g.particle_bytes(n), dtype=torch.uint8, device=dev)
        g.source_init(n, seed=SEED, out=parts)
        tally = torch.zeros(g.n_inst, dtype=torch.int64, device=dev)
        cnt = torch.zeros(N.NCOUNTERS, dtype=torch.int64, device=dev)
        row = {"particles": n}
        modes = [("event", N.MODE_EVENT)] + ([("history", N.MODE_HISTORY)] if n <= 1_000_000 else [])
        for mname, mode in modes:
            trackers = (("rect", N.TRACKER_RECT), ("csg", N.TRACKER_CSG))
            if mode == N.MODE_HISTORY:
                trackers += (("dp", N.TRACKER_DP),)
            for tname, tr in trackers:
                opts = N.default_opts(tracker=tr, mode=mode, seed=SEED, p_absorb=0.3, queue_depth=EVENT_SLOTS)
                wb = g.work_bytes(n, opts)
                work = torch.empty(wb + 256, dtype=torch.uint8, device=dev) if wb else None
                g.run_histories(parts, n, tally=tally, counters=cnt, opts=opts, work=work)
                reps = 1 if n >= 10_000_000 else 3
                cnt.zero_()
                barrier()
                a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                for _ in range(reps):
                    g.run_histories(parts, n, tally=tally, counters=cnt, opts=opts, work=work)
                e.record(stream)
                barrier()
                seg = int(cnt.cpu().numpy().view(np.uint64)[0])
                row[f"{tname}_{mname}"] = seg / (a.elapsed_time(e) / 1e3)
                del work
            row[f"csg_over_rect_{mname}"] = row[f"csg_{mname}"] / row[f"rect_{mname}"]
            if mode == N.MODE_HISTORY:
                row["dp_over_rect_history"] = row["dp_history"] / row["rect_history"]
        rows.append(row)
        del parts
    return {"workload": "17x17 pins (pitch 1.26, radii 0.41/0.475) in a reflecting box 21.42 x 21.42 x 100, "
                        "3 materials, absorption 0.3", "unit": UNIT, "rows": rows}


def run_config3(N, I, dev, stream, barrier, steps):
    """Hex core (127 assemblies of 91 pins, rings 6 of ring-6 lattices turned
    by 30 degrees), 1e7 particles, event kernel: the BVH-CSG tracker in FP64
    and FP32-local, and the array tracker (closed-form hex element search)
    in FP64."""
    import numpy as np
    import torch
    g = N.Geometry(I.to_json(I.config3()), device=dev)
    n = 10_000_000
    parts = torch.empty(g.particle_bytes(n), dtype=torch.uint8, device=dev)
    g.source_init(n, seed=SEED, out=parts)
    cnt = torch.zeros(N.NCOUNTERS, dtype=torch.int64, device=dev)
    tallies, counts = {}, {}
    out = {"workload": "hex core: 127 assemblies x 91 pins (rings 6 of ring-6 pin lattices turned 30 deg), "
                       "h=200, 5 materials, absorption 0.25, 1e7 particles", "unit": UNIT}
    g_bih = N.Geometry(I.to_json(dict(I.config3(), accel="bih")), device=dev)
    for name, tr, prec, gg in (("csg_fp64_event", N.TRACKER_CSG, N.FP64, g),
                               ("csg_fp32local_event", N.TRACKER_CSG, N.FP32_LOCAL, g),
                               ("array_fp64_event", N.TRACKER_RECT, N.FP64, g),
                               ("csg_fp64_event_bih", N.TRACKER_CSG, N.FP64, g_bih)):
        opts = N.default_opts(tracker=tr, mode=N.MODE_EVENT, precision=prec, seed=SEED,
                              p_absorb=P_ABSORB, queue_depth=EVENT_SLOTS)
        work = torch.empty(gg.work_bytes(n, opts) + 256, dtype=torch.uint8, device=dev)
        tally = torch.zeros(g.n_inst, dtype=torch.int64, device=dev)
        gg.run_histories(parts, n, tally=tally, counters=cnt, opts=opts, work=work)
        cnt.zero_()
        tally.zero_()
        barrier()
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            gg.run_histories(parts, n, tally=tally, counters=cnt, opts=opts, work=work)
        e.record(stream)
        barrier()
        c = cnt.cpu().numpy().view(np.uint64)
        tallies[name], counts[name] = tally, c.copy()
        out[name] = int(c[0]) / (a.elapsed_time(e) / 1e3)
        if prec == N.FP32_LOCAL:
            out["fp32local_close_call_fraction"] = float(c[10]) / max(1, int(c[0]))
        else:
            out["segments_per_particle"] = int(c[0]) / (n * steps)
        del work
    out["fp32local_over_fp64"] = out["csg_fp32local_event"] / out["csg_fp64_event"]
    out["csg_fp32local_error_vs_fp64"] = _guarded(lambda: tally_error(
        tallies["csg_fp32local_event"], tallies["csg_fp64_event"], counts["csg_fp32local_event"],
        counts["csg_fp64_event"]))
    out["csg_over_array"] = out["csg_fp64_event"] / out["array_fp64_event"]
    out["bih_over_bvh"] = out["csg_fp64_event_bih"] / out["csg_fp64_event"]
    return out


def run_mesh_tally(N, I, dev, stream, barrier, steps, csg_plain, rect_plain):
    """The main workload with the paper's active-cycle tally: track length on
    a superimposed 119 x 119 x 30 mesh over the core's box, event kernel,
    FP64, both trackers; the rates without the mesh tally are the main
    line's."""
    import numpy as np
    import torch
    desc = I.with_mesh(I.config2(), 119, 119, 30)
    g = N.Geometry(I.to_json(desc), device=dev)
    n = 10_000_000
    parts = torch.empty(g.particle_bytes(n), dtype=torch.uint8, device=dev)
    g.source_init(n, seed=SEED, out=parts)
    tally = torch.zeros(g.n_inst, dtype=torch.int64, device=dev)
    mesh = torch.zeros(g.mesh_bins, dtype=torch.int64, device=dev)
    cnt = torch.zeros(N.NCOUNTERS, dtype=torch.int64, device=dev)
    out = {"workload": "the main workload with a 119 x 119 x 30 superimposed mesh (424,830 bins) over the "
                       "core's box, track-length tally per segment", "unit": UNIT, "mesh_bins": g.mesh_bins}
    for name, tr, plain in (("csg", N.TRACKER_CSG, csg_plain), ("rect", N.TRACKER_RECT, rect_plain)):
        opts = N.default_opts(tracker=tr, mode=N.MODE_EVENT, seed=SEED, p_absorb=P_ABSORB, queue_depth=EVENT_SLOTS)
        opts.mesh_tally = mesh.data_ptr()
        work = torch.empty(g.work_bytes(n, opts) + 256, dtype=torch.uint8, device=dev)
        g.run_histories(parts, n, tally=tally, counters=cnt, opts=opts, work=work)
        cnt.zero_()
        barrier()
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            g.run_histories(parts, n, tally=tally, counters=cnt, opts=opts, work=work)
        e.record(stream)
        barrier()
        r = int(cnt.cpu().numpy().view(np.uint64)[0]) / (a.elapsed_time(e) / 1e3)
        out[f"{name}_fp64_event_with_mesh"] = r
        out[f"{name}_degradation"] = 1.0 - r / plain
        del work
    return out


def run_power(N, I, dev, stream, barrier, steps, plain_hist_per_s):
    """Power iteration (Alg. 1) on the main workload with a fissile fuel
    (nu = 2.4 in material 0): 2e6 histories per cycle, 2 inactive and 6
    active cycles per step, BVH-CSG tracker, event kernel, FP64.  Reported
    as histories per second over all cycles, against the main line's
    particles per second (source_init + run_histories, no fission bank)."""
    import numpy as np
    import torch
    desc = I.with_nu(I.config2(), [2.4, 0.0, 0.0, 0.0])
    g = N.Geometry(I.to_json(desc), device=dev)
    n, inactive, cycles = 2_000_000, 2, 8
    opts = N.default_opts(tracker=N.TRACKER_CSG, mode=N.MODE_EVENT, seed=SEED, p_absorb=P_ABSORB,
                          queue_depth=EVENT_SLOTS)
    tally = torch.zeros(g.n_inst, dtype=torch.int64, device=dev)
    cnt = torch.zeros(N.NCOUNTERS, dtype=torch.int64, device=dev)
    work = torch.empty(g.power_iteration_work_bytes(n, opts) + 256, dtype=torch.uint8, device=dev)
    k, bank, _, _ = g.power_iteration(n, inactive, cycles, tally=tally, counters=cnt, opts=opts, stream=stream,
                                      work=work)
    barrier()
    a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        k, bank, _, _ = g.power_iteration(n, inactive, cycles, tally=tally, counters=cnt, opts=opts, stream=stream,
                                          work=work)
    e.record(stream)
    barrier()
    ms = a.elapsed_time(e)
    kk = k.cpu().numpy()
    st = int(cnt.cpu().numpy().view(np.uint64)[N.K["status"]])
    hps = steps * n * cycles / (ms / 1e3)
    return {"workload": "main workload, fuel nu = 2.4, 2e6 histories per cycle, 2 inactive + 6 active cycles "
                        "per step, BVH-CSG, event kernel, FP64 (one work buffer reused by every call)",
            "histories_per_s": hps, "ms_per_cycle": ms / (steps * cycles),
            "over_plain_run": hps / plain_hist_per_s,
            "k_per_cycle": [float(x) for x in kk], "k_active_mean": float(kk[inactive:].mean()),
            "bank_per_cycle": [int(x) for x in bank.cpu().numpy()], "status": st}


def run_config5(N, I, dev, stream, barrier, steps):
    """Transmission of 2^20 boundary rays through the three-level core:
    forward (T per ray) and backward (gradients with respect to the four
    cross sections and the radii and pitch) times."""
    import torch
    desc, rays = I.config5()
    g = N.Geometry(I.to_json(desc), device=dev)
    R = torch.from_numpy(rays.packed()).to(dev)
    sigma = torch.tensor(desc["sigma"], dtype=torch.float64, device=dev)
    gT = torch.ones(R.shape[0], dtype=torch.float64, device=dev)
    pitch = 1.26
    work = torch.empty(max(8, g.transmission_bwd_work_bytes(R.shape[0])), dtype=torch.uint8, device=dev)
    for _ in range(2):
        T, _ = g.transmission_fwd(R, sigma, lens=False)
        g.transmission_bwd(R, sigma, pitch, gT, work=work)
    barrier()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    fwd = bwd = 0.0
    for _ in range(steps):
        ev[0].record(stream)
        T, _ = g.transmission_fwd(R, sigma, lens=False)
        ev[1].record(stream)
        g.transmission_bwd(R, sigma, pitch, gT, work=work)
        ev[2].record(stream)
        barrier()
        fwd += ev[0].elapsed_time(ev[1])
        bwd += ev[1].elapsed_time(ev[2])
    n = R.shape[0]
    return {"workload": "2^20 inward rays on the r=170, h=366 boundary of the three-level core",
            "rays": n, "fwd_ms": fwd / steps, "bwd_ms": bwd / steps,
            "rays_per_s_fwd_bwd": n / ((fwd + bwd) / steps / 1e3)}


if __name__ == "__main__":
    main()
