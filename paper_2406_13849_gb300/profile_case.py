"""Short launches of the tracking kernels on reduced workloads, for profilers.

The full benchmark holds ~1 GB on the device and launches many kernels; a
profiler that replays each captured launch dozens of times wants one short
launch instead.  Workloads:

  core          source_init, then `--launches` run_histories launches of one
                (tracker, mode, precision) on the three-level nested core
                (15x15 assemblies of 17x17 pins, the benchmark's geometry)
                with a particle count of the caller's choosing (default 3e6:
                180 MB of particle state, more than the 129 MB L2, so DRAM
                counters still mean something)
  hex           the same on the hexagonal core (127 assemblies of 91 pins)
  batch         the first `--members` geometries of the 64-geometry batch,
                `--launches` run_batched launches (event mode unless
                --mode history) at the benchmark's queue depth and chunk
  transmission  `--rays` boundary rays through the three-level core,
                `--launches` forward + backward passes

  python -m paper_2406_13849_gb300.profile_case [--workload core|hex|batch|transmission]
      [--tracker csg|rect|dp] [--mode event|history] [--precision fp64|fp32]
      [--particles N] [--launches L] [--members M] [--chunk C] [--batch-tracker auto|csg] [--rays R]

Prints one line with segments (or rays), kernel milliseconds and rates per
launch (CUDA events; meaningless under a profiler).
"""
from __future__ import annotations

import argparse
import json

import numpy as np
import torch

from . import inputs as I
from . import native as N


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="core", choices=["core", "hex", "batch", "transmission"])
    ap.add_argument("--tracker", default="csg", choices=["csg", "rect", "dp"])
    ap.add_argument("--trackers", default="", help="comma-separated trackers run one after another (overrides --tracker)")
    ap.add_argument("--mode", default="event", choices=["event", "history"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32"])
    ap.add_argument("--particles", type=int, default=3_000_000)
    ap.add_argument("--launches", type=int, default=1)
    ap.add_argument("--queue-depth", type=int, default=512)
    ap.add_argument("--sort-interval", type=int, default=0)
    ap.add_argument("--members", type=int, default=8)
    ap.add_argument("--chunk", type=int, default=4096)
    ap.add_argument("--batch-tracker", default="auto", choices=["auto", "csg"])
    ap.add_argument("--rays", type=int, default=1 << 18)
    args = ap.parse_args()
    dev = torch.device("cuda", 0)
    if args.workload == "batch":
        run_batch(dev, args)
        return
    if args.workload == "transmission":
        run_transmission(dev, args)
        return
    desc = I.config2() if args.workload == "core" else I.config3()
    g = N.Geometry(I.to_json(desc), device=dev)
    trk = {"csg": N.TRACKER_CSG, "rect": N.TRACKER_RECT, "dp": N.TRACKER_DP}
    names = args.trackers.split(",") if args.trackers else [args.tracker]
    n = args.particles
    for name in names:
        opts = N.default_opts(tracker=trk[name], mode=N.MODE_EVENT if args.mode == "event" else N.MODE_HISTORY,
                              precision=N.FP64 if args.precision == "fp64" else N.FP32_LOCAL,
                              seed=1, p_absorb=0.25, queue_depth=args.queue_depth, sort_interval=args.sort_interval)
        run_case(g, dev, n, opts, args, name)


def run_case(g, dev, n, opts, args, name):
    parts = torch.empty(g.particle_bytes(n), dtype=torch.uint8, device=dev)
    tally = torch.zeros(g.n_inst, dtype=torch.int64, device=dev)
    cnt = torch.zeros(N.NCOUNTERS, dtype=torch.int64, device=dev)
    wb = g.work_bytes(n, opts)
    work = torch.empty(wb + 256, dtype=torch.uint8, device=dev) if wb else None
    stream = torch.cuda.current_stream()
    out = []
    for _ in range(args.launches):
        g.source_init(n, seed=1, out=parts)
        cnt.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        g.run_histories(parts, n, tally=tally, counters=cnt, opts=opts, work=work)
        b.record(stream)
        torch.cuda.synchronize()
        c = cnt.cpu()
        seg = int(c[0])
        ms = a.elapsed_time(b)
        out.append({"segments": seg, "ms": ms, "segments_per_s": seg / (ms / 1e3),
                    "redone_in_fp64": int(c[N.K["close_calls"]]) / max(1, seg)})
    print(json.dumps({"workload": args.workload, "tracker": name, "mode": args.mode, "precision": args.precision,
                      "particles": n, "sort_interval": args.sort_interval, "queue_depth": args.queue_depth,
                      "launches": out}), flush=True)


def run_batch(dev, args):
    members = I.config4()[: args.members]
    geoms = [N.Geometry(I.to_json(d), device=dev) for d, _ in members]
    counts = [c for _, c in members]
    parts = [g.source_init(c, seed=1) for g, c in zip(geoms, counts)]
    b = N.Batch(geoms, parts, counts, tracker=N.TRACKER_CSG if args.batch_tracker == "csg" else N.TRACKER_AUTO)
    b.upload(args.chunk)
    opts = N.default_opts(seed=1, p_absorb=0.25, queue_depth=args.queue_depth,
                          mode=N.MODE_EVENT if args.mode == "event" else N.MODE_HISTORY,
                          precision=N.FP64 if args.precision == "fp64" else N.FP32_LOCAL)
    stream = torch.cuda.current_stream()
    out = []
    for _ in range(args.launches):
        b.zero()
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        b.run(opts)
        e.record(stream)
        torch.cuda.synchronize()
        seg = int(b.counters.cpu().numpy().view(np.uint64).reshape(-1, N.NCOUNTERS)[:, 0].sum())
        ms = a.elapsed_time(e)
        out.append({"segments": seg, "ms": ms, "segments_per_s": seg / (ms / 1e3)})
    print(json.dumps({"workload": "batch", "members": len(geoms), "particles": sum(counts), "mode": args.mode,
                      "precision": args.precision, "chunk": args.chunk, "queue_depth": args.queue_depth,
                      "batch_tracker": args.batch_tracker, "launches": out}), flush=True)


def run_transmission(dev, args):
    desc, rays = I.config5(n_rays=args.rays)
    g = N.Geometry(I.to_json(desc), device=dev)
    R = torch.from_numpy(rays.packed()).to(dev)
    sigma = torch.tensor(desc["sigma"], dtype=torch.float64, device=dev)
    gT = torch.ones(R.shape[0], dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    out = []
    for _ in range(args.launches):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ev[0].record(stream)
        g.transmission_fwd(R, sigma, lens=False)
        ev[1].record(stream)
        g.transmission_bwd(R, sigma, 1.26, gT)
        ev[2].record(stream)
        torch.cuda.synchronize()
        out.append({"fwd_ms": ev[0].elapsed_time(ev[1]), "bwd_ms": ev[1].elapsed_time(ev[2])})
    print(json.dumps({"workload": "transmission", "rays": int(R.shape[0]), "launches": out}), flush=True)


if __name__ == "__main__":
    main()
