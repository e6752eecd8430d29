"""One run_histories launch on a reduced-size workload, for profilers.

The full benchmark holds ~1 GB on the device and launches many kernels; a
profiler that replays each captured launch dozens of times wants one short
launch instead.  This runs source_init and then `--launches` run_histories
launches of one (tracker, mode, precision) on the three-level nested core
(15x15 assemblies of 17x17 pins, the benchmark's geometry) with a particle
count of the caller's choosing (default 3e6: 180 MB of particle state, more
than the 129 MB L2, so DRAM counters still mean something).

  python -m paper_2406_13849_gb300.profile_case [--tracker csg|rect|dp]
      [--mode event|history] [--precision fp64|fp32] [--particles N] [--launches L]

Prints one line with segments, kernel milliseconds and segments/s per launch
(CUDA events; meaningless under a profiler).
"""
from __future__ import annotations

import argparse
import json

import torch

from . import inputs as I
from . import native as N


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--tracker", default="csg", choices=["csg", "rect", "dp"])
    ap.add_argument("--trackers", default="", help="comma-separated trackers run one after another (overrides --tracker)")
    ap.add_argument("--mode", default="event", choices=["event", "history"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32"])
    ap.add_argument("--particles", type=int, default=3_000_000)
    ap.add_argument("--launches", type=int, default=1)
    ap.add_argument("--queue-depth", type=int, default=512)
    args = ap.parse_args()
    dev = torch.device("cuda", 0)
    g = N.Geometry(I.to_json(I.config2()), device=dev)
    trk = {"csg": N.TRACKER_CSG, "rect": N.TRACKER_RECT, "dp": N.TRACKER_DP}
    names = args.trackers.split(",") if args.trackers else [args.tracker]
    n = args.particles
    for name in names:
        opts = N.default_opts(tracker=trk[name], mode=N.MODE_EVENT if args.mode == "event" else N.MODE_HISTORY,
                              precision=N.FP64 if args.precision == "fp64" else N.FP32_LOCAL,
                              seed=1, p_absorb=0.25, queue_depth=args.queue_depth)
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
        seg = int(cnt.cpu()[0])
        ms = a.elapsed_time(b)
        out.append({"segments": seg, "ms": ms, "segments_per_s": seg / (ms / 1e3)})
    print(json.dumps({"tracker": name, "mode": args.mode, "precision": args.precision,
                      "particles": n, "launches": out}), flush=True)


if __name__ == "__main__":
    main()
