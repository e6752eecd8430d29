"""Algorithmic FP64 operation counts per unit of work, from the counting
build of the oracle (test infrastructure, like the rest of this package).

The counting build evaluates the oracle's arithmetic on a scalar type that
counts each FP64 add/sub, mul, div and sqrt once (comparisons apart), in
array-tracker mode, the fewest operations the method needs.  The figures are
the numerators of the benchmark's rooflines:

  tracking, configuration 2 (the main workload)    operations per segment
  tracking, configuration 4 (the 64-geometry batch) operations per segment
      of the array-lattice members, estimated per member on a sample and
      weighted by the member's population times its segments per particle.
      The hex members are reported apart and not used: the oracle scans a
      hex lattice's pseudo-array linearly, several times the operations of
      the closed-form element search, so its count is no minimum there; the
      array members' figure, applied to every segment, undercounts them.
  transmission, configuration 5                     operations per ray of the
      segment arithmetic (the oracle's derivative terms are plain doubles,
      not counted); the backward kernel recomputes the segments, so this is
      a lower bound of its work too

    python -m oracle.flop_counts        (prints one JSON object)
"""
from __future__ import annotations

import json
import sys

import numpy as np

import oracle as O
from paper_2406_13849_gb300 import inputs as I

SEED = 1
P_ABSORB = 0.25


def _ops(fc: dict) -> int:
    return fc["add"] + fc["mul"] + fc["div"] + fc["sqrt"]


def per_segment(desc: dict, particles: int) -> tuple[float, float]:
    """(operations per segment, segments per particle) on `particles`
    histories of the description."""
    g = O.Geometry(I.to_json(desc), O.MODE_RECT, counting=True)
    g.flop_counts(reset=True)
    r = g.run(particles, SEED, P_ABSORB, threads=1, records=False)
    fc = g.flop_counts()
    seg = float(r["counters"][O.K_SEGMENTS])
    return _ops(fc) / seg, seg / particles


def batch_per_segment(particles_per_member: int) -> dict:
    """Operations per segment of the batch's array-lattice and hex-lattice
    members (population-weighted)."""
    acc = {"rect": [0.0, 0.0], "hex": [0.0, 0.0]}
    for desc, count in I.config4():
        f, s = per_segment(desc, particles_per_member)
        kind = "hex" if any(u.get("type") == "hex" for u in desc["universes"]) else "rect"
        acc[kind][0] += f * s * count
        acc[kind][1] += s * count
    return {k: (v[0] / v[1] if v[1] else None) for k, v in acc.items()}


def transmission_per_ray(rays: int) -> float:
    desc, rs = I.config5(n_rays=rays)
    g = O.Geometry(I.to_json(desc), O.MODE_RECT, counting=True)
    sigma = np.asarray(desc["sigma"], np.float64)
    g.flop_counts(reset=True)
    g.transmission(rs.packed(), sigma, 1.26, grad=True)
    return _ops(g.flop_counts()) / rays


def main() -> None:
    c2, spp = per_segment(I.config2(), 2000)
    c4 = batch_per_segment(200)
    t = transmission_per_ray(512)
    json.dump({"config2_ops_per_segment": c2, "config2_segments_per_particle": spp,
               "config4_ops_per_segment_array_members": c4["rect"],
               "config4_ops_per_segment_hex_members_linear_scan": c4["hex"],
               "config5_ops_per_ray": t,
               "sample": {"config2_particles": 2000, "config4_particles_per_member": 200, "config5_rays": 512,
                          "seed": SEED, "p_absorb": P_ABSORB}}, sys.stdout, indent=1)
    print()


if __name__ == "__main__":
    main()
