"""Comparison of the CUDA path's fast build with the oracle under the
near-surface rule (test infrastructure, like the rest of this package).

The fast build contracts multiply-adds and takes the collision distance as
tau times a stored 1/Sigma, so its numbers differ from the oracle's FP64
evaluation by a few ulp per operation.  Such a difference changes a decision
only where the decision is taken within rounding distance of a surface; it
changes lengths by the rounding error propagated along the history.

Propagation.  Directions never depend on positions (collisions draw them
from the random numbers; crossings keep them; reflections flip a component
exactly), so the errors of a history are those of its position e and of its
tau, carried forward linearly to first order:
  crossing a surface with normal n (c = n . Omega): the length changes by
    dl = -(n . e) / c, the position error becomes e + dl Omega (projected
    onto the surface along Omega), tau's error loses Sigma dl;
  collision: dl = (tau error) / Sigma, the position error gains dl Omega,
    and the new tau is drawn afresh (no error).
Each segment adds fresh rounding of LOCAL_ULPS ulps of the coordinates' size
to the position, the length and tau.  The fresh roundings are independent,
so the expected size of the carried error follows from propagating the
covariance of (e, tau error) with these maps along the oracle's own path
(normals from Geometry.clearance, cross sections from the trace).  Its square
root times SAFETY bounds the length and position differences of the rule
below.  (The product of the maps' norms would be a rigorous bound but grows
by the incidence factor at every crossing, past any meaningful size within a
few dozen segments of the pin lattice, although an error along Omega is
absorbed at the next crossing.)

The rule per particle:
  - matched: the same leaf instances, and every segment length within
    max(1e-12 relative to the path's scale, SAFETY x the propagated bound);
  - near-surface: at the first mismatch the oracle shows the decision was
    taken within NEAR = 1e-9 cm of the surface that decided it;
  - drift: the decision's distance to that surface is above NEAR but within
    SAFETY x the propagated position error there (a history whose error has
    grown through many grazing crossings), reported separately;
  - anything else fails.

The deciding surface.  Where the first mismatch is in the cell entered after
segment k-1, ending at P: the nearest surface when the oracle collided at P
(the fast build crossed there), the nearest other than the crossed one when
the oracle crossed at P (the fast build took another surface, or a search
below decided differently), or, when one side collided where the other
crossed, the two events' distance along the ray.  Where the first mismatch is
in a length with the same cell: a cylinder hit or miss close to tangency
(the tangency |b - r| of the cylinders whose closest approach lies on that
segment or the next), or a collision close to a surface (the collision
point's distance to its nearest surface).

Distances are the oracle's global-frame surfaces (Geometry.clearance): |f| /
|grad f| for planes and |rho - r| for cylinders.
"""
from __future__ import annotations

import numpy as np

NEAR = 1e-9
REL = 1e-12
EPS = 2.0 ** -52
LOCAL_ULPS = 16.0
SAFETY = 10.0
MIN_INCIDENCE = 1e-12


def propagated_bounds(ol, kind, geo, normals):
    """Per segment: the expected size (standard deviation) of the fast
    build's length error, and of its position error at the segment's start,
    from propagating the covariance of (position error, tau error) along the
    oracle's path (see the module docstring)."""
    m = len(ol)
    blen = np.zeros(m)
    bpos = np.zeros(m)
    Cov = np.zeros((4, 4))
    for k in range(m):
        scale = float(np.abs(geo[k, :3]).max() + abs(ol[k]))
        local2 = (LOCAL_ULPS * EPS * max(scale, 1.0)) ** 2
        bpos[k] = np.sqrt(max(np.trace(Cov[:3, :3]), 0.0))
        w = geo[k, 3:6]
        sig = float(geo[k, 6])
        # dl = h . (e, tau error) and the state map A
        h = np.zeros(4)
        A = np.eye(4)
        if kind[k] == 1:
            h[3] = 1.0 / sig if sig > 0 else 0.0
            A[:3, 3] = w * h[3]
            A[3, :] = 0.0
        else:
            n = normals[k]
            c = float(n @ w)
            if abs(c) < MIN_INCIDENCE:
                c = MIN_INCIDENCE if c >= 0 else -MIN_INCIDENCE
            h[:3] = -n / c
            A[:3, :3] += np.outer(w, h[:3])
            A[3, :3] = -sig * h[:3]
        blen[k] = np.sqrt(max(float(h @ Cov @ h), 0.0) + local2)
        Cov = A @ Cov @ A.T + local2 * np.eye(4)
    return blen, bpos


def compare_traces(o, pids, g_inst: np.ndarray, g_len: np.ndarray, seed: int, p_absorb: float, cap: int) -> dict:
    """Classifies traced fast-build histories against the oracle.

    o: oracle Geometry; pids: particle ids; g_inst, g_len: the CUDA path's
    segment log rows for those particles (cap entries each, instance -1 past
    the end).  Returns counts and the per-particle findings."""
    out = {"compared": 0, "matched": 0, "near_surface": [], "drift": [], "failed": [], "segments_compared": 0,
           "max_rel_matched": 0.0, "max_abs_matched": 0.0}
    traces = [o.trace(int(pid), seed, p_absorb, cap=cap, geometry=True) for pid in pids]
    # the normal at every oracle segment's end (one clearance query for all)
    allgeo = [t[4] for t in traces if len(t[1])]
    inc = []
    if allgeo:
        cl = o.clearance(np.concatenate([g[:, :3] for g in allgeo]), np.concatenate([g[:, 3:6] for g in allgeo]),
                         np.concatenate([t[1] for t in traces if len(t[1])]))
        off = 0
        for t in traces:
            inc.append(cl[off: off + len(t[1]), 5:8])
            off += len(t[1])
    pending = []          # (pid, what, query selections, extra margins, position error bound)
    queries = []          # (start xyz, dir, length)

    def q(x, d, length):
        queries.append((np.asarray(x, np.float64), np.asarray(d, np.float64), float(length)))
        return len(queries) - 1

    for row, (pid, tr) in enumerate(zip(pids, traces)):
        oi, ol, ok, st, geo = tr
        gi = g_inst[row]
        gl = g_len[row]
        kg = int((gi >= 0).sum())
        ko = len(oi)
        m = min(ko, kg)
        out["compared"] += 1
        normals = inc[row] if ko else np.zeros((0, 3))
        blen, bpos = propagated_bounds(ol, ok, geo, normals)
        scale = np.abs(ol[:m]) + np.abs(geo[:m, :3]).max(axis=1)
        bar = np.maximum(REL * scale, SAFETY * blen[:m])
        dl = np.abs(gl[:m] - ol[:m])
        bad = (gi[:m] != oi[:m]) | (dl > bar)
        j = int(np.argmax(bad)) if bad.any() else (m if ko != kg else -1)
        if j < 0:
            out["matched"] += 1
            out["segments_compared"] += m
            if m:
                out["max_rel_matched"] = max(out["max_rel_matched"], float((dl / scale).max()))
                out["max_abs_matched"] = max(out["max_abs_matched"], float(dl.max()))
            continue
        epos = SAFETY * (bpos[min(j, ko - 1)] if ko else 0.0)
        inst_mismatch = j >= m or gi[j] != oi[j]
        if inst_mismatch:
            if j == 0:
                # the birth cell: find_cell at the birth point
                pending.append((int(pid), "birth cell", [("c1", q(geo[0, :3], geo[0, 3:6], 0.0))], [], 0.0))
                continue
            start, d = geo[j - 1, :3], geo[j - 1, 3:6]
            P = start + ol[j - 1] * d
            oracle_collided = ok[j - 1] == 1
            sel = [("c1" if oracle_collided else "c2", q(P, d, 0.0))]
            extra = []
            o_moved = j < ko and oi[j] != oi[j - 1]
            g_moved = j < kg and gi[j] != gi[j - 1]
            if not (o_moved and g_moved):
                # one side stayed in its cell (collision, reflection) or ended
                # where the other crossed: the two events' distance along the ray
                extra.append(float(abs(ol[j - 1] - gl[j - 1])))
            epos = SAFETY * (bpos[j - 1] + blen[j - 1])
            pending.append((int(pid), "cell after segment %d" % (j - 1), sel, extra, epos))
        else:
            X, D = geo[j, :3], geo[j, 3:6]
            Lo, Lg = float(ol[j]), float(gl[j])
            sel = [("tang", q(X, D, max(Lo, Lg) + 1e-4))]
            if j + 1 < ko and ok[j] == 0:
                sel.append(("tang", q(geo[j + 1, :3], geo[j + 1, 3:6], ol[j + 1])))
            if j + 1 < kg:
                sel.append(("tang", q(X + Lg * D, D, gl[j + 1])))
            if ok[j] == 1:
                sel.append(("c3", q(X, D, Lo)))
            pending.append((int(pid), "length of segment %d" % j, sel, [], epos))
    if queries:
        xyz = np.array([x for x, _, _ in queries])
        dirs = np.array([d for _, d, _ in queries])
        lens = np.array([ln for _, _, ln in queries])
        cl = o.clearance(xyz, dirs, lens)
        col = {"c1": 0, "c2": 1, "c3": 2, "tang": 4}
        for pid, what, sel, extra, epos in pending:
            margin = min([float(cl[qi, col[k]]) for k, qi in sel] + extra)
            rec = {"pid": pid, "at": what, "margin_cm": margin, "position_error_bound_cm": epos}
            if margin < NEAR:
                out["near_surface"].append(rec)
            elif margin <= epos:
                out["drift"].append(rec)
            else:
                out["failed"].append(rec)
    return out


def classify_distances(o, xyz, dirs, d_oracle, lev_oracle, d_gpu, lev_gpu) -> dict:
    """Per-point distance_to_surface of the fast build against the oracle:
    distances within 1e-12 relative to the coordinates' size (max(1 cm, d,
    the point's largest coordinate): a distance computed from coordinates of
    size |x| cannot be more accurate than their rounding, ~1e-16 |x|, times
    the formula's conditioning) and the same winning level, or else the
    oracle shows the distance is decided near a surface:
    the start point lies within NEAR of a surface (its distance to it is then
    a difference of nearly equal squares, as ill-conditioned as a decision
    there), the hit point d_oracle along the ray lies within NEAR of a second
    surface (a near-tie), or the ray passes within NEAR of a cylinder's
    tangency on its way there.  The start point carries no propagated error,
    so no drift is allowed here."""
    inside = np.isfinite(d_oracle) | np.isfinite(d_gpu)
    rel = np.zeros(len(d_oracle))
    both = np.isfinite(d_oracle) & np.isfinite(d_gpu)
    scale = np.maximum(np.maximum(1.0, np.abs(d_oracle)), np.abs(xyz).max(axis=1)) if len(xyz) else np.ones(0)
    rel[both] = np.abs(d_gpu[both] - d_oracle[both]) / scale[both]
    bad = inside & ((~both) | (rel > REL) | (lev_gpu != lev_oracle))
    idx = np.nonzero(bad)[0]
    res = {"points": int(inside.sum()), "outside_bar": len(idx), "near": [], "failed": [],
           "max_rel_within_bar": float(rel[inside & ~bad].max()) if (inside & ~bad).any() else 0.0}
    if len(idx):
        far = np.where(np.isfinite(d_oracle[idx]), d_oracle[idx], 0.0)
        far_g = np.where(np.isfinite(d_gpu[idx]), d_gpu[idx], 0.0)
        length = np.maximum(far, far_g) + 1e-4
        cl = o.clearance(xyz[idx], dirs[idx], length)
        hit = xyz[idx] + far[:, None] * dirs[idx]
        cl_hit = o.clearance(hit, dirs[idx], np.zeros(len(idx)))
        for k, i in enumerate(idx):
            margin = min(float(cl[k, 0]), float(cl_hit[k, 1]), float(cl[k, 4]))
            rec = {"point": int(i), "margin_cm": margin, "rel": float(rel[i]),
                   "level": (int(lev_oracle[i]), int(lev_gpu[i]))}
            (res["near"] if margin < NEAR else res["failed"]).append(rec)
    return res
