"""The fast build's event kernel (the benchmarked one: FMA contraction, the
collision distance from a stored 1/Sigma, queue depth 512, the launch shape
run_histories uses) against the oracle under the near-surface rule.

Per particle (oracle.compare): instance sequences equal and segment lengths
within 1e-12 relative to the path's scale, or, at the first mismatch, the
oracle shows the decision there was taken within 1e-9 cm of a surface; such
particles are counted and left out; anything else fails.  Per point,
distance_to_surface within 1e-12 relative with the same winning level, or a
near-tie / near-tangency the oracle confirms.

The traced kernel is the benchmarked kernel's template with the segment log
switched on; its tallies are checked bit for bit against the untraced
launch, so the two compute the same segments.
"""
import numpy as np
import pytest
import torch

import oracle as O
from oracle import compare as C
from paper_2406_13849_gb300 import inputs as I
from paper_2406_13849_gb300 import native as N

pytestmark = pytest.mark.gpu

SEED = 1
QUEUE_DEPTH = 512

CASES = {
    "c1": (I.config1(), 0.3, 10_007),
    "small_core": (I.small_core(), 0.25, 6_001),
    "c3": (I.config3(), 0.25, 1_201),
}


def _u64(t):
    return t.cpu().numpy().view(np.uint64)


def _event_opts(tracker, pa, **kw):
    return N.default_opts(tracker=tracker, mode=N.MODE_EVENT, queue_depth=QUEUE_DEPTH, p_absorb=pa, seed=SEED, **kw)


def _traced(g, n, pa, tracker, cap, rows=None):
    """Segment logs of the event kernel for the particles in `rows` (all
    when None), after checking that the traced launch computes what the
    benchmarked one does."""
    parts = g.source_init(n, seed=SEED)
    opts = _event_opts(tracker, pa)
    inst, ln, tally, cnt = g.trace(parts, n, cap, opts=opts)
    # the benchmarked launch (no segment log) on the same particles
    t0, c0, _ = g.run_histories(parts, n, opts=opts)
    torch.cuda.synchronize()
    assert np.array_equal(_u64(tally), _u64(t0)), "traced and benchmarked event kernels differ"
    assert np.array_equal(_u64(cnt)[:11], _u64(c0)[:11])
    if rows is not None:
        r = torch.from_numpy(np.asarray(rows, np.int64)).cuda()
        inst, ln = inst[r], ln[r]
    return inst.cpu().numpy(), ln.cpu().numpy(), _u64(cnt)


def _report(name, res):
    print(f"\n{name}: compared {res['compared']}, matched {res['matched']}, "
          f"near-surface {len(res['near_surface'])}, drift {len(res['drift'])}, failed {len(res['failed'])}, "
          f"segments {res['segments_compared']}, max rel (matched) {res['max_rel_matched']:.3g}, "
          f"max abs (matched) {res['max_abs_matched']:.3g}")
    for r in res["near_surface"][:10] + res["drift"][:10]:
        print("  near/drift:", r)
    for r in res["failed"][:10]:
        print("  FAILED:", r)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("tracker,mode", [(N.TRACKER_CSG, O.MODE_CSG), (N.TRACKER_RECT, O.MODE_RECT)])
def test_fast_event_kernel_near_surface_rule(name, tracker, mode):
    desc, pa, n = CASES[name]
    g = N.Geometry(I.to_json(desc), exact=False)
    assert g.lib.trk_exact_build() == 0
    cap = 1024
    inst, ln, cnt = _traced(g, n, pa, tracker, cap)
    assert cnt[N.K["lost"]] == 0 and cnt[N.K["status"]] == 0
    o = O.Geometry(I.to_json(desc), mode)
    res = C.compare_traces(o, np.arange(n), inst, ln, SEED, pa, cap)
    _report(f"{name} tracker {tracker}", res)
    assert res["compared"] == n
    assert not res["failed"], res["failed"][:5]
    # divergences are rare: a decision within rounding distance of a surface
    assert len(res["near_surface"]) + len(res["drift"]) <= max(3, n // 500)


def test_fast_event_kernel_config2_full_size_sampled():
    # the benchmark's workload and launch: 1e7 particles, BVH-CSG, event
    # kernel at queue depth 512; 200 particles compared one by one
    desc = I.config2()
    n, pa, cap = 10_000_000, 0.25, 96
    g = N.Geometry(I.to_json(desc), exact=False)
    ids = np.random.default_rng(17).choice(n, 200, replace=False)
    inst, ln, cnt = _traced(g, n, pa, N.TRACKER_CSG, cap, rows=ids)
    assert cnt[N.K["lost"]] == 0 and cnt[N.K["status"]] == 0
    o = O.Geometry(I.to_json(desc), O.MODE_CSG)
    res = C.compare_traces(o, ids, inst, ln, SEED, pa, cap)
    _report("c2 sampled", res)
    assert not res["failed"], res["failed"][:5]
    assert len(res["near_surface"]) + len(res["drift"]) <= 3


@pytest.mark.parametrize("name", ["c1", "c2", "small_hex_core"])
@pytest.mark.parametrize("tracker,mode", [(N.TRACKER_CSG, O.MODE_CSG), (N.TRACKER_RECT, O.MODE_RECT)])
def test_fast_distance_near_surface_rule(name, tracker, mode):
    desc = {"c1": I.config1(), "c2": I.config2(), "small_hex_core": I.small_hex_core()}[name]
    rng = np.random.default_rng(6)
    lo, hi = np.array(desc["source_box"][:3]), np.array(desc["source_box"][3:])
    n = 20_011
    xyz = lo + rng.uniform(size=(n, 3)) * (hi - lo)
    w = rng.normal(size=(n, 3))
    w /= np.linalg.norm(w, axis=1)[:, None]
    o = O.Geometry(I.to_json(desc), mode)
    od, ol, oi = o.distance(xyz, w)
    g = N.Geometry(I.to_json(desc), exact=False)
    d, lev, inst = g.distance_to_surface(torch.from_numpy(xyz).cuda(), torch.from_numpy(w).cuda(), tracker=tracker)
    gd, gl, gi = d.cpu().numpy(), lev.cpu().numpy(), inst.cpu().numpy()
    # the point's cell: find_cell is exact integer/sign work; a point within
    # rounding of a surface may land on either side, and must then be near it
    diff = np.nonzero(gi != oi)[0]
    if len(diff):
        cl = o.clearance(xyz[diff], w[diff], np.zeros(len(diff)))
        assert (cl[:, 0] < C.NEAR).all(), cl[:, 0]
    same = gi == oi
    res = C.classify_distances(o, xyz[same], w[same], od[same], ol[same], gd[same], gl[same])
    print(f"\n{name} tracker {tracker}: points {res['points']}, outside the bar {res['outside_bar']}, "
          f"near {len(res['near'])}, failed {len(res['failed'])}, max rel within bar {res['max_rel_within_bar']:.3g}, "
          f"cell differs {len(diff)}")
    for r in res["failed"][:10]:
        print("  FAILED:", r)
    assert not res["failed"], res["failed"][:5]
    assert np.isnan(gd[oi < 0]).all()


@pytest.mark.parametrize("name", ["c1", "c2", "c3"])
@pytest.mark.parametrize("tracker,mode", [(N.TRACKER_CSG, O.MODE_CSG), (N.TRACKER_RECT, O.MODE_RECT)])
def test_fp32_local_distance_per_point(name, tracker, mode):
    # FP32-local precision (fast build): every distance the FP32-local flight
    # takes is within 1e-5 relative (to max(1 cm, d)) of the oracle's FP64
    # distance with the same winning level; the distances it redoes in FP64
    # (close calls, ill-conditioned cylinders) meet the FP64 rule above
    desc = {"c1": I.config1(), "c2": I.config2(), "c3": I.config3()}[name]
    rng = np.random.default_rng(9)
    lo, hi = np.array(desc["source_box"][:3]), np.array(desc["source_box"][3:])
    n = 40_009
    xyz = lo + rng.uniform(size=(n, 3)) * (hi - lo)
    w = rng.normal(size=(n, 3))
    w /= np.linalg.norm(w, axis=1)[:, None]
    o = O.Geometry(I.to_json(desc), mode)
    od, ol, oi = o.distance(xyz, w)
    g = N.Geometry(I.to_json(desc), exact=False)
    d, lev, inst, close = g.distance_to_surface(torch.from_numpy(xyz).cuda(), torch.from_numpy(w).cuda(),
                                                tracker=tracker, precision=N.FP32_LOCAL, with_close=True)
    gd, gl, gi, cc = d.cpu().numpy(), lev.cpu().numpy(), inst.cpu().numpy(), close.cpu().numpy().astype(bool)
    # find_cell (FP64 in both precisions): a point within rounding of a
    # surface may land on either side, and must then be near it
    diff = np.nonzero(gi != oi)[0]
    if len(diff):
        cl = o.clearance(xyz[diff], w[diff], np.zeros(len(diff)))
        assert (cl[:, 0] < C.NEAR).all(), (diff[:5], cl[:5, 0])
    inside = (oi >= 0) & (gi == oi)
    f32 = inside & ~cc & np.isfinite(od)
    rel = np.abs(gd[f32] - od[f32]) / np.maximum(1.0, np.abs(od[f32]))
    lev_ok = gl[f32] == ol[f32]
    print(f"\n{name} tracker {tracker}: points {inside.sum()}, FP32 {f32.sum()}, redone in FP64 {(inside & cc).sum()}, "
          f"max rel {rel.max():.3g}, p99.9 {np.quantile(rel, 0.999):.3g}, level differs {(~lev_ok).sum()}, "
          f"cell differs {len(diff)}")
    assert (rel <= 1e-5).all() and lev_ok.all()
    # the redone ones: the FP64 rule
    red = inside & cc
    res = C.classify_distances(o, xyz[red], w[red], od[red], ol[red], gd[red], gl[red])
    assert not res["failed"], res["failed"][:5]
    assert (inside & cc).mean() < 0.05
