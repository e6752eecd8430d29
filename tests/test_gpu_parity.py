"""GPU parity: the CUDA path (through the C-ABI) against the CPU oracle.

Bars:
  --fmad=false build: bit-exact per particle (digest of the instance and
    segment-length sequence, segment count, status), bit-exact u64 tallies
    and counters, bit-exact birth states and find_cell.
  fast build: identical instance sequences for all but a tiny fraction of
    particles (a near-surface decision can go either way under contraction),
    segment lengths within 1e-12 relative plus 1e-11 cm for 99% of histories
    and within 1e-6 cm for all (near-tangent hits are ill-conditioned), totals
    within 1e-9 relative.
Sizes: several thousand histories per case (many blocks plus a ragged tail),
plus sampled particles of the full-size workloads in the benchmark's launch
configuration.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle as O
from paper_2406_13849_gb300 import inputs as I
from paper_2406_13849_gb300 import native as N

pytestmark = pytest.mark.gpu

SEED = 1

CASES = {
    "c1": (I.config1(), 0.3, 10_007),
    "small_core": (I.small_core(), 0.25, 6_001),
    "c2": (I.config2(), 0.25, 3_001),
    "tiny3": (I.random_tiny(3), 0.3, 4_099),
    "tiny8": (I.random_tiny(8), 0.3, 4_099),
    "pin_vacuum": (I.single_pin(bc="vacuum"), 0.3, 2_053),
}
HEX_CASES = {
    "c3": (I.config3(), 0.25, 1_201),
    "small_hex_core": (I.small_hex_core(), 0.25, 3_001),
    "hex_rot": (I.small_hex(rings=3, rot30=True), 0.3, 2_003),
}


def _oracle(desc, mode):
    return O.Geometry(I.to_json(desc), mode)


def _gpu(desc, exact):
    return N.Geometry(I.to_json(desc), exact=exact)


def _u64(t):
    return t.cpu().numpy().view(np.uint64)


def _run_gpu(g, n, pa, tracker, records=True, **kw):
    parts = g.source_init(n, seed=SEED)
    tally, cnt, rec = g.run_histories(parts, n, records=records, tracker=tracker, p_absorb=pa, seed=SEED, **kw)
    torch.cuda.synchronize()
    return parts, _u64(tally), _u64(cnt), rec


# ---------------------------------------------------------------------------
# birth states and find_cell
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name", list(CASES) + list(HEX_CASES))
def test_source_bit_exact(name):
    desc, pa, n = {**CASES, **HEX_CASES}[name]
    o = _oracle(desc, O.MODE_CSG)
    ref, st = o.source(n, SEED)
    g = _gpu(desc, exact=True)
    buf = g.source_init(n, seed=SEED)
    d, gst = N.Geometry.particles_as_arrays(buf, n)
    got = d.cpu().numpy().T
    assert np.array_equal(gst.cpu().numpy(), st)
    assert np.array_equal(got.view(np.uint64), ref.view(np.uint64))


@pytest.mark.parametrize("name", list(CASES) + list(HEX_CASES))
def test_find_cell_exact(name):
    desc, _, _ = {**CASES, **HEX_CASES}[name]
    lo, hi = np.array(desc["source_box"][:3]), np.array(desc["source_box"][3:])
    pts = lo + np.random.default_rng(3).uniform(0, 1, (20_000, 3)) * (hi - lo)
    g = _gpu(desc, exact=True)
    xyz = torch.from_numpy(pts).cuda()
    trackers = [(N.TRACKER_CSG, O.MODE_CSG), (N.TRACKER_RECT, O.MODE_RECT)]
    for tr, mode in trackers:
        ref = _oracle(desc, mode).find_cell(pts)
        got = g.find_cell(xyz, tracker=tr).cpu().numpy()
        assert np.array_equal(got, ref), (name, tr)


# ---------------------------------------------------------------------------
# histories: exact build, bit for bit
# ---------------------------------------------------------------------------

def _compare_exact(desc, pa, n, tracker, mode, **kw):
    o = _oracle(desc, mode).run(n, SEED, pa, threads=8, **{k: v for k, v in kw.items()})
    g = _gpu(desc, exact=True)
    gkw = {}
    if "max_segments" in kw:
        gkw["max_segments"] = kw["max_segments"]
    if "max_path" in kw:
        gkw["max_path"] = kw["max_path"]
    _, tally, cnt, rec = _run_gpu(g, n, pa, tracker, **gkw)
    h, nseg, st = N.unpack_records(rec)
    assert np.array_equal(st, o["status"])
    assert np.array_equal(nseg, o["nseg"])
    assert np.array_equal(h, o["hash"])
    assert np.array_equal(tally, o["tally"])
    assert np.array_equal(cnt[:10], o["counters"][:10])
    assert cnt[N.K["status"]] == 0
    return o


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("tracker,mode", [(N.TRACKER_RECT, O.MODE_RECT), (N.TRACKER_CSG, O.MODE_CSG)])
def test_histories_bit_exact(name, tracker, mode):
    desc, pa, n = CASES[name]
    o = _compare_exact(desc, pa, n, tracker, mode)
    assert o["counters"][O.K_SEGMENTS] > n


@pytest.mark.parametrize("name", list(HEX_CASES))
@pytest.mark.parametrize("tracker,mode", [(N.TRACKER_RECT, O.MODE_RECT), (N.TRACKER_CSG, O.MODE_CSG)])
def test_histories_bit_exact_hex(name, tracker, mode):
    # the array tracker on hex arrays: closed-form element search, checked
    # against the oracle's pseudo-array scan
    desc, pa, n = HEX_CASES[name]
    _compare_exact(desc, pa, n, tracker, mode)


@pytest.mark.parametrize("name", list(HEX_CASES))
def test_hex_array_and_csg_trackers_identical(name):
    # same histories from the closed-form hex search and the BVH search,
    # history and event kernels (exact build)
    desc, pa, n = HEX_CASES[name]
    g = _gpu(desc, exact=True)
    res = []
    for tr in (N.TRACKER_RECT, N.TRACKER_CSG):
        for mode in (N.MODE_HISTORY, N.MODE_EVENT):
            _, tally, cnt, rec = _run_gpu(g, n, pa, tr, mode=mode)
            res.append((tally, _u64(rec)))
    for t, r in res[1:]:
        assert np.array_equal(t, res[0][0]) and np.array_equal(r, res[0][1])


def test_hex_find_points_on_faces():
    # points on element faces and vertices of a hex lattice (the + side of a
    # face holds it): the closed-form search against the oracle's scan
    desc = I.small_hex(rings=3, rot30=True)
    g = _gpu(desc, exact=True)
    hp = 0.5
    pts = []
    rng = np.random.default_rng(11)
    a1, a2, nrm = I._hex_frame(1.0, rot30=True)
    for q in range(-3, 4):
        for r in range(-3, 4):
            cx, cy = q * a1[0] + r * a2[0], q * a1[1] + r * a2[1]
            for k in range(3):
                for sgn in (-1, 1):
                    nx, ny = nrm[k]
                    t = rng.uniform(-0.2, 0.2)
                    # face midpoint plus a shift along the face
                    pts.append([cx + sgn * hp * nx - t * ny, cy + sgn * hp * ny + t * nx, 1.0])
    pts = np.array(pts)
    ref = _oracle(desc, O.MODE_RECT).find_cell(pts)
    got = g.find_cell(torch.from_numpy(pts).cuda(), tracker=N.TRACKER_RECT).cpu().numpy()
    assert np.array_equal(got, ref)


def test_segment_cap_and_cutoff_exact():
    desc = I.config1()
    o = _compare_exact(desc, 0.0, 1_000, N.TRACKER_RECT, O.MODE_RECT, max_segments=7)
    assert np.all(o["status"] == O.P_MAXSEG)
    d0 = I.config1(sigma=(0.0, 0.0, 0.0))
    o = _compare_exact(d0, 0.3, 1_000, N.TRACKER_CSG, O.MODE_CSG, max_path=150.0)
    assert np.all(o["status"] == O.P_CUTOFF)


def test_rect_and_csg_trackers_identical_on_gpu():
    for desc, pa, n in (CASES["c1"], CASES["small_core"]):
        g = _gpu(desc, exact=False)
        ra = _run_gpu(g, n, pa, N.TRACKER_RECT)
        rb = _run_gpu(g, n, pa, N.TRACKER_CSG)
        assert np.array_equal(ra[1], rb[1])
        assert np.array_equal(_u64(ra[3]), _u64(rb[3]))


# ---------------------------------------------------------------------------
# histories: fast build, within tolerance
# ---------------------------------------------------------------------------

def _traces_oracle(o, ids, pa):
    out = {}
    for i in ids:
        inst, ln, kind, st = o.trace(int(i), SEED, pa)
        out[int(i)] = (inst, ln)
    return out


@pytest.mark.parametrize("name", ["c1", "small_core", "tiny3"])
@pytest.mark.parametrize("tracker,mode", [(N.TRACKER_RECT, O.MODE_RECT), (N.TRACKER_CSG, O.MODE_CSG)])
def test_histories_fast_within_tolerance(name, tracker, mode):
    desc, pa, n = CASES[name]
    n = min(n, 3000)
    o = _oracle(desc, mode)
    ref = o.run(n, SEED, pa, threads=8)
    g = _gpu(desc, exact=False)
    parts = g.source_init(n, seed=SEED)
    cap = 4096
    inst, ln, tally, cnt = g.trace(parts, n, cap, tracker=tracker, p_absorb=pa, seed=SEED)
    inst, ln = inst.cpu().numpy(), ln.cpu().numpy()
    mism = 0
    loose = 0
    for i in range(n):
        oi, ol, _, _ = o.trace(i, SEED, pa, cap=cap)
        k = len(oi)
        gi, gl = inst[i], ln[i]
        gk = int((gi >= 0).sum())
        if gk != k or not np.array_equal(gi[:k], oi):
            mism += 1
            continue
        # Contraction changes each rounding by ~1 ulp of coordinates up to ~20 cm;
        # a well-conditioned history stays within 1e-12 relative + 1e-11 cm.  A
        # near-tangent cylinder hit amplifies position differences by
        # 1/sqrt(disc), so a few histories drift further; every history must
        # stay within 1e-6 cm.
        err = np.abs(gl[:k] - ol)
        assert err.max() <= 1e-6, (i, err.max())
        if (err - (1e-12 * np.abs(ol) + 1e-11)).max() > 0:
            loose += 1
    assert mism <= max(2, n // 1000), mism
    assert loose <= n // 100, loose
    t_ref = ref["tally"].astype(np.float64).sum()
    t_got = tally.cpu().numpy().view(np.uint64).astype(np.float64).sum()
    assert abs(t_got - t_ref) <= 1e-9 * t_ref + 1e-6 * 2**32 * mism * 100


# ---------------------------------------------------------------------------
# full-size workloads, sampled particles, benchmark launch configuration
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("exact", [True, False])
def test_config2_full_size_sampled(exact):
    desc = I.config2()
    n, pa = 10_000_000, 0.25
    g = _gpu(desc, exact=exact)
    parts = g.source_init(n, seed=SEED)
    tally, cnt, rec = g.run_histories(parts, n, records=True, tracker=N.TRACKER_CSG, p_absorb=pa, seed=SEED)
    torch.cuda.synchronize()
    h, nseg, st = N.unpack_records(rec)
    c = _u64(cnt)
    # properties that hold at any size
    assert c[N.K["lost"]] == 0 and c[N.K["status"]] == 0
    assert c[N.K["absorbed"]] + c[N.K["escaped"]] + c[N.K["maxseg"]] == n
    assert c[N.K["segments"]] == c[N.K["crossings"]] + c[N.K["collisions"]]
    assert nseg.sum() == c[N.K["segments"]]
    # sampled particles one by one in the oracle
    o = _oracle(desc, O.MODE_CSG)
    ids = np.random.default_rng(7).choice(n, 200, replace=False)
    same = 0
    for i in ids:
        r = o.run(1, SEED, pa, first_id=int(i))
        if exact:
            assert r["hash"][0] == h[i] and r["nseg"][0] == nseg[i] and r["status"][0] == st[i], int(i)
        else:
            same += int(r["nseg"][0] == nseg[i] and r["status"][0] == st[i])
    if not exact:
        assert same >= 198


def test_config3_full_size_sampled():
    desc = I.config3()
    n, pa = 10_000_000, 0.25
    g = _gpu(desc, exact=True)
    parts = g.source_init(n, seed=SEED)
    tally, cnt, rec = g.run_histories(parts, n, records=True, tracker=N.TRACKER_CSG, p_absorb=pa, seed=SEED)
    torch.cuda.synchronize()
    h, nseg, st = N.unpack_records(rec)
    c = _u64(cnt)
    assert c[N.K["status"]] == 0
    assert c[N.K["lost"]] <= n * 1e-6
    o = _oracle(desc, O.MODE_CSG)
    for i in np.random.default_rng(8).choice(n, 60, replace=False):
        r = o.run(1, SEED, pa, first_id=int(i))
        assert r["hash"][0] == h[i] and r["nseg"][0] == nseg[i], int(i)


# ---------------------------------------------------------------------------
# edge cases and errors
# ---------------------------------------------------------------------------

def test_edge_cases():
    desc = I.config1()
    g = _gpu(desc, exact=True)
    parts = g.source_init(1, seed=SEED)
    tally, cnt, rec = g.run_histories(parts, 0, records=True)
    assert _u64(cnt).sum() == 0
    o = _oracle(desc, O.MODE_RECT).run(1, SEED, 0.3)
    tally, cnt, rec = g.run_histories(parts, 1, records=True, p_absorb=0.3, seed=SEED)
    h, nseg, st = N.unpack_records(rec)
    assert h[0] == o["hash"][0] and nseg[0] == o["nseg"][0]
    out = np.zeros(g.n_inst)
    assert g.lib.tally_read(g.h, N._ptr(tally), out.ctypes.data_as(ctypes.c_void_p), g.n_inst - 1,
                            None, None) == -1
    assert g.lib.tally_read(g.h, N._ptr(tally), None, g.n_inst, None, None) == -1
    hexg = _gpu(I.small_hex(), exact=False)
    p = hexg.source_init(10)
    assert hexg.rect_ok   # the array tracker runs hex arrays (closed-form search)
    hexg.run_histories(p, 10, tracker=N.TRACKER_RECT)
    with pytest.raises(N.TrkError) as e:
        hexg.run_histories(p, 10, tracker=7)
    assert e.value.code == -1
    with pytest.raises(N.TrkError) as e:
        g.run_histories(parts, 1, p_absorb=1.5)
    assert e.value.code == -1


def test_tally_read_units():
    desc = I.config1()
    g = _gpu(desc, exact=True)
    n = 2000
    parts = g.source_init(n, seed=SEED)
    tally, cnt, _ = g.run_histories(parts, n, p_absorb=0.3, seed=SEED)
    cm = g.tally_read(tally, cnt)
    ref = _oracle(desc, O.MODE_RECT).run(n, SEED, 0.3)["tally"]
    assert np.array_equal(cm, ref.astype(np.float64) * 2.0**-32)


# ---------------------------------------------------------------------------
# transmission forward / backward
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("tracker,mode", [(N.TRACKER_RECT, O.MODE_RECT), (N.TRACKER_CSG, O.MODE_CSG)])
def test_transmission_against_oracle(tracker, mode):
    r_out = 0.5 * 3 * 5 * 1.26 * 1.2
    desc = I.small_core(height=20.0, r_outer=r_out)
    sigma = np.array(desc["sigma"])
    rays = I.boundary_rays(4000, r_outer=r_out, height=20.0, seed=11).packed()
    ref = _oracle(desc, mode).transmission(rays, sigma, pitch=1.26)
    g = _gpu(desc, exact=True)
    R = torch.from_numpy(rays).cuda()
    S = torch.from_numpy(sigma).cuda()
    T, L = g.transmission_fwd(R, S, tracker=tracker)
    assert np.array_equal(L.cpu().numpy(), ref["lens"])
    assert np.allclose(T.cpu().numpy(), ref["T"], rtol=1e-14, atol=0)
    gT = torch.from_numpy(np.random.default_rng(2).normal(size=len(rays))).cuda()
    grad = g.transmission_bwd(R, S, 1.26, gT, tracker=tracker).cpu().numpy()
    expect = (gT.cpu().numpy()[:, None] * ref["dT"]).sum(0)
    assert np.allclose(grad, expect, rtol=1e-10, atol=1e-14 * np.abs(expect).max())


# ---------------------------------------------------------------------------
# event-based persistent kernel
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name", ["c1", "small_core", "c2", "tiny8"])
@pytest.mark.parametrize("tracker,mode", [(N.TRACKER_RECT, O.MODE_RECT), (N.TRACKER_CSG, O.MODE_CSG)])
def test_event_bit_exact(name, tracker, mode):
    desc, pa, n = CASES[name]
    o = _oracle(desc, mode).run(n, SEED, pa, threads=8)
    g = _gpu(desc, exact=True)
    parts = g.source_init(n, seed=SEED)
    tally, cnt, rec = g.run_histories(parts, n, records=True, tracker=tracker, mode=N.MODE_EVENT,
                                      p_absorb=pa, seed=SEED)
    torch.cuda.synchronize()
    h, nseg, st = N.unpack_records(rec)
    assert np.array_equal(st, o["status"])
    assert np.array_equal(nseg, o["nseg"])
    assert np.array_equal(h, o["hash"])
    assert np.array_equal(_u64(tally), o["tally"])
    c = _u64(cnt)
    assert np.array_equal(c[:10], o["counters"][:10]) and c[N.K["status"]] == 0


@pytest.mark.parametrize("name", list(HEX_CASES))
def test_event_bit_exact_hex(name):
    desc, pa, n = HEX_CASES[name]
    o = _oracle(desc, O.MODE_CSG).run(n, SEED, pa, threads=8)
    g = _gpu(desc, exact=True)
    parts = g.source_init(n, seed=SEED)
    tally, cnt, rec = g.run_histories(parts, n, records=True, tracker=N.TRACKER_CSG, mode=N.MODE_EVENT,
                                      p_absorb=pa, seed=SEED)
    h, nseg, st = N.unpack_records(rec)
    assert np.array_equal(h, o["hash"]) and np.array_equal(_u64(tally), o["tally"])


@pytest.mark.parametrize("depth,grid", [(32, 1), (64, 3), (100, 0), (128, 0), (512, 2)])
def test_event_queue_shapes(depth, grid):
    desc, pa, n = CASES["small_core"]
    n = 2_999
    g = _gpu(desc, exact=True)
    parts = g.source_init(n, seed=SEED)
    ref = g.run_histories(parts, n, records=True, tracker=N.TRACKER_CSG, p_absorb=pa, seed=SEED)
    got = g.run_histories(parts, n, records=True, tracker=N.TRACKER_CSG, mode=N.MODE_EVENT,
                          queue_depth=depth, grid=grid, p_absorb=pa, seed=SEED)
    torch.cuda.synchronize()
    assert np.array_equal(_u64(ref[2]), _u64(got[2]))
    assert np.array_equal(_u64(ref[0]), _u64(got[0]))
    assert np.array_equal(_u64(ref[1]), _u64(got[1]))


@pytest.mark.parametrize("depth", [32, 100, 512])
@pytest.mark.parametrize("tracker", [N.TRACKER_CSG, N.TRACKER_RECT])
def test_fp32_local_event_equals_history(depth, tracker):
    # FP32-local, fast build: the event kernel queues the flights it redoes
    # in FP64 and runs them in a later pass, the history kernel redoes them
    # at once; each particle's arithmetic is the same, so the records,
    # tallies and counters are identical at every queue depth (full batches,
    # carried tails and the redo queue included)
    desc, pa, n = CASES["small_core"]
    n = 4_001
    g = _gpu(desc, exact=False)
    parts = g.source_init(n, seed=SEED)
    kw = dict(records=True, tracker=tracker, precision=N.FP32_LOCAL, p_absorb=pa, seed=SEED)
    ref = g.run_histories(parts, n, **kw)
    got = g.run_histories(parts, n, mode=N.MODE_EVENT, queue_depth=depth, **kw)
    torch.cuda.synchronize()
    assert np.array_equal(_u64(ref[2]), _u64(got[2]))
    assert np.array_equal(_u64(ref[0]), _u64(got[0]))
    c_ref, c_got = _u64(ref[1]), _u64(got[1])
    assert np.array_equal(c_ref, c_got)
    assert c_ref[N.K["close_calls"]] > 0   # the redo path ran


def test_event_cutoff_segment_cap_and_tiny_n():
    desc = I.config1()
    g = _gpu(desc, exact=True)
    for n, kw, mode in ((1, {}, O.MODE_RECT), (5, {"max_segments": 3}, O.MODE_RECT),
                        (700, {"max_path": 40.0}, O.MODE_CSG)):
        o = _oracle(desc, mode).run(n, SEED, 0.3, **kw)
        parts = g.source_init(n, seed=SEED)
        tally, cnt, rec = g.run_histories(parts, n, records=True, mode=N.MODE_EVENT,
                                          tracker=N.TRACKER_RECT if mode == O.MODE_RECT else N.TRACKER_CSG,
                                          p_absorb=0.3, seed=SEED, **kw)
        h, nseg, st = N.unpack_records(rec)
        assert np.array_equal(h, o["hash"]) and np.array_equal(st, o["status"])


def test_event_full_size_matches_history():
    desc = I.config2()
    n, pa = 10_000_000, 0.25
    g = _gpu(desc, exact=True)
    parts = g.source_init(n, seed=SEED)
    a = g.run_histories(parts, n, records=True, tracker=N.TRACKER_CSG, p_absorb=pa, seed=SEED)
    b = g.run_histories(parts, n, records=True, tracker=N.TRACKER_CSG, mode=N.MODE_EVENT, p_absorb=pa, seed=SEED)
    torch.cuda.synchronize()
    assert np.array_equal(_u64(a[0]), _u64(b[0]))
    assert np.array_equal(_u64(a[1]), _u64(b[1]))
    assert np.array_equal(_u64(a[2]), _u64(b[2]))


# ---------------------------------------------------------------------------
# FP32-local precision (fast build): error against the FP64 oracle
# ---------------------------------------------------------------------------

def _fp32_stats(desc, pa, n, tracker, mode, cap=4096):
    o = _oracle(desc, mode)
    g = _gpu(desc, exact=False)
    parts = g.source_init(n, seed=SEED)
    inst, ln, tally, cnt = g.trace(parts, n, cap, tracker=tracker, precision=N.FP32_LOCAL, p_absorb=pa, seed=SEED)
    inst, ln = inst.cpu().numpy(), ln.cpu().numpy()
    ref = o.run(n, SEED, pa, threads=8)
    mism, rel, ab = 0, [], []
    for i in range(n):
        oi, ol, _, _ = o.trace(i, SEED, pa, cap=cap)
        k = len(oi)
        gk = int((inst[i] >= 0).sum())
        if gk != k or not np.array_equal(inst[i, :k], oi):
            mism += 1
            continue
        d = np.abs(ln[i, :k] - ol)
        ab.append(d.max())
        big = ol > 1e-3
        if big.any():
            rel.append((d[big] / ol[big]).max())
    t_ref = ref["tally"].astype(np.float64)
    t_got = _u64(tally).astype(np.float64)
    sel = t_ref > 1e-3 * t_ref.max()
    bin_rel = np.abs(t_got[sel] - t_ref[sel]) / t_ref[sel]
    return dict(mism=mism, rel=np.array(rel), ab=np.array(ab), l1=np.abs(t_got - t_ref).sum() / t_ref.sum(),
                linf=bin_rel.max(), close=int(_u64(cnt)[N.K["close_calls"]]), seg=int(_u64(cnt)[0]))


@pytest.mark.parametrize("name,tracker,mode", [("c1", N.TRACKER_RECT, O.MODE_RECT), ("c1", N.TRACKER_CSG, O.MODE_CSG),
                                               ("small_core", N.TRACKER_CSG, O.MODE_CSG),
                                               ("small_core", N.TRACKER_RECT, O.MODE_RECT)])
def test_fp32_local_error_bounds(name, tracker, mode):
    desc, pa, n = CASES[name]
    n = min(n, 3000)
    st = _fp32_stats(desc, pa, n, tracker, mode)
    print(name, tracker, {k: (v if not isinstance(v, np.ndarray) else (float(np.quantile(v, 0.5)),
                                                                        float(np.quantile(v, 0.99)), float(v.max())))
                          for k, v in st.items()})
    # FP32 distances in element-local frames carry ~1e-7 relative error per
    # segment.  A history couples its position error to where its collisions
    # fall (tau is spent by material), so long histories drift further; the
    # bars are on the typical history and on the aggregate tally.
    assert st["mism"] <= max(3, n // 200)
    assert np.median(st["rel"]) < 1e-5
    assert np.quantile(st["rel"], 0.75) < 1e-4
    assert st["l1"] < 1e-4
    assert st["close"] < 0.05 * st["seg"]


def test_fp32_local_hex():
    desc, pa, n = HEX_CASES["small_hex_core"]
    st = _fp32_stats(desc, pa, n, N.TRACKER_CSG, O.MODE_CSG)
    print("hex", {k: (v if not isinstance(v, np.ndarray) else float(np.quantile(v, 0.99))) for k, v in st.items()})
    assert st["mism"] <= max(3, n // 200)
    assert np.median(st["rel"]) < 1e-5
    assert st["l1"] < 1e-4


@pytest.mark.parametrize("mode", [N.MODE_HISTORY, N.MODE_EVENT])
def test_fp32_local_full_size_counts(mode):
    desc = I.config2()
    n, pa = 10_000_000, 0.25
    g = _gpu(desc, exact=False)
    parts = g.source_init(n, seed=SEED)
    a = g.run_histories(parts, n, records=True, tracker=N.TRACKER_CSG, p_absorb=pa, seed=SEED)
    b = g.run_histories(parts, n, records=True, tracker=N.TRACKER_CSG, mode=mode, precision=N.FP32_LOCAL,
                        p_absorb=pa, seed=SEED)
    torch.cuda.synchronize()
    ca, cb = _u64(a[1]), _u64(b[1])
    assert cb[N.K["lost"]] == 0 and cb[N.K["status"]] == 0
    assert cb[N.K["absorbed"]] + cb[N.K["escaped"]] == n
    _, na, sa = N.unpack_records(a[2])
    _, nb, sb = N.unpack_records(b[2])
    same = (na == nb) & (sa == sb)
    print("fp32 full", mode, same.mean(), cb[N.K["close_calls"]] / cb[0])
    assert same.mean() > 0.995
    ta, tb = _u64(a[0]).astype(np.float64), _u64(b[0]).astype(np.float64)
    assert abs(tb.sum() - ta.sum()) / ta.sum() < 1e-4


# ---------------------------------------------------------------------------
# failure detection without a GPU fault: the event kernel's round limit
# ---------------------------------------------------------------------------

def test_event_round_limit_reports_timeout():
    desc, pa, n = CASES["small_core"]
    g = _gpu(desc, exact=False)
    parts = g.source_init(n, seed=SEED)
    tally, cnt, _ = g.run_histories(parts, n, tracker=N.TRACKER_CSG, mode=N.MODE_EVENT, max_rounds=2,
                                    p_absorb=pa, seed=SEED)
    torch.cuda.synchronize()
    c = cnt.cpu().numpy()
    assert c[N.K["status"]] == -7                       # TRK_E_TIMEOUT, read on the host
    with pytest.raises(N.TrkError) as e:
        g.tally_read(tally, cnt)
    assert e.value.code == -7
    # the context stays usable: a normal run afterwards completes
    tally2, cnt2, _ = g.run_histories(parts, n, tracker=N.TRACKER_CSG, mode=N.MODE_EVENT, p_absorb=pa, seed=SEED)
    g.tally_read(tally2, cnt2)
    assert int(cnt2.cpu()[N.K["status"]]) == 0
