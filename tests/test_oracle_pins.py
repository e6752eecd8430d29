"""Pins for the CPU oracle: each check compares it with something other than itself.

- Philox4x32-10 against published known-answer vectors (tests/golden).
- The own log against the C library's log (<= 2 ulp) and E[-log xi] = 1.
- Marsaglia directions: unit length, zero mean, E[w^2] = 1/3.
- Hierarchical find_cell (Alg. 7, both tracker modes) against brute force over
  every leaf instance evaluated in the global frame.
- Segment sums along straight rays against closed-form chords (cylinder by
  impact parameter, box and hex prism by the slab method).
- Cauchy's mean-chord law 4V/S for cosine-law rays, whole body and per cell.
- Track-length volume estimates in a reflecting box converging to pi r^2 h.
- Collision count per history ~ Geometric(p_a); total path ~ Exp(p_a sigma).
- rect-tracker mode vs CSG (pseudo-array) mode: identical histories.
- Analytic transmission gradient against central finite differences.
"""
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2406_13849_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _geom(desc, mode=O.MODE_RECT):
    return O.Geometry(I.to_json(desc), mode)


# ---------------------------------------------------------------------------
# random numbers
# ---------------------------------------------------------------------------

def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = O.philox4x32_10(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


def test_uniform_range_and_moments():
    xs = np.array([O.uniform2(i, 0, 2, 0, 1, 0) for i in range(20000)]).ravel()
    assert xs.min() > 0.0 and xs.max() <= 1.0
    assert abs(xs.mean() - 0.5) < 5 * math.sqrt(1 / 12 / len(xs))
    # the resolution is 2^-53: every value is an integer multiple of it
    assert np.all(np.floor(xs * 2.0**53) == xs * 2.0**53)


def test_log_within_two_ulp():
    rng = np.random.default_rng(0)
    xs = np.concatenate([rng.uniform(0, 1, 20000)[1:], 2.0 ** -rng.uniform(0, 53, 20000),
                         rng.uniform(0.5, 2.0, 20000), [1.0, 0.5, 2.0, 2.0**-53, 1 - 2.0**-53]])
    worst = 0.0
    for x in xs:
        a, b = O.own_log(x), math.log(x)
        if a != b:
            worst = max(worst, abs(a - b) / np.spacing(abs(b)))
    assert worst <= 2.0
    assert O.own_log(1.0) == 0.0


def test_log_split_constant():
    from decimal import Decimal, getcontext
    from fractions import Fraction
    getcontext().prec = 50
    ln2 = Fraction(Decimal(2).ln())
    hi = float.fromhex("0x1.62e42fefp-1")
    lo = float.fromhex("0x1.473de6af278edp-34")
    assert abs(float(ln2 - Fraction(hi) - Fraction(lo))) <= 0.5 * float(np.spacing(lo))
    # exact -log of every xi = 2^-k, a case the series does not touch (m = 1)
    for k in range(1, 54):
        assert abs(-O.own_log(2.0**-k) - k * math.log(2.0)) <= 2 * np.spacing(k * math.log(2.0))


def test_exponential_mean():
    xi = np.array([O.uniform2(i, 0, 2, 0, 3, 0)[1] for i in range(40000)])
    tau = np.array([-O.own_log(x) for x in xi])
    assert abs(tau.mean() - 1.0) < 5 / math.sqrt(len(tau))
    assert abs(tau.var() - 1.0) < 0.05


def test_isotropic_directions():
    d = np.array([O.isotropic(i, 1, 7, 0)[0] for i in range(30000)])
    assert np.max(np.abs(np.linalg.norm(d, axis=1) - 1.0)) < 1e-15
    n = len(d)
    assert np.all(np.abs(d.mean(0)) < 5 * math.sqrt(1 / 3 / n))
    assert abs((d[:, 2] ** 2).mean() - 1 / 3) < 5 * math.sqrt(4 / 45 / n)
    assert abs((d[:, 0] * d[:, 1]).mean()) < 5 * math.sqrt(1 / 15 / n)


# ---------------------------------------------------------------------------
# find_cell against brute force over every leaf instance
# ---------------------------------------------------------------------------

def _members_by_kind():
    """First configuration-4 members of each (lattice, levels) kind."""
    seen = {}
    for i in range(64):
        d, _ = I.config4_member(i)
        kind = (any(u["type"] == "hex" for u in d["universes"]), len(d["universes"]))
        seen.setdefault(kind, i)
    return sorted(seen.values())


def _points(desc, n, seed):
    lo = np.array(desc["source_box"][:3])
    hi = np.array(desc["source_box"][3:])
    rng = np.random.default_rng(seed)
    return lo + rng.uniform(0, 1, (n, 3)) * (hi - lo)


@pytest.mark.parametrize("name,desc,modes", [
    ("c1", I.config1(), (O.MODE_RECT, O.MODE_CSG)),
    ("small_core", I.small_core(), (O.MODE_RECT, O.MODE_CSG)),
    ("small_hex_core", I.small_hex_core(), (O.MODE_CSG,)),
    ("hex_rot", I.small_hex(rings=3, rot30=True), (O.MODE_CSG,)),
    ("tiny5", I.random_tiny(5), (O.MODE_RECT, O.MODE_CSG)),
    ("tiny11", I.random_tiny(11), (O.MODE_RECT, O.MODE_CSG)),
    ("c2", I.config2(), (O.MODE_RECT, O.MODE_CSG)),
    ("c3", I.config3(), (O.MODE_RECT, O.MODE_CSG)),
] + [(f"c4m{m}", I.config4_member(m)[0], (O.MODE_RECT, O.MODE_CSG)) for m in _members_by_kind()])
def test_find_cell_matches_brute_force(name, desc, modes):
    # the full-size cores have 191,929 and 27,686 leaves: fewer points there
    pts = _points(desc, {"c2": 300, "c3": 600}.get(name, 3000), 11)
    # the leaves evaluated in the global frame are the same in both modes
    brute, count, near, nleaf = _geom(desc, modes[0]).find_cell_brute(pts)
    far = near > 1e-9
    assert far.mean() > 0.99
    # away from surfaces exactly one leaf instance holds the point
    assert np.all(count[far & (brute >= 0)] == 1)
    for mode in modes:
        g = _geom(desc, mode)
        assert nleaf == g.n_inst
        hier = g.find_cell(pts)
        assert np.array_equal(hier[far], brute[far]), (name, mode)


def test_instance_counts():
    assert _geom(I.config1()).n_inst == 867
    assert _geom(I.config2()).n_inst == 191_929
    assert _geom(I.config3(), O.MODE_CSG).n_inst == 27_686


# ---------------------------------------------------------------------------
# chords
# ---------------------------------------------------------------------------

def test_cylinder_chord_by_impact_parameter():
    R, z0, z1 = 0.41, 0.0, 10.0
    g = _geom(I.bare_cylinder(R, z0, z1), O.MODE_CSG)
    rays = I.cylinder_rays(4000, R, z0, z1, seed=3)
    res = g.transmission(rays.packed(), [0.0], grad=False)
    o, d = rays.origin, rays.direction
    sxy = np.hypot(d[:, 0], d[:, 1])
    b = np.abs(o[:, 0] * d[:, 1] - o[:, 1] * d[:, 0]) / sxy   # impact parameter
    s0 = (o[:, 0] * d[:, 0] + o[:, 1] * d[:, 1]) / sxy       # start along the projected line
    # remaining half-chord beyond the closest approach, from the (inset) start point
    chord = (np.sqrt(R * R - b * b) - s0) / sxy
    # keep rays that enter and leave through the lateral face
    lateral = np.abs(np.hypot(o[:, 0], o[:, 1]) - R) < 1e-6
    zend = o[:, 2] + chord * d[:, 2]
    ok = lateral & (zend > z0 + 1e-6) & (zend < z1 - 1e-6)
    assert ok.sum() > 500
    tot = res["lens"].sum(1)
    assert np.all(res["status"][ok] == O.P_ESCAPED)
    assert np.max(np.abs(tot[ok] - chord[ok]) / chord[ok]) < 1e-9


def _slab_exit(o, d, lo, hi):
    t = np.full(len(o), np.inf)
    for k in range(3):
        with np.errstate(divide="ignore", invalid="ignore"):
            tk = np.where(d[:, k] > 0, (hi[k] - o[:, k]) / d[:, k],
                          np.where(d[:, k] < 0, (lo[k] - o[:, k]) / d[:, k], np.inf))
        t = np.minimum(t, tk)
    return t


@pytest.mark.parametrize("mode", [O.MODE_RECT, O.MODE_CSG])
def test_box_chord_through_lattice(mode):
    desc = I.config1(sigma=(0.0, 0.0, 0.0), bc="vacuum")
    g = _geom(desc, mode)
    lo, hi = np.array(desc["source_box"][:3]), np.array(desc["source_box"][3:])
    rays = I.box_rays(2000, lo, hi, seed=4)
    res = g.transmission(rays.packed(), [0, 0, 0], grad=False)
    ref = _slab_exit(rays.origin, rays.direction, lo, hi)
    assert np.all(res["status"] == O.P_ESCAPED)
    assert np.max(np.abs(res["lens"].sum(1) - ref) / ref) < 1e-10


def test_hex_prism_chord():
    # a single hex cell (rings 0) is the intersection of 3 slabs and a z slab
    pitch, h = 2.0, 4.0
    desc = I.small_hex(rings=0, pitch=pitch, r_pin=0.3, height=h, sigma=(0.0, 0.0))
    g = _geom(desc, O.MODE_CSG)
    rng = np.random.default_rng(8)
    n = 3000
    apo = pitch / 2
    o = np.stack([rng.uniform(-0.5, 0.5, n), rng.uniform(-0.5, 0.5, n), rng.uniform(0.5, 3.5, n)], 1)
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    res = g.transmission(np.concatenate([o, d], 1), [0.0, 0.0], grad=False)
    t = np.full(n, np.inf)
    for ang in (0.0, 60.0, 120.0):
        nv = np.array([math.cos(math.radians(ang)), math.sin(math.radians(ang)), 0.0])
        on, dn = o @ nv, d @ nv
        with np.errstate(divide="ignore"):
            t = np.minimum(t, np.where(dn > 0, (apo - on) / dn, np.where(dn < 0, (-apo - on) / dn, np.inf)))
    t = np.minimum(t, np.where(d[:, 2] > 0, (h - o[:, 2]) / d[:, 2], -o[:, 2] / d[:, 2]))
    assert np.max(np.abs(res["lens"].sum(1) - t) / t) < 1e-9


# ---------------------------------------------------------------------------
# Cauchy mean chord and track-length volumes
# ---------------------------------------------------------------------------

def test_cauchy_cylinder():
    R, H = 0.41, 3.0
    g = _geom(I.bare_cylinder(R, 0.0, H), O.MODE_CSG)
    rays = I.cylinder_rays(60000, R, 0.0, H, seed=12)
    tot = g.transmission(rays.packed(), [0.0], grad=False)["lens"].sum(1)
    expect = 2 * R * H / (H + R)
    assert abs(tot.mean() - expect) < 5 * tot.std() / math.sqrt(len(tot))


@pytest.mark.parametrize("mode", [O.MODE_RECT, O.MODE_CSG])
def test_cauchy_box_per_cell(mode):
    n, p, h = 3, 1.26, 4.0
    desc = I.config1(sigma=(0.0, 0.0, 0.0), n=n, height=h, bc="vacuum")
    g = _geom(desc, mode)
    lo, hi = np.array(desc["source_box"][:3]), np.array(desc["source_box"][3:])
    a, b, c = hi - lo
    rays = I.box_rays(40000, lo, hi, seed=13)
    lens = g.transmission(rays.packed(), [0, 0, 0], grad=False)["lens"]
    S = 2 * (a * b + b * c + c * a)
    tot = lens.sum(1)
    assert abs(tot.mean() - 4 * a * b * c / S) < 5 * tot.std() / math.sqrt(len(tot))
    vf = n * n * math.pi * 0.41**2 * h
    vc = n * n * math.pi * (0.475**2 - 0.41**2) * h
    for m, v in ((0, vf), (1, vc)):
        assert abs(lens[:, m].mean() - 4 * v / S) < 5 * lens[:, m].std() / math.sqrt(len(tot))


@pytest.mark.parametrize("mode", [O.MODE_RECT, O.MODE_CSG])
def test_track_length_volumes(mode):
    # sigma = 0, reflecting walls: uniform isotropic phase space stays so, and
    # V_cell = V_box * tally_cell / (N L) for histories cut at path length L.
    n, h = 17, 100.0
    desc = I.config1(sigma=(0.0, 0.0, 0.0))
    g = _geom(desc, mode)
    L, N, B = 300.0, 400, 6
    vbox = (n * 1.26) ** 2 * h
    est = []
    for b in range(B):
        r = g.run(N, seed=21, p_absorb=0.3, first_id=b * N, max_path=L, records=False)
        assert r["counters"][O.K_CUTOFF] == N
        t = r["tally"].astype(np.float64).reshape(n * n, 3).sum(0) / 2.0**32
        est.append(vbox * t / (N * L))
    est = np.array(est)
    m, s = est.mean(0), est.std(0, ddof=1) / math.sqrt(B)
    exact = np.array([math.pi * 0.41**2 * h, math.pi * (0.475**2 - 0.41**2) * h,
                      1.26**2 * h - math.pi * 0.475**2 * h]) * n * n
    assert np.all(np.abs(m - exact) < 5 * s + 1e-3 * exact)
    assert abs(m.sum() - vbox) < 1e-6 * vbox


# ---------------------------------------------------------------------------
# collision physics
# ---------------------------------------------------------------------------

def test_collision_count_geometric_and_path_exponential():
    from scipy import stats
    sig, pa = 0.5, 0.3
    g = _geom(I.config1(sigma=(sig, sig, sig)))
    ncoll, path = [], []
    for pid in range(6000):
        inst, ln, kind, st = g.trace(pid, seed=5, p_absorb=pa)
        assert st == O.P_ABSORBED
        ncoll.append(int((kind == 1).sum()))
        path.append(ln.sum())
    ncoll = np.array(ncoll)
    kmax = 12
    obs = np.array([(ncoll == k).sum() for k in range(1, kmax)] + [(ncoll >= kmax).sum()])
    pk = np.array([(1 - pa) ** (k - 1) * pa for k in range(1, kmax)] + [(1 - pa) ** (kmax - 1)])
    chi2 = ((obs - pk * len(ncoll)) ** 2 / (pk * len(ncoll))).sum()
    assert stats.chi2.sf(chi2, kmax - 1) > 1e-4
    # a geometric sum of Exp(sigma) free paths is Exp(p_a sigma)
    assert stats.kstest(np.array(path), "expon", args=(0, 1 / (pa * sig))).pvalue > 1e-4


@pytest.mark.parametrize("mode", [O.MODE_RECT, O.MODE_CSG])
def test_counting_build_is_the_same_arithmetic(mode):
    """The operation count behind the benchmark's roofline comes from the
    oracle compiled on a counting scalar type: its histories must equal the
    plain build's bit for bit, its counts must add up over disjoint particle
    ranges, and they must cover what every segment needs at least (the
    collision distance tau / Sigma: one division; the move r + l Omega:
    three multiplications and three additions)."""
    desc = I.to_json(I.small_core())
    plain = O.Geometry(desc, mode).run(300, 5, 0.25)
    gc = O.Geometry(desc, mode, counting=True)
    gc.flop_counts(reset=True)
    cnt = gc.run(300, 5, 0.25)
    whole = gc.flop_counts()
    assert np.array_equal(cnt["hash"], plain["hash"]) and np.array_equal(cnt["tally"], plain["tally"])
    gc.flop_counts(reset=True)
    gc.run(100, 5, 0.25)
    part = gc.flop_counts()
    gc.flop_counts(reset=True)
    gc.run(200, 5, 0.25, first_id=100)
    rest = gc.flop_counts()
    assert all(part[k] + rest[k] == whole[k] for k in whole)
    seg = int(plain["counters"][O.K_SEGMENTS])
    assert whole["div"] >= seg and whole["mul"] >= 3 * seg and whole["add"] >= 3 * seg


def test_rect_and_csg_modes_identical():
    for desc in (I.config1(), I.small_core(), I.random_tiny(3)):
        ra = _geom(desc, O.MODE_RECT).run(1500, 1, 0.3)
        rb = _geom(desc, O.MODE_CSG).run(1500, 1, 0.3)
        assert np.array_equal(ra["hash"], rb["hash"])
        assert np.array_equal(ra["tally"], rb["tally"])
        assert np.array_equal(ra["counters"], rb["counters"])


def test_thread_count_invariance():
    g = _geom(I.small_core())
    a = g.run(3000, 2, 0.25, threads=1)
    b = g.run(3000, 2, 0.25, threads=4)
    for k in ("tally", "counters", "hash", "nseg", "status"):
        assert np.array_equal(a[k], b[k])


def test_sharding_sums_to_whole():
    g = _geom(I.config1())
    whole = g.run(2000, 9, 0.3, records=False)
    parts = [g.run(500, 9, 0.3, first_id=500 * k, records=False) for k in range(4)]
    assert np.array_equal(sum(p["tally"] for p in parts), whole["tally"])
    assert np.array_equal(sum(p["counters"] for p in parts), whole["counters"])


def test_source_in_box_and_root():
    desc = I.config2()
    g = _geom(desc)
    src, st = g.source(5000, 1)
    assert np.all(st == 0)
    r = np.hypot(src[:, 0], src[:, 1])
    assert np.all(r < 170.0) and np.all((src[:, 2] >= 0) & (src[:, 2] < 366.0))
    assert np.max(np.abs(np.linalg.norm(src[:, 3:6], axis=1) - 1)) < 1e-15
    assert np.all(src[:, 6] >= 0)


def test_source_distributions():
    """Births are uniform over the root volume (Alg. 2), isotropic, with
    tau ~ Exp(1): for the r = 170 cylinder of configuration 2 (source box the
    circumscribed square), r^2/R^2, z/H and the azimuth are U(0, 1) when the
    rejection step keeps whole points; each direction component is U(-1, 1)
    (Archimedes); tau = -log(xi) is Exp(1).  A rejection loop that redrew one
    coordinate, a swapped random stream or a wrong source box fails one of
    these."""
    from scipy import stats
    g = _geom(I.config2(), O.MODE_CSG)
    src, st = g.source(20000, 7)
    assert np.all(st == 0)
    R, H = 170.0, 366.0
    x, y, z = src[:, 0], src[:, 1], src[:, 2]
    checks = {
        "r^2": (x * x + y * y) / (R * R),
        "z": z / H,
        "phi": (np.arctan2(y, x) + math.pi) / (2 * math.pi),
        "u": (src[:, 3] + 1) / 2, "v": (src[:, 4] + 1) / 2, "w": (src[:, 5] + 1) / 2,
    }
    for name, vals in checks.items():
        assert stats.kstest(vals, "uniform").pvalue > 1e-4, name
    assert stats.kstest(src[:, 6], "expon").pvalue > 1e-4
    # first_id shifts the stream: ids k..k+n-1 reproduce the tail of a longer run
    tail, _ = g.source(100, 7, first_id=19900)
    assert np.array_equal(tail, src[19900:])


def test_max_segments_and_escape_status():
    g = _geom(I.config1())
    r = g.run(50, 1, 0.0, max_segments=10)
    assert np.all(r["status"] == O.P_MAXSEG) and np.all(r["nseg"] == 10)
    v = _geom(I.single_pin(bc="vacuum", sigma=(0.01, 0.01, 0.01))).run(500, 1, 0.3)
    assert (v["status"] == O.P_ESCAPED).mean() > 0.9


def test_bad_descriptions_rejected():
    d = I.config1()
    d["universes"][1]["fill"] = [0] * 5
    with pytest.raises(ValueError):
        _geom(d)
    d = I.config1()
    d["surfaces"][0]["bc"] = "reflect"
    with pytest.raises(ValueError):
        _geom(d)
    with pytest.raises(ValueError):
        O.Geometry("{not json", O.MODE_RECT)


def _negative_fill(cell):
    del cell["material"]
    cell["fill"] = -2


@pytest.mark.parametrize("mutate", [
    lambda d: d["universes"].append(dict(d["universes"][0])),                 # unreachable universe
    lambda d: d.update(root=-0.5),                                              # not an integer index
    lambda d: d["universes"][0]["cells"][0].update(material=-1),
    lambda d: _negative_fill(d["universes"][0]["cells"][0]),
    lambda d: d["universes"][0]["cells"][0]["surfaces"][0].__setitem__(0, 0.5),
    lambda d: d["universes"][0]["cells"][0]["surfaces"][0].__setitem__(1, 0),
    lambda d: d["surfaces"][0].update(rparam=3),
    lambda d: d["universes"][1].update(pscale=2),
    lambda d: d["universes"][1]["fill"].__setitem__(0, 0.5),
    lambda d: d["universes"][1]["grid"][0].__setitem__(0, -1e999),
    lambda d: d.update(source_box=[0, 0, 0, 0, 1, 1]),
    lambda d: d.update(sigma=[0.8, -0.3, 0.1]),
    lambda d: d.update(geometry_id=1e30),
])
def test_descriptions_with_bad_indices_or_numbers_rejected(mutate):
    """The oracle's reader rejects what the library's builder rejects: a
    universe the root never reaches, indices that are not integers in
    range, tags out of range, non-finite or empty geometry."""
    d = I.config1()
    mutate(d)
    with pytest.raises(ValueError):
        O.Geometry(I.to_json(d).replace("Infinity", "1e999"), O.MODE_RECT)


def test_rect_mode_tracks_hex_arrays_as_pseudo_arrays():
    # the rect-mode oracle keeps rect arrays by index and turns hex arrays
    # into pseudo-arrays: on hex geometries (two and three hex levels) it
    # must agree with CSG mode, as on a rect geometry
    for d in (I.small_hex_core(), I.config4_member(1)[0], I.config4_member(4)[0]):
        a = _geom(d, O.MODE_RECT).run(300, 1, 0.3, threads=4)
        b = _geom(d, O.MODE_CSG).run(300, 1, 0.3, threads=4)
        assert np.array_equal(a["hash"], b["hash"]) and np.array_equal(a["tally"], b["tally"])


# ---------------------------------------------------------------------------
# transmission gradient
# ---------------------------------------------------------------------------

def test_transmission_sigma_gradient_exact():
    desc = I.small_core(height=20.0)
    g = _geom(desc)
    rays = I.boundary_rays(300, r_outer=desc["surfaces"][9]["coef"][2], height=20.0, seed=2).packed()
    sigma = np.array(desc["sigma"])
    res = g.transmission(rays, sigma)
    assert np.allclose(res["dT"][:, :4], -res["lens"] * res["T"][:, None], rtol=0, atol=0)
    assert np.allclose(res["T"], np.exp(-(res["lens"] * sigma).sum(1)), rtol=1e-15)


def _inside_cylinder(o, d, cx, cy, r, t_end):
    """Length of {t in [0, t_end]: (o + t d - c)_xy inside radius r}, from the
    ray's closest approach to the axis (no walk, no cells)."""
    return _chords(o, d, np.array([cx]), np.array([cy]), r, t_end)


@pytest.mark.parametrize("mode", [O.MODE_RECT, O.MODE_CSG])
def test_transmission_lengths_by_closed_form(mode):
    """Per-material lengths of transmission rays through the 17x17 pin lattice
    in a vacuum box against a computation that never walks the geometry: the
    box exit by the slab method, and per pin the ray's interval inside each
    cylinder (fuel = r_fuel chord, clad = r_clad chord - r_fuel chord,
    moderator = the rest).  A dropped segment, a swapped material or a wrong
    element frame would each move a length by a chord."""
    pitch, n, rf, rc, height = 1.26, 17, 0.41, 0.475, 100.0
    desc = I.config1(bc="vacuum", pitch=pitch, n=n, r_fuel=rf, r_clad=rc, height=height)
    half = n / 2.0 * pitch
    lo, hi = np.array([-half, -half, 0.0]), np.array([half, half, height])
    rng = np.random.default_rng(17)
    m = 300
    org = lo + rng.uniform(0.0, 1.0, (m, 3)) * (hi - lo)
    w = rng.normal(size=(m, 3))
    w /= np.linalg.norm(w, axis=1)[:, None]
    w[:10] = np.eye(3)[rng.integers(0, 3, 10)] * rng.choice([-1.0, 1.0], (10, 1))   # axis-parallel rays
    rays = np.concatenate([org, w], axis=1)
    sigma = np.array(desc["sigma"])
    res = _geom(desc, mode).transmission(rays, sigma, grad=False)
    assert (res["status"] == 2).all()     # every ray leaves through the vacuum box (escaped)
    centres = [(i - half / pitch + 0.5) * pitch for i in range(n)]
    cxs, cys = (np.array(v).ravel() for v in np.meshgrid(centres, centres))
    for k in range(m):
        o, d = org[k], w[k]
        t_exit = min(((hi[a] if d[a] > 0 else lo[a]) - o[a]) / d[a] for a in range(3) if d[a] != 0.0)
        fuel = _chords(o, d, cxs, cys, rf, t_exit)
        clad_out = _chords(o, d, cxs, cys, rc, t_exit)
        expect = np.array([fuel, clad_out - fuel, t_exit - clad_out])
        assert np.allclose(res["lens"][k], expect, rtol=1e-12, atol=1e-11), (k, res["lens"][k], expect)
    assert np.allclose(res["T"], np.exp(-(res["lens"] * sigma).sum(1)), rtol=1e-15)


@pytest.mark.parametrize("rot30", [False, True])
@pytest.mark.parametrize("mode", [O.MODE_RECT, O.MODE_CSG])
def test_transmission_lengths_hex_lattice_by_closed_form(rot30, mode):
    """Per-material lengths through a rings-3 hex lattice of pins (vacuum):
    the exit is the first point outside every hexagon (brute force over all
    elements at the face-plane crossings along the ray; the lattice's outline
    is not convex) and the fuel length is the sum over elements of the chord
    through the pin at q a1 + r a2, clipped to that exit."""
    rings, pitch, r_pin, height = 3, 1.0, 0.4, 5.0
    desc = I.small_hex(rings=rings, pitch=pitch, r_pin=r_pin, height=height, rot30=rot30)
    hx = desc["universes"][1]
    a1, a2, nrm, hp = np.array(hx["a1"]), np.array(hx["a2"]), np.array(hx["normals"]), hx["half_pitch"]
    centres = np.array([q * a1 + r * a2 for q, r in I.hex_elements(rings)])

    def inside(pt):
        rel = pt[None, :2] - centres
        return bool((np.abs(rel @ nrm.T) <= hp).all(1).any()) and 0.0 <= pt[2] <= height

    rng = np.random.default_rng(23)
    m, rays = 120, []
    while len(rays) < m:
        c = centres[rng.integers(len(centres))]
        xy = c + rng.uniform(-hp, hp, 2)
        pt = np.array([xy[0], xy[1], rng.uniform(0.0, height)])
        if not (np.abs((xy - c) @ nrm.T) < hp).all():
            continue
        w = rng.normal(size=3)
        rays.append(np.concatenate([pt, w / np.linalg.norm(w)]))
    rays = np.array(rays)
    res = _geom(desc, mode).transmission(rays, np.array(desc["sigma"]), grad=False)
    assert (res["status"] == 2).all()
    jmax = 4 * (rings + 2)
    for k in range(m):
        o, d = rays[k, :3], rays[k, 3:]
        t_z = (height - o[2]) / d[2] if d[2] > 0 else (-o[2] / d[2] if d[2] < 0 else np.inf)
        cuts = [t_z]
        for nk in nrm:
            on, dn = nk @ o[:2], nk @ d[:2]
            if dn != 0.0:
                cuts += [(j * hp - on) / dn for j in range(-jmax, jmax + 1)]
        cuts = np.unique([t for t in cuts if 0.0 < t <= t_z])
        t_exit, prev = t_z, 0.0
        for t in cuts:
            if not inside(o + 0.5 * (prev + t) * d):
                t_exit = prev
                break
            prev = t
        fuel = sum(_inside_cylinder(o, d, c[0], c[1], r_pin, t_exit) for c in centres)
        expect = np.array([fuel, t_exit - fuel])
        assert np.allclose(res["lens"][k], expect, rtol=1e-12, atol=1e-11), (k, res["lens"][k], expect)


def _chords(o, d, cx, cy, r, t_end):
    """Summed length of {t in [0, t_end]} inside each cylinder (centres cx, cy,
    radius r).  Far pins make b^2 - a c cancel (both ~|q|^2), so the chord is
    taken from the point of closest approach p = q - ((q.w)/a) w instead:
    t in t_c -+ sqrt((r^2 - |p|^2) / a)."""
    qx, qy = o[0] - cx, o[1] - cy
    a = d[0] * d[0] + d[1] * d[1]
    if a == 0.0:
        return t_end * np.count_nonzero(qx * qx + qy * qy < r * r)
    tc = -(qx * d[0] + qy * d[1]) / a
    px, py = qx + tc * d[0], qy + tc * d[1]
    h2 = (r * r - (px * px + py * py)) / a
    s = np.sqrt(np.maximum(h2, 0.0))
    seg = np.minimum(tc + s, t_end) - np.maximum(tc - s, 0.0)
    return float(np.where(h2 > 0.0, np.maximum(seg, 0.0), 0.0).sum())


@pytest.mark.parametrize("mode", [O.MODE_RECT, O.MODE_CSG])
def test_transmission_lengths_three_level_core_by_closed_form(mode):
    """The benchmark's three-level core (15 x 15 assemblies of 17 x 17 pins in
    the r = 170 cylinder): boundary rays' per-material lengths against chords
    through every pin at (core element centre + assembly element centre),
    fuel or guide tube as the description's assembly fill says, clipped to
    the exit from the cylinder and its caps (convex, so the first exit)."""
    desc = I.config2()
    n_core, n_assm, pitch, R, H = 15, 17, 1.26, 170.0, 366.0
    rf, rc, rg = 0.41, 0.475, 0.56
    fill = np.array(desc["universes"][2]["fill"])
    ca = (np.arange(n_assm) - n_assm / 2.0 + 0.5) * pitch
    cc = (np.arange(n_core) - n_core / 2.0 + 0.5) * n_assm * pitch
    px = (cc[:, None] + ca[None, :]).ravel()            # all pin x centres (core i, pin a)
    gx, gy = np.meshgrid(px, px, indexing="xy")
    ai = np.tile(np.arange(n_assm), n_core)              # pin index within its assembly along x
    ei = (ai[None, :] + n_assm * ai[:, None])            # element index i + 17 j (i fastest)
    guide = fill[ei] == 1
    fx, fy = gx[~guide], gy[~guide]
    tx, ty = gx[guide], gy[guide]
    rays = I.boundary_rays(60, r_outer=R, height=H, seed=41).packed()
    res = _geom(desc, mode).transmission(rays, np.array(desc["sigma"]), grad=False)
    assert (res["status"] == 2).all()
    for k in range(len(rays)):
        o, d = rays[k, :3], rays[k, 3:]
        t_z = (H - o[2]) / d[2] if d[2] > 0 else (-o[2] / d[2] if d[2] < 0 else np.inf)
        a = d[0] ** 2 + d[1] ** 2
        b = o[0] * d[0] + o[1] * d[1]
        c = o[0] ** 2 + o[1] ** 2 - R * R
        t_r = (-b + math.sqrt(b * b - a * c)) / a if a > 0 else np.inf
        t_exit = min(t_z, t_r)
        fuel = _chords(o, d, fx, fy, rf, t_exit)
        clad = _chords(o, d, fx, fy, rc, t_exit) - fuel
        tube = _chords(o, d, tx, ty, rg, t_exit)
        expect = np.array([fuel, clad, t_exit - fuel - clad - tube, tube])
        # ~500 chord ends per ray, each within a few ulp of a 300 cm path: 2e-10 cm is 5x the
        # largest difference seen over 200 rays
        assert np.allclose(res["lens"][k], expect, rtol=0.0, atol=2e-10), (k, res["lens"][k], expect)


def _crossings(o, d, cx, cy, r, t_end):
    """Parameters t in (0, t_end) where the ray crosses the cylinders
    (centres cx, cy, radius r), from the closest approach."""
    qx, qy = o[0] - cx, o[1] - cy
    a = d[0] * d[0] + d[1] * d[1]
    if a == 0.0:
        return np.zeros(0)
    tc = -(qx * d[0] + qy * d[1]) / a
    px, py = qx + tc * d[0], qy + tc * d[1]
    h2 = (r * r - (px * px + py * py)) / a
    hit = h2 > 0.0
    s = np.sqrt(h2[hit])
    t = np.concatenate([tc[hit] - s, tc[hit] + s])
    return t[(t > 0.0) & (t < t_end)]


@pytest.mark.parametrize("mode", [O.MODE_RECT, O.MODE_CSG])
def test_straight_histories_segment_sequence_three_level_core(mode):
    """Absolute segment counts and lengths on the benchmark's three-level core.
    With every sigma = 0 a history is a straight ray from its birth point to
    the vacuum boundary, and its segments end exactly where the ray crosses a
    surface that bounds its cell: each pin cylinder (fuel and clad, or guide
    tube), each pin-pitch plane inside the core square (an assembly's outer
    face is the core lattice's plane: one crossing), the core square's four
    planes anywhere inside the cylinder (they also bound the moderator
    fillers), then the r = 170 cylinder or a z plane.  The segment lengths are
    the gaps between the sorted crossings; the count is their number + 1."""
    n_core, n_assm, pitch, R, H = 15, 17, 1.26, 170.0, 366.0
    desc = I.config2(sigma=[0.0, 0.0, 0.0, 0.0])
    g = _geom(desc, mode)
    fill = np.array(desc["universes"][2]["fill"])
    ca = (np.arange(n_assm) - n_assm / 2.0 + 0.5) * pitch
    cc = (np.arange(n_core) - n_core / 2.0 + 0.5) * n_assm * pitch
    pc = (cc[:, None] + ca[None, :]).ravel()
    gx, gy = np.meshgrid(pc, pc, indexing="xy")
    ai = np.tile(np.arange(n_assm), n_core)
    guide = fill[ai[None, :] + n_assm * ai[:, None]] == 1
    half = n_core * n_assm * pitch / 2.0
    planes = -half + pitch * np.arange(n_core * n_assm + 1)
    births, st = g.source(150, 3)
    assert (st == 0).all()
    total = 0
    for pid in range(len(births)):
        o, d = births[pid, :3], births[pid, 3:6]
        t_z = (H - o[2]) / d[2] if d[2] > 0 else (-o[2] / d[2] if d[2] < 0 else np.inf)
        a, b = d[0] ** 2 + d[1] ** 2, o[0] * d[0] + o[1] * d[1]
        c = o[0] ** 2 + o[1] ** 2 - R * R
        t_exit = min(t_z, (-b + math.sqrt(b * b - a * c)) / a if a > 0 else np.inf)
        ts = [_crossings(o, d, gx[~guide], gy[~guide], 0.41, t_exit),
              _crossings(o, d, gx[~guide], gy[~guide], 0.475, t_exit),
              _crossings(o, d, gx[guide], gy[guide], 0.56, t_exit)]
        for ax in (0, 1):
            if d[ax] == 0.0:
                continue
            t = (planes - o[ax]) / d[ax]
            t = t[(t > 0.0) & (t < t_exit)]
            other = np.abs(o[1 - ax] + t * d[1 - ax])
            outer = (np.abs(t * d[ax] + o[ax]) > half - 0.5 * pitch)      # the square's own planes
            ts.append(t[(other < half) | outer])
        cuts = np.sort(np.concatenate(ts))
        expect = np.diff(np.concatenate([[0.0], cuts, [t_exit]]))
        inst, ln, kind, status = g.trace(pid, 3, 0.3)
        assert status == O.P_ESCAPED and (kind == 0).all()
        assert len(ln) == len(expect), (pid, len(ln), len(expect))
        assert np.allclose(ln, expect, rtol=0.0, atol=2e-10), pid
        total += len(ln)
    assert total > 150 * 100      # paths cross hundreds of surfaces on average


def _hex_holder(pts, centres, nrm, hp):
    """Index of the hexagon (centres, face normals, half pitch) whose interior
    holds each 2-D point, -1 for none: brute force over every hexagon."""
    proj = np.abs((pts[:, None, :] - centres[None, :, :]) @ nrm.T)
    inside = (proj < hp).all(-1)
    return np.where(inside.any(1), inside.argmax(1), -1)


def _plane_cuts(o2, d2, nrm, hp, lo, hi, jmax):
    """t in (lo, hi) where o2 + t d2 crosses a face plane n_k . x = j hp."""
    out = []
    for nk in nrm:
        dn = nk @ d2
        if dn != 0.0:
            t = (np.arange(-jmax, jmax + 1) * hp - nk @ o2) / dn
            out.append(t[(t > lo) & (t < hi)])
    return np.concatenate(out) if out else np.zeros(0)


@pytest.mark.parametrize("mode", [O.MODE_RECT, O.MODE_CSG])
def test_straight_histories_segment_sequence_hex_core(mode):
    """The hex core (127 assemblies of 127-element pin lattices turned by 30
    degrees, pins in rings 0-5, ring 6 a fill clipped by the assembly
    hexagon) with every sigma = 0: each history's segments against a
    computation that never walks the geometry.  All candidate crossings
    (face planes of the core lattice, face planes of the pin lattice of each
    assembly the path enters, pin cylinders) split the straight path; the
    identity of each piece (assembly hexagon, pin hexagon within it, inside
    the pin or not) comes from brute-force classification of its midpoint; a
    segment ends exactly where that identity changes (a face plane through
    element centres splits nothing), and the path ends at the first piece
    outside every assembly or at a z plane."""
    desc = I.config3(sigma=[0.0] * 5)
    g = _geom(desc, mode)
    U = desc["universes"]
    core, assm = U[-1], U[-2]
    a1c, a2c, nrmc, hpc = np.array(core["a1"]), np.array(core["a2"]), np.array(core["normals"]), core["half_pitch"]
    a1p, a2p, nrmp, hpp = np.array(assm["a1"]), np.array(assm["a2"]), np.array(assm["normals"]), assm["half_pitch"]
    H = core["z"][1]
    cc = np.array([q * a1c + r * a2c for q, r in I.hex_elements(core["rings"])])
    pe = np.array([q * a1p + r * a2p for q, r in I.hex_elements(assm["rings"])])
    has_pin = np.array([f != 3 for f in assm["fill"]])
    r_pin = desc["surfaces"][0]["coef"][2]
    births, st = g.source(100, 5)
    assert (st == 0).all()
    total = 0
    for pid in range(len(births)):
        o, d = births[pid, :3], births[pid, 3:6]
        o2, d2 = o[:2], d[:2]
        t_z = (H - o[2]) / d[2] if d[2] > 0 else (-o[2] / d[2] if d[2] < 0 else np.inf)
        cuts = np.unique(np.concatenate([[0.0], _plane_cuts(o2, d2, nrmc, hpc, 0.0, t_z, 60), [t_z]]))
        asm = _hex_holder(o2 + 0.5 * (cuts[:-1] + cuts[1:])[:, None] * d2, cc, nrmc, hpc)
        assert asm[0] >= 0
        out = np.flatnonzero(asm < 0)
        t_exit = cuts[out[0]] if out.size else t_z
        cand = [cuts[(cuts > 0.0) & (cuts < t_exit)]]
        for A in np.unique(asm[asm >= 0]):
            span = np.flatnonzero(asm == A)
            lo, hi = cuts[span.min()], min(cuts[span.max() + 1], t_exit)
            oa = o2 - cc[A]
            cand.append(_plane_cuts(oa, d2, nrmp, hpp, lo, hi, 30))
            cand.append(_crossings(np.array([oa[0], oa[1], 0.0]), d, pe[has_pin, 0], pe[has_pin, 1], r_pin, hi))
        pts = np.unique(np.concatenate(cand))
        pts = pts[(pts > 0.0) & (pts < t_exit)]
        edges = np.concatenate([[0.0], pts, [t_exit]])
        mid = o2 + 0.5 * (edges[:-1] + edges[1:])[:, None] * d2
        ia = _hex_holder(mid, cc, nrmc, hpc)
        assert (ia >= 0).all()
        local = mid - cc[ia]
        ip = _hex_holder(local, pe, nrmp, hpp)
        assert (ip >= 0).all()
        rr = np.hypot(*(local - pe[ip]).T)
        inpin = has_pin[ip] & (rr < r_pin)
        ident = np.stack([ia, ip, inpin.astype(int)], 1)
        change = np.flatnonzero((ident[1:] != ident[:-1]).any(1))
        bounds = np.concatenate([[0.0], pts[change], [t_exit]])
        expect = np.diff(bounds)
        inst, ln, kind, status = g.trace(pid, 5, 0.3)
        assert status == O.P_ESCAPED and (kind == 0).all()
        assert len(ln) == len(expect), (pid, len(ln), len(expect))
        assert np.allclose(ln, expect, rtol=0.0, atol=1e-10), pid
        total += len(ln)
    assert total > 100 * 50


@pytest.mark.parametrize("member", _members_by_kind())
@pytest.mark.parametrize("mode", [O.MODE_RECT, O.MODE_CSG])
def test_straight_histories_against_brute_force_batch_members(member, mode):
    """Configuration-4 members (rect and hex lattices, two and three levels)
    with every sigma = 0: along each straight history, points at 2..98% of
    every segment lie in that segment's cell instance by brute force over
    every leaf in the global frame (a missed crossing would put some in
    another cell), consecutive segments lie in different cells, every
    segment ends on a bounding surface of its cell (an extra crossing or a
    wrong length would not), and past the last one the path is outside
    every cell (vacuum)."""
    desc, _ = I.config4_member(member)
    desc = dict(desc, sigma=[0.0] * len(desc["sigma"]))
    g = _geom(desc, mode)
    births, st = g.source(40, 11)
    assert (st == 0).all()
    fr = np.array([0.02, 0.25, 0.5, 0.75, 0.98])
    nseg = 0
    for pid in range(len(births)):
        o, d = births[pid, :3], births[pid, 3:6]
        inst, ln, kind, status = g.trace(pid, 11, 0.3)
        assert status == O.P_ESCAPED and (kind == 0).all() and (ln > 0).all()
        t0 = np.concatenate([[0.0], np.cumsum(ln)[:-1]])
        pts = o + (t0[:, None] + fr[None, :] * ln[:, None]).reshape(-1, 1) * d
        bi, cnt, _, _ = g.find_cell_brute(pts)
        assert np.array_equal(bi.reshape(-1, len(fr)), np.repeat(inst[:, None], len(fr), 1)), pid
        assert (cnt == 1).all()
        assert (inst[1:] != inst[:-1]).all()
        ends = o + np.cumsum(ln)[:-1, None] * d
        if len(ends):
            _, _, near, _ = g.find_cell_brute(ends - 1e-12 * d)
            assert near.max() < 1e-9, pid
        past, _, _, _ = g.find_cell_brute((o + (ln.sum() + 1e-7) * d)[None, :])
        assert past[0] == -1
        nseg += len(ln)
    assert nseg > 40 * 3


def _uniform2(pid, event, tag, k, seed, gid):
    """Two doubles in (0, 1] from Philox4x32-10 with key (seed_lo32, geometry
    id) and counter (particle, event, tag, k): xi = ((u64 >> 11) + 1) 2^-53
    for u64 = (c1 << 32) | c0 and (c3 << 32) | c2."""
    c = [int(x) for x in O.philox4x32_10([pid, event, tag, k], [seed & 0xffffffff, gid])]
    return [(((c[hi] << 32 | c[lo]) >> 11) + 1) * 2.0 ** -53 for lo, hi in ((0, 1), (2, 3))]


def _marsaglia(pid, event, seed, gid):
    for k in range(64):
        xa, xb = _uniform2(pid, event, 1, k, seed, gid)
        u, v = 2.0 * xa - 1.0, 2.0 * xb - 1.0
        s = u * u + v * v
        if 0.0 < s < 1.0:
            w = math.sqrt(1.0 - s)
            return np.array([2.0 * u * w, 2.0 * v * w, 1.0 - 2.0 * s])
    raise AssertionError("no direction in 64 attempts")


def _leaf_materials(desc):
    """Material of every leaf cell instance in the tally numbering: a
    universe's cells in order (a daughter contributes all of its instances in
    place), rect elements i fastest, then j, then k, hex elements in rows
    r = -R..R with q ascending."""
    U = desc["universes"]

    def walk(u):
        un = U[u]
        if un["type"] == "csg":
            out = []
            for c in un["cells"]:
                out += [c["material"]] if "material" in c else walk(c["fill"])
            return out
        return [m for f in un["fill"] for m in walk(f)]
    return np.array(walk(desc["root"]))


def _box_reflect(half, height):
    def reflect(end, w):
        for ax, lo, hi in ((0, -half, half), (1, -half, half), (2, 0.0, height)):
            if abs(end[ax] - hi) < 1e-9 or abs(end[ax] - lo) < 1e-9:
                w[ax] = -w[ax]
    return reflect


# (geometry, absorption, histories, reflection rule, membership by brute force?)  The full-size
# benchmark core has 191,929 leaves: there membership comes from the hierarchical find_cell (pinned
# against brute force on the same geometry) and crossing ends from distance_to_surface (pinned by
# hand-worked rays), instead of brute force per point.
FLIGHT_CASES = {
    "config1_reflecting": (lambda: I.config1(), 0.3, 120, _box_reflect(17 * 1.26 / 2.0, 100.0), True),
    "three_level_core": (lambda: I.small_core(), 0.25, 80, None, True),
    "config3_hex_core": (lambda: I.config3(), 0.25, 25, None, True),
    "config2_full_core": (lambda: I.config2(), 0.25, 400, None, False),
}
for _m in _members_by_kind():     # configuration-4 members: rect and hex lattices, two and three levels
    FLIGHT_CASES[f"config4_member{_m}"] = (lambda _m=_m: I.config4_member(_m)[0], 0.3, 100, None, False)


@pytest.mark.parametrize("case", list(FLIGHT_CASES))
@pytest.mark.parametrize("mode", [O.MODE_RECT, O.MODE_CSG])
def test_histories_with_collisions_follow_the_flight_rules(case, mode):
    """Whole histories re-derived from the flight rules of Alg. 2 without the
    oracle's walk: from the birth state, each segment's material comes from
    its instance (numbering rebuilt here from the description); a collision
    flight is exactly tau / Sigma and a crossing is shorter; tau loses
    Sigma l at each crossing; at the e-th collision the absorption test, the
    new tau and the Marsaglia direction come from the Philox counters
    (pid, e, 2, 0) and (pid, e, 1, k); a crossing that ends on a reflecting
    box face reverses that component.  Along the path rebuilt this way,
    points at 2..98% of every segment lie in the segment's instance by brute
    force over every leaf, crossings end on a bounding surface, and an
    escaping history's path then leaves every cell."""
    make, pa, n, reflect, brute = FLIGHT_CASES[case]
    desc = make()
    g = _geom(desc, mode)
    sigma = np.array(desc["sigma"])
    mat = _leaf_materials(desc)
    assert len(mat) == g.n_inst
    seed, gid = 13, desc["geometry_id"]
    births, st = g.source(n, seed)
    fr = np.array([0.02, 0.25, 0.5, 0.75, 0.98])
    ncoll = 0
    for pid in range(len(births)):
        r, w, tau = births[pid, :3].copy(), births[pid, 3:6].copy(), births[pid, 6]
        inst, ln, kind, status = g.trace(pid, seed, pa)
        assert status in (O.P_ABSORBED, O.P_ESCAPED)
        pts, ends, past = [], [], None
        event = 0
        for k in range(len(ln)):
            sig = sigma[mat[inst[k]]]
            dc = tau / sig
            pts.append(r + (fr * ln[k])[:, None] * w)
            end = r + ln[k] * w
            if kind[k] == 1:
                assert abs(ln[k] - dc) <= 1e-12 * dc, (pid, k)
                event += 1
                ncoll += 1
                xa, xt = _uniform2(pid, event, 2, 0, seed, gid)
                if xa < pa:
                    assert k == len(ln) - 1 and status == O.P_ABSORBED, (pid, k)
                    break
                w = _marsaglia(pid, event, seed, gid)
                tau = -math.log(xt)
            else:
                assert kind[k] == 0 and ln[k] < dc * (1 + 1e-12), (pid, k)
                tau = tau - sig * ln[k]
                ends.append((end - 1e-12 * w, end - 1e-9 * w, w.copy()))
                if k == len(ln) - 1:
                    assert status == O.P_ESCAPED
                    past = end + 1e-7 * w
                elif reflect is not None:
                    reflect(end, w)
            r = end
        m = len(inst) * len(fr)
        if brute:
            # one brute-force pass per history: points along the segments, just
            # before each crossing, and past the exit
            q = np.concatenate(pts + [np.array([e[0] for e in ends]).reshape(-1, 3),
                                      np.zeros((0, 3)) if past is None else past[None, :]])
            bi, cnt, near, _ = g.find_cell_brute(q)
            assert (near[m:m + len(ends)] < 1e-9).all(), pid
        else:
            q = np.concatenate(pts + [np.zeros((0, 3)) if past is None else past[None, :]])
            bi = g.find_cell(q)
            if ends:
                dd, _, di = g.distance(np.array([e[1] for e in ends]), np.array([e[2] for e in ends]))
                assert np.all(np.abs(dd - 1e-9) < 1e-11), pid      # the boundary ahead is the crossing
                assert np.array_equal(di, inst[kind[:len(inst)] == 0][:len(ends)]), pid
        assert np.array_equal(bi[:m].reshape(-1, len(fr)), np.repeat(inst[:, None], len(fr), 1)), (pid, case)
        if past is not None:
            assert bi[-1] == -1
    assert ncoll > n


def _chord_end_rates(o, d, cx, cy, r, t_end, pitch):
    """For cylinders (centres cx, cy, radius r) the sums over the chord ends
    inside (0, t_end) of dt_end/dr and dt_end/dpitch, signed so that they add
    up to d(length inside)/dtheta, with the centres at k pitch.  An end at
    t = tc -+ s (s the half chord in t, P the closest-approach vector, w the
    xy direction, a = |w|^2) moves by -+ (r/a)/s with r, and by
    (w.c -+ P.c/s) / (a pitch) with the pitch; the entering end counts with
    a minus sign.  Ends at 0 or t_end (fixed boundaries) do not move."""
    qx, qy = o[0] - cx, o[1] - cy
    wx, wy = d[0], d[1]
    a = wx * wx + wy * wy
    tc = -(qx * wx + qy * wy) / a
    px, py = qx + tc * wx, qy + tc * wy
    h2 = (r * r - (px * px + py * py)) / a
    hit = h2 > 0.0
    s = np.sqrt(np.where(hit, h2, 1.0))
    t1, t2 = tc - s, tc + s
    wc = (wx * cx + wy * cy) / a
    pc = (px * cx + py * cy) / (a * s)
    dr = dp = 0.0
    inner = hit & (t1 > 0.0) & (t1 < t_end)        # entering end inside the path
    outer = hit & (t2 > 0.0) & (t2 < t_end)        # leaving end inside the path
    dr += ((r / a) / s)[inner].sum() + ((r / a) / s)[outer].sum()
    dp += (-(wc - pc) / pitch)[inner].sum() + ((wc + pc) / pitch)[outer].sum()
    return dr, dp, float(np.min(s[hit & (inner | outer)], initial=np.inf))


def test_transmission_gradient_by_closed_form():
    """The analytic transmission gradient (reading c19) against the
    derivative of the closed-form chords on the reduced three-level core:
    per material, d l / d r_j is the sum over moving chord ends of (r/a)/s
    (fuel gains what clad loses, guide interior what moderator loses), and
    d l / d pitch moves every pin centre c = k pitch; the outer cylinder and
    the z planes are fixed, and the core-square planes separate moderator
    from moderator.  dT/dtheta = -T sum_m sigma_m d l_m / d theta."""
    pitch, n_core, n_assm, height = 1.26, 3, 5, 20.0
    r_out = 0.5 * n_core * n_assm * pitch * 1.2
    sigma = np.array([0.9, 0.4, 0.2, 0.6])
    desc = I.small_core(height=height, r_outer=r_out, sigma=sigma)
    rays = I.boundary_rays(300, r_outer=r_out, height=height, seed=8).packed()
    res = _geom(desc).transmission(rays, sigma, pitch=pitch)
    fill = np.array(desc["universes"][2]["fill"])
    ca = (np.arange(n_assm) - n_assm / 2.0 + 0.5) * pitch
    cc = (np.arange(n_core) - n_core / 2.0 + 0.5) * n_assm * pitch
    pc = (cc[:, None] + ca[None, :]).ravel()
    gx, gy = np.meshgrid(pc, pc, indexing="xy")
    ai = np.tile(np.arange(n_assm), n_core)
    guide = fill[ai[None, :] + n_assm * ai[:, None]] == 1
    checked = 0
    for k in range(len(rays)):
        o, d = rays[k, :3], rays[k, 3:]
        if d[0] * d[0] + d[1] * d[1] == 0.0:
            continue
        t_z = (height - o[2]) / d[2] if d[2] > 0 else (-o[2] / d[2] if d[2] < 0 else np.inf)
        a = d[0] ** 2 + d[1] ** 2
        b = o[0] * d[0] + o[1] * d[1]
        t_exit = min(t_z, (-b + math.sqrt(b * b - a * (o[0] ** 2 + o[1] ** 2 - r_out ** 2))) / a)
        drf, dpf, sf = _chord_end_rates(o, d, gx[~guide], gy[~guide], 0.41, t_exit, pitch)
        drc, dpc, sc = _chord_end_rates(o, d, gx[~guide], gy[~guide], 0.475, t_exit, pitch)
        drg, dpg, sg = _chord_end_rates(o, d, gx[guide], gy[guide], 0.56, t_exit, pitch)
        if min(sf, sc, sg) < 1e-3:
            continue                      # near-tangent chords: the rates grow like 1/s
        # d l_m / d theta for theta = (r_fuel, r_clad, r_guide, pitch); materials 0 fuel, 1 clad, 2 moderator, 3 guide
        dl = np.array([[drf, 0.0, 0.0, dpf],
                       [-drf, drc, 0.0, dpc - dpf],
                       [0.0, -drc, -drg, -dpc - dpg],
                       [0.0, 0.0, drg, dpg]])
        expect = -res["T"][k] * (sigma @ dl)
        got = res["dT"][k, 4:]
        # rounding: relative to the terms summed, plus 1e-12 T for the core-square planes, whose
        # moderator-to-moderator crossings cancel in the oracle's per-crossing sum up to rounding
        scale = res["T"][k] * (np.abs(sigma)[:, None] * np.abs(dl)).sum(0)
        assert np.all(np.abs(got - expect) <= 1e-10 * scale + 1e-12 * res["T"][k]), (k, got, expect)
        checked += 1
    assert checked > 200


def test_transmission_geometry_gradient_vs_fd():
    base = dict(n_core=3, n_assm=5, height=20.0)
    r_out = 0.5 * 3 * 5 * 1.26 * 1.2
    rays = I.boundary_rays(400, r_outer=r_out, height=20.0, seed=4).packed()
    sigma = np.array([0.9, 0.4, 0.2, 0.6])
    h = 1e-6
    params = dict(r_fuel=0.41, r_clad=0.475, r_guide=0.56, pitch=1.26)

    def run(**kw):
        p = dict(params, **kw)
        desc = I.small_core(**base, r_outer=r_out, sigma=sigma, **p)
        return _geom(desc).transmission(rays, sigma, pitch=p["pitch"])

    ref = run()
    names = ["r_fuel", "r_clad", "r_guide", "pitch"]

    def fd_err(j, nm, step):
        hi_ = run(**{nm: params[nm] + step})
        lo_ = run(**{nm: params[nm] - step})
        same = (hi_["hash"] == ref["hash"]) & (lo_["hash"] == ref["hash"])
        fd = (hi_["T"] - lo_["T"]) / (2 * step)
        an = ref["dT"][:, 4 + j]
        scale = np.maximum(np.abs(an), 1e-3 * ref["T"])
        return np.abs(fd - an) / scale, same, an

    for j, nm in enumerate(names):
        err, same, an = fd_err(j, nm, h)
        assert same.mean() > 0.95
        assert np.any(np.abs(an[same]) > 0), nm
        assert np.median(err[same]) < 1e-7, nm
        assert np.quantile(err[same], 0.99) < 1e-4, nm
        # the residual is central-difference truncation: it shrinks like h^2
        err10, same10, _ = fd_err(j, nm, 10 * h)
        both = same & same10
        big = both & (err10 > 1e-6)
        if big.any():
            assert np.median(err[big] / err10[big]) < 0.05, nm


# ---------------------------------------------------------------------------
# superimposed mesh track-length tally
# ---------------------------------------------------------------------------

def _clip_len(r, d, length, lo, hi):
    """Length of the segment r + t d, 0 <= t <= length, inside the box
    [lo, hi] (slab clipping, an independent computation)."""
    t0, t1 = 0.0, length
    for a in range(3):
        if d[a] == 0.0:
            if not (lo[a] <= r[a] <= hi[a]):
                return 0.0
            continue
        ta, tb = (lo[a] - r[a]) / d[a], (hi[a] - r[a]) / d[a]
        t0, t1 = max(t0, min(ta, tb)), min(t1, max(ta, tb))
    return max(0.0, t1 - t0)


def test_mesh_segment_against_box_clipping():
    # random segments, many starting outside the mesh, against the length
    # inside each bin box by slab clipping (brute force over all bins)
    d = I.with_mesh(I.single_pin(), 4, 3, 5, box=[-0.5, -0.4, 1.0, 0.7, 0.5, 8.0])
    o = _geom(d, O.MODE_CSG)
    gx, gy, gz = d["mesh"]["grid"]
    rng = np.random.default_rng(7)
    for _ in range(200):
        r = rng.uniform([-1.0, -1.0, 0.0], [1.0, 1.0, 10.0])
        v = rng.normal(size=3)
        v /= np.linalg.norm(v)
        length = rng.uniform(0.0, 6.0)
        got = o.mesh_segment(r, v, length).astype(np.float64) / 2**32
        exp = np.zeros(len(got))
        for k in range(5):
            for j in range(3):
                for i in range(4):
                    exp[i + 4 * (j + 3 * k)] = _clip_len(r, v, length, (gx[i], gy[j], gz[k]),
                                                         (gx[i + 1], gy[j + 1], gz[k + 1]))
        assert np.abs(got - exp).max() <= 1e-9, (r, v, length)


def test_mesh_segment_along_an_axis():
    # a segment along +x from the middle of bin 0 for 3.5 bin widths: pieces
    # of half, one, one and one width (closed form), nothing elsewhere
    d = I.with_mesh(I.single_pin(), 8, 2, 2, box=[0.0, 0.0, 0.0, 8.0, 2.0, 2.0])
    o = _geom(d, O.MODE_CSG)
    got = o.mesh_segment([0.5, 0.5, 0.5], [1.0, 0.0, 0.0], 3.5)
    exp = np.zeros(32, np.uint64)
    exp[0] = 2**31
    exp[1:4] = 2**32
    assert np.array_equal(got, exp)
    # the same backwards from the far side, starting outside the mesh
    got = o.mesh_segment([9.0, 1.5, 1.5], [-1.0, 0.0, 0.0], 3.0)
    exp = np.zeros(32, np.uint64)
    exp[7 + 8 * (1 + 2 * 1)] = 2**32
    exp[6 + 8 * (1 + 2 * 1)] = 2**32
    assert np.array_equal(got, exp)


def test_mesh_total_equals_track_length():
    # every segment lies in the geometry, which the mesh covers: the mesh
    # tally's total is the cell tally's total up to each piece's rounding to
    # 2^-32 cm
    for d in (I.with_mesh(I.config1(), 17, 17, 10), I.with_mesh(I.small_core(), 9, 7, 5)):
        r = _geom(d, O.MODE_RECT).run_mesh(2000, 1, 0.3, threads=4)
        a = float(r["mesh"].sum()) / 2**32
        b = float(r["tally"].sum()) / 2**32
        assert abs(a - b) <= 1e-9 * b
        assert (r["mesh"] > 0).mean() > 0.5


# ---------------------------------------------------------------------------
# power iteration with the synthetic fission source
# ---------------------------------------------------------------------------

def test_power_infinite_medium_k_equals_nu():
    # one material everywhere, reflecting box: every history ends in an
    # absorption, so every cycle's estimate is nu exactly; after the first
    # cycle (normalised by k = 1) each history banks floor(1 + xi) = 1 site
    d = I.with_nu(I.config1(sigma=(0.5, 0.5, 0.5)), (2.5, 2.5, 2.5))
    n = 2000
    r = _geom(d).power(n, 1, 0.3, 2, 5, threads=4)
    assert r["ok"] and np.all(r["k"] == 2.5)
    assert np.all(r["bank"][1:] == n)
    assert abs(r["bank"][0] - 2.5 * n) <= 5 * np.sqrt(n)


def test_power_bank_size_matches_estimate():
    # E[sites] = sum(nu) / k_prev = n k_c / k_{c-1}; each history's count
    # varies by less than one site
    d = I.with_nu(I.small_core(), (2.4, 0.0, 0.0, 0.0))
    n = 20_000
    r = _geom(d).power(n, 1, 0.25, 2, 6, threads=8)
    assert r["ok"]
    k, b = r["k"], r["bank"]
    assert abs(b[0] - n * k[0]) <= 5 * np.sqrt(n)
    for c in range(1, 6):
        assert abs(b[c] - n * k[c] / k[c - 1]) <= 5 * np.sqrt(n), c
    assert 0.3 < k.mean() < 2.4


@pytest.mark.parametrize("mode", [O.MODE_RECT, O.MODE_CSG])
def test_power_first_cycle_exact(mode):
    """Cycle 0 of Alg. 1's iteration re-derived history by history: its
    particles are the source's (ids 0..n-1), each history that ends in an
    absorption at its e-th collision in a material with yield nu > 0 banks
    min(8, floor(nu / 1 + xi)) sites (xi from Philox counter (pid, e, 3, 0))
    and adds llrint(nu 2^32) to the cycle's production; k_0 is that integer
    sum times 2^-32 over n."""
    nu = (2.4, 0.0, 1.3, 0.0)
    desc = I.with_nu(I.small_core(), nu)
    g = _geom(desc, mode)
    n, seed, pa = 400, 3, 0.25
    r = g.power(n, seed, pa, 1, 2)
    assert r["ok"]
    mat = _leaf_materials(desc)
    sites, prod = 0, 0
    for pid in range(n):
        inst, ln, kind, status = g.trace(pid, seed, pa)
        if status != O.P_ABSORBED:
            continue
        m = mat[inst[-1]]
        if nu[m] > 0.0:
            e = int((kind == 1).sum())
            xf, _ = _uniform2(pid, e, 3, 0, seed, desc["geometry_id"])
            sites += min(8, int(math.floor(nu[m] / 1.0 + xf)))
            prod += int(np.rint(nu[m] * 4294967296.0))
    assert r["bank"][0] == sites
    assert r["k"][0] == (float(prod) * 2.0 ** -32) / n
    assert sites > n // 2


@pytest.mark.parametrize("mode", [O.MODE_RECT, O.MODE_CSG])
def test_power_second_cycle_exact(mode):
    """Cycle 1 of the power iteration rebuilt from cycle 0: the bank is the
    absorption points of cycle 0's fissile absorptions in history order (each
    point rebuilt here from the birth state, the traced segment lengths and
    the Marsaglia directions of the collision counters), repeated by its site
    count; particle i of cycle 1 (id n + i) takes site floor(xi B) with xi
    from counter (pid, 0, 4, 0), and its own history, traced from that site,
    banks floor(nu / k_0 + xi) sites.  Bank size and k of cycle 1 must equal
    the iteration's."""
    nu = (2.4, 0.0, 1.3, 0.0)
    desc = I.with_nu(I.small_core(), nu)
    g = _geom(desc, mode)
    n, seed, pa = 300, 3, 0.25
    gid = desc["geometry_id"]
    r = g.power(n, seed, pa, 1, 2)
    assert r["ok"]
    mat = _leaf_materials(desc)
    births, _ = g.source(n, seed)
    bank = []
    for pid in range(n):
        inst, ln, kind, status = g.trace(pid, seed, pa)
        if status != O.P_ABSORBED or nu[mat[inst[-1]]] <= 0.0:
            continue
        pos, w, e = births[pid, :3].copy(), births[pid, 3:6].copy(), 0
        for k in range(len(ln)):
            pos = pos + ln[k] * w
            if kind[k] == 1:
                e += 1
                if k < len(ln) - 1:
                    w = _marsaglia(pid, e, seed, gid)
        xf, _ = _uniform2(pid, e, 3, 0, seed, gid)
        bank += [pos] * min(8, int(math.floor(nu[mat[inst[-1]]] / 1.0 + xf)))
    assert len(bank) == r["bank"][0]
    k0, nb = r["k"][0], len(bank)
    sites = prod = 0
    for i in range(n):
        pid = n + i
        xb, _ = _uniform2(pid, 0, 4, 0, seed, gid)
        site = bank[min(int(math.floor(xb * nb)), nb - 1)]
        inst, ln, kind, status = g.trace_from_site(pid, seed, pa, k0, site)
        if status != O.P_ABSORBED or nu[mat[inst[-1]]] <= 0.0:
            continue
        e = int((kind == 1).sum())
        xf, _ = _uniform2(pid, e, 3, 0, seed, gid)
        sites += min(8, int(math.floor(nu[mat[inst[-1]]] / k0 + xf)))
        prod += int(np.rint(nu[mat[inst[-1]]] * 4294967296.0))
    assert r["bank"][1] == sites
    assert r["k"][1] == (float(prod) * 2.0 ** -32) / n


def test_power_deterministic_and_sharded_threads():
    d = I.with_nu(I.config1(), (2.0, 0.0, 0.0))
    a = _geom(d).power(3000, 3, 0.3, 1, 3, threads=1)
    b = _geom(d).power(3000, 3, 0.3, 1, 3, threads=7)
    assert np.array_equal(a["k"], b["k"]) and np.array_equal(a["bank"], b["bank"])
    assert np.array_equal(a["tally"], b["tally"])


def test_power_without_fissile_material_stops():
    r = _geom(I.config1()).power(500, 1, 0.3, 1, 3)
    assert not r["ok"] and r["k"][0] == 0.0


# ---------------------------------------------------------------------------
# distance_to_surface from points (the diagnostic entry)
# ---------------------------------------------------------------------------

def _c1_distance_brute(p, w, pitch=1.26, n=17, radii=(0.41, 0.475), height=100.0):
    """Configuration 1 by hand in the global frame: the element's four side
    faces, the box's z planes and the pin's two cylinders (smallest positive
    root of the quadratic); returns (distance, level: 0 faces, 1 cylinders)."""
    grid = np.array([(i - n / 2.0) * pitch for i in range(n + 1)])
    cand = []
    for d in range(2):
        i = int(np.searchsorted(grid, p[d], side="right") - 1)
        if w[d] > 0:
            cand.append(((grid[i + 1] - p[d]) / w[d], 0))
        elif w[d] < 0:
            cand.append(((grid[i] - p[d]) / w[d], 0))
    if w[2] > 0:
        cand.append(((height - p[2]) / w[2], 0))
    elif w[2] < 0:
        cand.append(((0.0 - p[2]) / w[2], 0))
    ix = int(np.searchsorted(grid, p[0], side="right") - 1)
    iy = int(np.searchsorted(grid, p[1], side="right") - 1)
    cx, cy = 0.5 * (grid[ix] + grid[ix + 1]), 0.5 * (grid[iy] + grid[iy + 1])
    qx, qy = p[0] - cx, p[1] - cy
    a = w[0] ** 2 + w[1] ** 2
    b = qx * w[0] + qy * w[1]
    for r in radii:
        c = qx * qx + qy * qy - r * r
        disc = b * b - a * c
        if a > 0 and disc > 0:
            for t in ((-b - np.sqrt(disc)) / a, (-b + np.sqrt(disc)) / a):
                if t > 1e-12:
                    cand.append((t, 1))
                    break
    cand.sort()
    return cand[0][0], cand[0][1], (cand[1][0] if len(cand) > 1 else np.inf)


@pytest.mark.parametrize("mode", [O.MODE_RECT, O.MODE_CSG])
def test_distance_against_hand_computed_config1(mode):
    # random points and isotropic directions: the oracle's hierarchical
    # distance equals the global-frame closed forms (ties excluded)
    rng = np.random.default_rng(11)
    n = 3000
    xyz = np.column_stack([rng.uniform(-10.7, 10.7, n), rng.uniform(-10.7, 10.7, n), rng.uniform(0.1, 99.9, n)])
    w = rng.normal(size=(n, 3))
    w /= np.linalg.norm(w, axis=1)[:, None]
    d, lev, inst = _geom(I.config1(), mode).distance(xyz, w)
    checked = 0
    for k in range(n):
        t, l, t2 = _c1_distance_brute(xyz[k], w[k])
        if t2 - t < 1e-9 * max(1.0, t):
            continue
        assert abs(d[k] - t) <= 1e-12 * max(1.0, t), (k, d[k], t)
        assert lev[k] == l and inst[k] >= 0
        checked += 1
    assert checked > 0.99 * n


def test_distance_closed_forms_and_outside():
    g = _geom(I.config1(), O.MODE_RECT)
    # from a pin's axis the fuel cylinder lies r / sqrt(u^2 + v^2) away
    c = 0.5 * ((0 - 8.5) * 1.26 + (1 - 8.5) * 1.26)      # centre of element 8
    xyz = np.array([[0.0, 0.0, 50.0], [c, c, 50.0], [c, 0.0, 20.0], [0.0, 0.0, 50.0]])
    w = np.array([[1.0, 0.0, 0.0], [0.6, 0.0, 0.8], [0.0, -1.0, 0.0], [0.0, 0.0, 1.0]])
    d, lev, _ = g.distance(xyz, w)
    assert abs(d[0] - 0.41) <= 1e-15 and lev[0] == 1
    assert abs(d[1] - 0.41 / 0.6) <= 1e-15 and lev[1] == 1
    assert abs(d[2] - 0.41) <= 1e-15 and lev[2] == 1
    # straight up the axis: the top of the box, at the root level
    assert d[3] == 50.0 and lev[3] == 0
    # outside the box: NaN, no level, no cell
    d, lev, inst = g.distance(np.array([[11.0, 0.0, 5.0]]), np.array([[1.0, 0.0, 0.0]]))
    assert np.isnan(d[0]) and lev[0] == -1 and inst[0] == -1


def test_distance_rect_and_csg_modes_identical():
    # pseudo-array planes are the lattice's own grid values in the same frames
    rng = np.random.default_rng(12)
    for desc in (I.small_core(), I.random_tiny(5)):
        lo, hi = np.array(desc["source_box"][:3]), np.array(desc["source_box"][3:])
        xyz = lo + rng.uniform(size=(2000, 3)) * (hi - lo)
        w = rng.normal(size=(2000, 3))
        w /= np.linalg.norm(w, axis=1)[:, None]
        a = _geom(desc, O.MODE_RECT).distance(xyz, w)
        b = _geom(desc, O.MODE_CSG).distance(xyz, w)
        assert np.array_equal(a[0], b[0], equal_nan=True) and np.array_equal(a[1], b[1])
        assert np.array_equal(a[2], b[2])


# ---------------------------------------------------------------------------
# test infrastructure of the near-surface rule: the oracle's segment geometry
# and its clearance query
# ---------------------------------------------------------------------------

def test_trace_geometry_chains_through_collisions():
    # each segment starts where the previous one ended (same FP64 operations:
    # r + len * dir per component), births are source_init's, and after a
    # collision the direction is the Marsaglia direction of that event
    desc = I.config1()
    o = O.Geometry(I.to_json(desc), O.MODE_CSG)
    births, _ = o.source(40, 1)
    for pid in range(40):
        inst, ln, kind, st, geo = o.trace(pid, 1, 0.3, geometry=True)
        assert np.array_equal(geo[0, :3], births[pid, :3]) and np.array_equal(geo[0, 3:6], births[pid, 3:6])
        event = 0
        for k in range(len(ln) - 1):
            end = geo[k, :3] + ln[k] * geo[k, 3:6]
            assert np.array_equal(geo[k + 1, :3], end)
            if kind[k] == 1:
                event += 1
                d, ok = O.isotropic(pid, event, 1, desc["geometry_id"])
                assert ok and np.array_equal(geo[k + 1, 3:6], d)
            else:
                # a crossing keeps the direction except at a reflecting wall,
                # where one component changes sign
                flip = geo[k + 1, 3:6] != geo[k, 3:6]
                assert flip.sum() <= 1 and np.array_equal(np.abs(geo[k + 1, 3:6]), np.abs(geo[k, 3:6]))


def test_clearance_by_hand_single_pin():
    # one pin (cylinders r = 0.41, 0.475 about the z axis) in the box
    # [-0.63, 0.63]^2 x [0, 10]: distances worked by hand
    o = O.Geometry(I.to_json(I.single_pin(bc="vacuum")), O.MODE_CSG)
    pts = np.array([[0.2, 0.0, 5.0], [0.41, 0.0, 5.0], [0.6, 0.0, 9.99], [0.0, 0.3, 0.001]])
    cl = o.clearance(pts, np.tile([1.0, 0.0, 0.0], (4, 1)), np.zeros(4))
    want = [(0.21, 0.275), (0.0, 0.065), (0.01, 0.03), (0.001, 0.11)]
    for (c1, c2), row in zip(want, cl):
        assert row[0] == pytest.approx(c1, abs=1e-12) and row[1] == pytest.approx(c2, abs=1e-12)
        # the end point of a zero-length segment is its start
        assert row[2] == row[0] and row[3] == row[1]
    # end point: 0.5 cm along +x from (0.2, 0, 5) is (0.7, 0, 5), outside the
    # box by 0.07; the nearest surface is the x = 0.63 face
    cl = o.clearance(pts[:1], np.array([[1.0, 0.0, 0.0]]), np.array([0.5]))
    assert cl[0, 2] == pytest.approx(0.07, abs=1e-12) and cl[0, 3] == pytest.approx(0.225, abs=1e-12)


def test_clearance_tangency_by_hand():
    o = O.Geometry(I.to_json(I.single_pin(bc="vacuum")), O.MODE_CSG)
    # a line along +x at impact parameter b passes closest to the axis at x = 0
    for b in (0.4, 0.47, 0.2):
        start = np.array([[-0.5, b, 5.0]])
        cl = o.clearance(start, np.array([[1.0, 0.0, 0.0]]), np.array([1.0]))
        assert cl[0, 4] == pytest.approx(min(abs(b - 0.41), abs(b - 0.475)), abs=1e-12)
        # the closest approach lies beyond a shorter segment: no tangency
        cl = o.clearance(start, np.array([[1.0, 0.0, 0.0]]), np.array([0.4]))
        assert cl[0, 4] == np.inf
    # an oblique ray: the xy projection decides; (-0.3, 0.45) + t (0.6, 0)
    # is closest to the axis at t = 0.5 (x = 0), distance 0.45
    cl = o.clearance(np.array([[-0.3, 0.45, 2.0]]), np.array([[0.6, 0.0, 0.8]]), np.array([1.0]))
    assert cl[0, 4] == pytest.approx(0.025, abs=1e-12)
    # a ray along the axis direction has no xy closest approach
    cl = o.clearance(np.array([[0.1, 0.1, 2.0]]), np.array([[0.0, 0.0, 1.0]]), np.array([3.0]))
    assert cl[0, 4] == np.inf


def test_clearance_general_planes_hex():
    # a hex lattice element's faces are general planes n.x = d: a point at the
    # element centre plus s along a face normal is (pitch/2 - s) from that face
    desc = I.small_hex(rings=0, pitch=1.0, r_pin=0.3)
    o = O.Geometry(I.to_json(desc), O.MODE_CSG)
    a1, a2, nrm = I._hex_frame(1.0, rot30=False)
    nx, ny = nrm[0]
    s = 0.42
    pt = np.array([[s * nx, s * ny, 2.5]])
    cl = o.clearance(pt, np.array([[0.0, 0.0, 1.0]]), np.zeros(1))
    # nearest: the face at 0.5 - 0.42 = 0.08; then the pin at 0.42 - 0.3 = 0.12
    assert cl[0, 0] == pytest.approx(0.08, abs=1e-12)
    assert cl[0, 1] == pytest.approx(0.12, abs=1e-12)


def test_trace_comparison_flags_planted_mistakes():
    # the near-surface comparison (oracle.compare) on the oracle's own traces:
    # identical rows match; a changed instance or a length off by 1e-7 cm
    # fails (the decision points are not near any surface); a length change
    # far below the propagated rounding bound still matches
    from oracle import compare as C
    desc = I.config1()
    o = O.Geometry(I.to_json(desc), O.MODE_CSG)
    n, cap = 60, 2048
    rows_i = np.full((n, cap), -1, np.int32)
    rows_l = np.zeros((n, cap))
    for pid in range(n):
        inst, ln, kind, st = o.trace(pid, 1, 0.3, cap=cap)
        rows_i[pid, :len(inst)] = inst
        rows_l[pid, :len(ln)] = ln
    res = C.compare_traces(o, np.arange(n), rows_i, rows_l, 1, 0.3, cap)
    assert res["matched"] == n and not res["failed"]
    long_ = [p for p in range(n) if (rows_i[p] >= 0).sum() > 12]
    a, b, c = long_[:3]
    bad_i, bad_l = rows_i.copy(), rows_l.copy()
    # a different cell after segment 6 (the neighbour's instance number)
    bad_i[a, 7] = bad_i[a, 7] + 1 if bad_i[a, 7] + 1 != bad_i[a, 6] else bad_i[a, 7] + 2
    bad_l[b, 4] += 1e-7
    bad_l[c, 4] *= 1.0 + 1e-15
    res = C.compare_traces(o, np.array([a, b, c]), bad_i[[a, b, c]], bad_l[[a, b, c]], 1, 0.3, cap)
    failed = {r["pid"] for r in res["failed"]}
    assert failed == {a, b} and res["matched"] == 1
    # a history cut short (one segment missing at the end) is a mismatch too
    short_i, short_l = rows_i[[a]].copy(), rows_l[[a]].copy()
    k = int((short_i[0] >= 0).sum())
    short_i[0, k - 1] = -1
    res = C.compare_traces(o, np.array([a]), short_i, short_l, 1, 0.3, cap)
    assert res["matched"] == 0
