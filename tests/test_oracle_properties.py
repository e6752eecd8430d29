"""Property tests of the oracle on randomly drawn small geometries (CPU).

A geometry is a rect lattice (1..3 x 1..3 x 1..2 elements, pitch 1..2 cm) of
one pin universe: 1..3 concentric cylinders about a common offset centre,
materials 0, 1, 2 inside them and 3 outside.  Properties:
  - hierarchical find_cell equals brute force over every leaf instance in
    the global frame (both modes), away from surfaces;
  - transmission lengths per material equal closed-form chords through
    every pin, clipped to the box exit (vacuum box);
  - the rect and CSG modes give identical histories.
Hex lattices (rings 0..3, either orientation) of pins of one cylinder are
drawn too: find_cell against brute force, and transmission lengths against
chords clipped at the first exit from the union of hexagons.
"""
import numpy as np
import pytest

hyp = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

import oracle as O  # noqa: E402
from paper_2406_13849_gb300 import inputs as I  # noqa: E402


@st.composite
def pin_lattices(draw, bc=None):
    ncyl = draw(st.integers(1, 3))
    pitch = draw(st.floats(1.0, 2.0))
    fr = sorted(draw(st.lists(st.floats(0.05, 0.45), min_size=ncyl, max_size=ncyl, unique=True)))
    if any(b - a < 1e-3 for a, b in zip(fr, fr[1:])):
        fr = [0.05 + 0.4 * (k + 1) / (ncyl + 1) for k in range(ncyl)]
    radii = [f * pitch for f in fr]
    off = draw(st.floats(-0.03, 0.03)), draw(st.floats(-0.03, 0.03))
    nx, ny, nz = draw(st.integers(1, 3)), draw(st.integers(1, 3)), draw(st.integers(1, 2))
    bcs = [bc or draw(st.sampled_from(["vacuum", "reflect"])) for _ in range(6)]
    S = [{"type": "cz", "coef": [off[0], off[1], r]} for r in radii]
    cells = [{"surfaces": [[0, -1]], "material": 0}]
    cells += [{"surfaces": [[k - 1, 1], [k, -1]], "material": k % 3} for k in range(1, ncyl)]
    cells.append({"surfaces": [[ncyl - 1, 1]], "material": 3})
    gx = [(i - nx / 2.0) * pitch for i in range(nx + 1)]
    gy = [(j - ny / 2.0) * pitch for j in range(ny + 1)]
    gz = [k * 2.5 for k in range(nz + 1)]
    desc = {"format": I.FORMAT, "name": "prop", "geometry_id": draw(st.integers(0, 9)),
            "sigma": [draw(st.floats(0.05, 1.5)) for _ in range(4)], "surfaces": S,
            "universes": [{"type": "csg", "cells": cells},
                          {"type": "rect", "grid": [gx, gy, gz], "fill": [0] * (nx * ny * nz), "bc": bcs}],
            "root": 1, "source_box": [gx[0], gy[0], gz[0], gx[-1], gy[-1], gz[-1]]}
    return desc, radii, off


@settings(max_examples=40, deadline=None, derandomize=True, database=None)
@given(geo=pin_lattices(), seed=st.integers(0, 2**31))
def test_find_cell_equals_brute_force(geo, seed):
    desc, _, _ = geo
    lo, hi = np.array(desc["source_box"][:3]), np.array(desc["source_box"][3:])
    pts = lo - 0.1 + np.random.default_rng(seed).uniform(size=(400, 3)) * (hi - lo + 0.2)
    for mode in (O.MODE_RECT, O.MODE_CSG):
        g = O.Geometry(I.to_json(desc), mode)
        inst = g.find_cell(pts)
        bi, cnt, near, _ = g.find_cell_brute(pts)
        far = near > 1e-9
        assert np.array_equal(inst[far], bi[far])
        assert (cnt[far] <= 1).all()


@settings(max_examples=30, deadline=None, derandomize=True, database=None)
@given(geo=pin_lattices(bc="vacuum"), seed=st.integers(0, 2**31))
def test_transmission_lengths_equal_chords(geo, seed):
    desc, radii, off = geo
    lo, hi = np.array(desc["source_box"][:3]), np.array(desc["source_box"][3:])
    rng = np.random.default_rng(seed)
    m = 40
    org = lo + rng.uniform(0.01, 0.99, (m, 3)) * (hi - lo)
    w = rng.normal(size=(m, 3))
    w /= np.linalg.norm(w, axis=1)[:, None]
    res = O.Geometry(I.to_json(desc), O.MODE_CSG).transmission(np.concatenate([org, w], 1), desc["sigma"],
                                                                grad=False)
    gx, gy = desc["universes"][1]["grid"][0], desc["universes"][1]["grid"][1]
    cx = np.array([(gx[i] + gx[i + 1]) / 2 + off[0] for i in range(len(gx) - 1) for _ in range(len(gy) - 1)])
    cy = np.array([(gy[j] + gy[j + 1]) / 2 + off[1] for _ in range(len(gx) - 1) for j in range(len(gy) - 1)])
    for k in range(m):
        o, d = org[k], w[k]
        t_exit = min(((hi[a] if d[a] > 0 else lo[a]) - o[a]) / d[a] for a in range(3) if d[a] != 0.0)
        inside = [_chords(o, d, cx, cy, r, t_exit) for r in radii]
        lens = np.zeros(4)
        lens[0] += inside[0]
        for j in range(1, len(radii)):
            lens[j % 3] += inside[j] - inside[j - 1]
        lens[3] += t_exit - inside[-1]
        assert np.allclose(res["lens"][k], lens, rtol=0.0, atol=1e-11), (k, res["lens"][k], lens)


@settings(max_examples=25, deadline=None, derandomize=True, database=None)
@given(geo=pin_lattices(), seed=st.integers(1, 2**31), pa=st.floats(0.05, 0.9))
def test_rect_and_csg_modes_identical(geo, seed, pa):
    desc, _, _ = geo
    ra = O.Geometry(I.to_json(desc), O.MODE_RECT).run(200, seed, pa)
    rb = O.Geometry(I.to_json(desc), O.MODE_CSG).run(200, seed, pa)
    assert np.array_equal(ra["hash"], rb["hash"]) and np.array_equal(ra["tally"], rb["tally"])
    assert np.array_equal(ra["counters"], rb["counters"])


def _chords(o, d, cx, cy, r, t_end):
    """Summed length of {t in [0, t_end]} inside each cylinder (closest-approach form)."""
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


@st.composite
def hex_lattices(draw):
    rings = draw(st.integers(0, 3))
    pitch = draw(st.floats(0.5, 2.0))
    rot30 = draw(st.booleans())
    r_pin = draw(st.floats(0.1, 0.45)) * pitch
    off = draw(st.floats(-0.02, 0.02)) * pitch, draw(st.floats(-0.02, 0.02)) * pitch
    height = draw(st.floats(1.0, 6.0))
    desc = I.small_hex(rings=rings, pitch=pitch, r_pin=r_pin, height=height, rot30=rot30,
                       sigma=(draw(st.floats(0.05, 1.5)), draw(st.floats(0.05, 1.5))))
    desc["surfaces"][0]["coef"][:2] = [off[0], off[1]]
    return desc, r_pin, off


@settings(max_examples=30, deadline=None, derandomize=True, database=None)
@given(geo=hex_lattices(), seed=st.integers(0, 2**31))
def test_hex_find_cell_equals_brute_force(geo, seed):
    desc, _, _ = geo
    lo, hi = np.array(desc["source_box"][:3]), np.array(desc["source_box"][3:])
    pts = lo + np.random.default_rng(seed).uniform(size=(400, 3)) * (hi - lo)
    for mode in (O.MODE_RECT, O.MODE_CSG):
        g = O.Geometry(I.to_json(desc), mode)
        bi, cnt, near, _ = g.find_cell_brute(pts)
        far = near > 1e-9
        assert np.array_equal(g.find_cell(pts)[far], bi[far])
        assert (cnt[far] <= 1).all()


@settings(max_examples=25, deadline=None, derandomize=True, database=None)
@given(geo=hex_lattices(), seed=st.integers(0, 2**31))
def test_hex_transmission_lengths_equal_chords(geo, seed):
    desc, r_pin, off = geo
    hx = desc["universes"][1]
    a1, a2, nrm, hp = np.array(hx["a1"]), np.array(hx["a2"]), np.array(hx["normals"]), hx["half_pitch"]
    height = hx["z"][1]
    centres = np.array([q * a1 + r * a2 for q, r in I.hex_elements(hx["rings"])])

    def holder(pts):
        proj = np.abs((pts[:, None, :] - centres[None, :, :]) @ nrm.T)
        inside = (proj < hp).all(-1)
        return np.where(inside.any(1), inside.argmax(1), -1)

    rng = np.random.default_rng(seed)
    m = 30
    el = rng.integers(0, len(centres), m)
    org = np.zeros((m, 3))
    for k in range(m):
        while True:       # a point inside the drawn element's hexagon
            xy = centres[el[k]] + rng.uniform(-hp, hp, 2)
            if (np.abs((xy - centres[el[k]]) @ nrm.T) < hp).all():
                break
        org[k] = [xy[0], xy[1], rng.uniform(0.0, height)]
    w = rng.normal(size=(m, 3))
    w /= np.linalg.norm(w, axis=1)[:, None]
    for mode in (O.MODE_RECT, O.MODE_CSG):
        res = O.Geometry(I.to_json(desc), mode).transmission(np.concatenate([org, w], 1), desc["sigma"], grad=False)
        for k in range(m):
            o, d = org[k], w[k]
            t_z = (height - o[2]) / d[2] if d[2] > 0 else (-o[2] / d[2] if d[2] < 0 else np.inf)
            cuts = [t_z]
            for nk in nrm:
                dn = nk @ d[:2]
                if dn != 0.0:
                    cuts += list((np.arange(-40, 41) * hp - nk @ o[:2]) / dn)
            cuts = np.unique([t for t in cuts if 0.0 < t <= t_z])
            mids = np.concatenate([[0.0], cuts[:-1]]) + 0.5 * np.diff(np.concatenate([[0.0], cuts]))
            out = np.flatnonzero(holder(o[:2] + mids[:, None] * d[:2]) < 0)
            t_exit = (np.concatenate([[0.0], cuts])[out[0]]) if out.size else t_z
            fuel = _chords(o, d, centres[:, 0] + off[0], centres[:, 1] + off[1], r_pin, t_exit)
            assert np.allclose(res["lens"][k], [fuel, t_exit - fuel], rtol=0.0, atol=1e-11), (mode, k)
