"""Cylinder tests that the kernels first decide in FP32 (the sense of a point
against a cylinder, and the distance scan's screen that skips an upper-level
cylinder lying beyond the running best) must give the FP64 decision every
time.  These points are placed where those certificates are most likely to
be wrong: at relative distances 1e-16..1e-2 from every pin radius of the
benchmark's three-level core and from its r = 170 outer cylinder, and just
inside the outer cylinder, where its distance and the lower levels' best
distance are of the same size.  find_cell and distance_to_surface of the
--fmad=false build must equal the oracle's bit for bit."""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2406_13849_gb300 import inputs as I
from paper_2406_13849_gb300 import native as N

pytestmark = pytest.mark.gpu

N_CORE, N_ASSM, PITCH, R_OUT, HEIGHT = 15, 17, 1.26, 170.0, 366.0


def _near_cylinders(desc, n, seed):
    rng = np.random.default_rng(seed)
    fill = np.array(desc["universes"][2]["fill"])
    ci, cj = rng.integers(0, N_CORE, (2, n))
    a, b = rng.integers(0, N_ASSM, (2, n))
    guide = fill[a + N_ASSM * b] == 1
    cx = (ci - N_CORE / 2.0 + 0.5) * N_ASSM * PITCH + (a - N_ASSM / 2.0 + 0.5) * PITCH
    cy = (cj - N_CORE / 2.0 + 0.5) * N_ASSM * PITCH + (b - N_ASSM / 2.0 + 0.5) * PITCH
    r = np.where(guide, 0.56, rng.choice([0.41, 0.475], n))
    outer = rng.uniform(size=n) < 0.25
    cx[outer], cy[outer], r[outer] = 0.0, 0.0, R_OUT
    rel = 10.0 ** rng.uniform(-16.0, -2.0, n) * rng.choice([-1.0, 1.0], n)
    rho = r * (1.0 + rel)
    phi = rng.uniform(0.0, 2.0 * math.pi, n)
    xyz = np.stack([cx + rho * np.cos(phi), cy + rho * np.sin(phi), rng.uniform(0.0, HEIGHT, n)], 1)
    return xyz


def _inside_outer(n, seed):
    rng = np.random.default_rng(seed)
    rho = R_OUT - rng.uniform(0.0, 2.0, n)
    phi = rng.uniform(0.0, 2.0 * math.pi, n)
    return np.stack([rho * np.cos(phi), rho * np.sin(phi), rng.uniform(0.0, HEIGHT, n)], 1)


def _directions(n, seed):
    w = np.random.default_rng(seed).normal(size=(n, 3))
    return w / np.linalg.norm(w, axis=1)[:, None]


@pytest.mark.parametrize("tracker,mode", [(N.TRACKER_RECT, O.MODE_RECT), (N.TRACKER_CSG, O.MODE_CSG)])
def test_find_cell_at_cylinder_surfaces(tracker, mode):
    desc = I.config2()
    xyz = _near_cylinders(desc, 200_000, 31)
    ref = O.Geometry(I.to_json(desc), mode).find_cell(xyz)
    g = N.Geometry(I.to_json(desc), exact=True)
    got = g.find_cell(torch.from_numpy(xyz).cuda(), tracker=tracker).cpu().numpy()
    assert np.array_equal(got, ref)
    assert (ref < 0).any() and (ref >= 0).mean() > 0.7


@pytest.mark.parametrize("tracker,mode", [(N.TRACKER_RECT, O.MODE_RECT), (N.TRACKER_CSG, O.MODE_CSG)])
def test_distance_at_cylinder_surfaces_and_screen_threshold(tracker, mode):
    desc = I.config2()
    xyz = np.concatenate([_near_cylinders(desc, 60_000, 32), _inside_outer(60_000, 33)])
    w = _directions(len(xyz), 34)
    od, ol, oi = O.Geometry(I.to_json(desc), mode).distance(xyz, w)
    g = N.Geometry(I.to_json(desc), exact=True)
    d, lev, inst = g.distance_to_surface(torch.from_numpy(xyz).cuda(), torch.from_numpy(w).cuda(), tracker=tracker)
    torch.cuda.synchronize()
    gd, gl, gi = d.cpu().numpy(), lev.cpu().numpy(), inst.cpu().numpy()
    assert np.array_equal(gi, oi) and np.array_equal(gl, ol)
    assert np.array_equal(gd, od, equal_nan=True)
    # the outer cylinder wins from some of the points just inside it: the screen's threshold is crossed
    band = np.arange(len(xyz)) >= 60_000
    assert ((ol == 0) & band).sum() > 100 and ((ol > 0) & band).sum() > 100


def _near_tangent(xyz, n_frac, seed):
    """Directions: isotropic, except a fraction turned nearly perpendicular
    to the radius of the nearest pin axis (grazing rays)."""
    rng = np.random.default_rng(seed)
    n = len(xyz)
    w = _directions(n, seed)
    k = rng.uniform(size=n) < n_frac
    # radial direction from the nearest pin axis (the 15 x 17 = 255 pins per
    # row are centred on the origin: axes at multiples of the pitch)
    cx = np.round(xyz[:, 0] / PITCH) * PITCH
    cy = np.round(xyz[:, 1] / PITCH) * PITCH
    rx, ry = xyz[:, 0] - cx, xyz[:, 1] - cy
    rn = np.hypot(rx, ry) + 1e-300
    tx, ty = -ry / rn, rx / rn
    tilt = 10.0 ** rng.uniform(-9.0, -1.0, n) * rng.choice([-1.0, 1.0], n)
    wz = rng.uniform(-0.9, 0.9, n)
    sxy = np.sqrt(1.0 - wz * wz)
    gx, gy = tx + tilt * rx / rn, ty + tilt * ry / rn
    gn = np.hypot(gx, gy)
    w[k] = np.stack([sxy * gx / gn, sxy * gy / gn, wz], 1)[k]
    return w


def test_fast_build_distances_near_cylinders_and_tangents():
    # the fast build (contracted multiply-adds) near every cylinder of the
    # core and at grazing incidence, where the cylinder formulas lose the
    # most digits: every distance within 1e-12 of the oracle's (relative to
    # the coordinates' size) with the same winning level, unless the oracle
    # confirms a decision near a surface (oracle.compare.classify_distances)
    from oracle import compare as C
    desc = I.config2()
    xyz = np.concatenate([_near_cylinders(desc, 100_000, 41), _inside_outer(20_000, 42)])
    w = _near_tangent(xyz, 0.5, 43)
    o = O.Geometry(I.to_json(desc), O.MODE_CSG)
    od, ol, oi = o.distance(xyz, w)
    g = N.Geometry(I.to_json(desc), exact=False)
    d, lev, inst = g.distance_to_surface(torch.from_numpy(xyz).cuda(), torch.from_numpy(w).cuda(),
                                         tracker=N.TRACKER_CSG)
    torch.cuda.synchronize()
    gd, gl, gi = d.cpu().numpy(), lev.cpu().numpy(), inst.cpu().numpy()
    diff = np.nonzero(gi != oi)[0]
    if len(diff):
        cl = o.clearance(xyz[diff], w[diff], np.zeros(len(diff)))
        assert (cl[:, 0] < C.NEAR).all(), cl[:, 0]
    same = gi == oi
    res = C.classify_distances(o, xyz[same], w[same], od[same], ol[same], gd[same], gl[same])
    print(f"\npoints {res['points']}, outside the bar {res['outside_bar']}, near {len(res['near'])}, "
          f"failed {len(res['failed'])}, max rel within bar {res['max_rel_within_bar']:.3g}, cell differs {len(diff)}")
    assert not res["failed"], res["failed"][:5]
