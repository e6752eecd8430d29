"""Seeded synthetic inputs: nested-geometry descriptions and ray sets.

This module is the only code shared by the CUDA path and the CPU oracle.  It
writes explicit FP64 numbers (grid planes, radii, lattice vectors, sigma) into
a JSON description and draws the deterministic ray set of the transmission
workload.  It contains none of the tracking arithmetic: no distances, no
containment tests, no translations of frames.

Description format ("nested-csg-geometry-v1"), the nested universes of the
paper's Sec. 1 (Table 1, Fig. 3) and Sec. 3.2:

  sigma       per-material constant attenuation coefficient (1/cm)
  surfaces    list of {"type": "px"|"py"|"pz"|"p"|"cz", "coef": [...],
              optional "bc": "vacuum"|"reflect", "rparam": k, "pscale": 1}
                px/py/pz: [g]            plane x=g (y=g, z=g)
                p:        [nx,ny,nz,d]   plane n.x = d
                cz:       [x0,y0,r]      cylinder about z
  universes   list of
                {"type": "csg", "cells": [{"surfaces": [[sid, +1|-1], ...],
                 "material": m} | {..., "fill": u, "translation": [x,y,z]}]}
                {"type": "rect", "grid": [[x0..xn],[y0..yn],[z0..zn]],
                 "fill": [u per element, i fastest, then j, then k],
                 "bc": [xlo,xhi,ylo,yhi,zlo,zhi], "pscale": 0|1}
                {"type": "hex", "rings": R, "a1": [x,y], "a2": [x,y],
                 "normals": [[x,y],[x,y],[x,y]], "half_pitch": h,
                 "z": [z0,z1], "fill": [u per element, rows r=-R..R,
                 q ascending], "bc": [side, zlo, zhi]}
  root        index of the root universe
  source_box  [xlo,ylo,zlo,xhi,yhi,zhi] of the uniform birth distribution

The optional "rparam"/"pscale" tags name the design parameters a surface
depends on (pin radii, lattice pitch) for the transmission gradient.

Other optional keys: "geometry_id" (integer in [0, 2^31), keys the random
numbers), "accel" ("bvh" or "bih"), "nu" (fission yield per material, in
[0, 7]) and "mesh" ({"grid": [x planes, y planes, z planes]}).

The builder rejects (TRK_E_DESC) a description in which a universe is not
reached from the root, an index (surface, material, universe) is out of
range or not an integer, a sense is not +1/-1, "rparam" is not -1, 0, 1 or
2, "pscale" is not 0 or 1, a coordinate is not finite, or the JSON nests
more than 64 deep.
"""
from __future__ import annotations

import json
import math
from dataclasses import dataclass

import numpy as np

FORMAT = "nested-csg-geometry-v1"

SQRT3_2 = math.sqrt(3.0) / 2.0


def to_json(desc: dict) -> str:
    """Serialise a description; floats use Python's shortest round-trip repr."""
    return json.dumps(desc, separators=(",", ":"))


def hex_elements(rings: int):
    """Axial (q, r) of a hex lattice with rings 0..R, rows r=-R..R, q ascending."""
    out = []
    for r in range(-rings, rings + 1):
        for q in range(max(-rings, -rings - r), min(rings, rings - r) + 1):
            out.append((q, r))
    return out


def hex_ring(q: int, r: int) -> int:
    return max(abs(q), abs(r), abs(q + r))


def _hex_frame(pitch: float, rot30: bool):
    """Lattice vectors and face normals of a hex lattice (explicit FP64 numbers).

    Without rotation e1=(1,0), e2=(1/2,sqrt3/2); with rot30 the lattice is turned
    by 30 degrees: e1=(sqrt3/2,1/2), e2=(0,1).  Face normals are e1, e2, e2-e1.
    """
    if rot30:
        e1 = (SQRT3_2, 0.5)
        e2 = (0.0, 1.0)
        n2 = (-SQRT3_2, 0.5)
    else:
        e1 = (1.0, 0.0)
        e2 = (0.5, SQRT3_2)
        n2 = (-0.5, SQRT3_2)
    a1 = [pitch * e1[0], pitch * e1[1]]
    a2 = [pitch * e2[0], pitch * e2[1]]
    return a1, a2, [list(e1), list(e2), list(n2)]


# ---------------------------------------------------------------------------
# Config 1: 17x17 pin lattice in a reflecting box
# ---------------------------------------------------------------------------

def config1(sigma=(0.8, 0.3, 0.1), pitch=1.26, n=17, r_fuel=0.41, r_clad=0.475,
            height=100.0, bc="reflect", geometry_id=0) -> dict:
    """One n x n square lattice of 3-cell pins filling a box with reflecting sides."""
    half = n / 2.0
    grid_xy = [(i - half) * pitch for i in range(n + 1)]
    surfaces = [
        {"type": "cz", "coef": [0.0, 0.0, r_fuel], "rparam": 0},
        {"type": "cz", "coef": [0.0, 0.0, r_clad], "rparam": 1},
    ]
    pin = {"type": "csg", "cells": [
        {"surfaces": [[0, -1]], "material": 0},
        {"surfaces": [[0, 1], [1, -1]], "material": 1},
        {"surfaces": [[1, 1]], "material": 2},
    ]}
    root = {"type": "rect", "grid": [grid_xy, list(grid_xy), [0.0, height]],
            "fill": [0] * (n * n), "bc": [bc] * 6, "pscale": 1}
    return {
        "format": FORMAT, "name": f"pin_lattice_{n}x{n}", "geometry_id": geometry_id,
        "sigma": [float(s) for s in sigma], "surfaces": surfaces,
        "universes": [pin, root], "root": 1,
        "source_box": [grid_xy[0], grid_xy[0], 0.0, grid_xy[-1], grid_xy[-1], height],
    }


# ---------------------------------------------------------------------------
# Config 2 (and the transmission geometry): core of 15x15 assemblies of 17x17 pins
# ---------------------------------------------------------------------------

def config2(n_core=15, n_assm=17, pitch=1.26, r_fuel=0.41, r_clad=0.475, r_guide=0.56,
            r_outer=170.0, height=366.0, sigma=None, guide_frac=0.05, seed=1,
            geometry_id=0) -> dict:
    """Three-level nested rectilinear core inside a vacuum-bounded cylinder.

    Levels: root CSG (core box clipped by the cylinder, plus 4 convex moderator
    fillers) -> core rect lattice -> assembly rect lattice -> pin CSG.  Pin
    universes have no box; the assembly lattice's pitch planes bound them.
    Materials: 0 fuel, 1 clad, 2 moderator, 3 guide-tube interior.
    """
    if sigma is None:
        sigma = np.random.default_rng(seed).uniform(0.05, 1.0, size=4)
    n_pins = n_assm * n_assm
    n_guides = int(round(guide_frac * n_pins))
    guides = set(int(i) for i in np.random.default_rng(seed).permutation(n_pins)[:n_guides])

    ha = n_assm / 2.0
    assm_pitch = n_assm * pitch
    hc = n_core / 2.0
    grid_a = [(j - ha) * pitch for j in range(n_assm + 1)]
    grid_c = [(i - hc) * assm_pitch for i in range(n_core + 1)]
    lo, hi = grid_c[0], grid_c[-1]

    S = []
    def surf(t, coef, **kw):
        S.append(dict({"type": t, "coef": coef}, **kw))
        return len(S) - 1
    s_fuel = surf("cz", [0.0, 0.0, r_fuel], rparam=0, pscale=1)
    s_clad = surf("cz", [0.0, 0.0, r_clad], rparam=1, pscale=1)
    s_guide = surf("cz", [0.0, 0.0, r_guide], rparam=2, pscale=1)
    s_xlo = surf("px", [lo], pscale=1)
    s_xhi = surf("px", [hi], pscale=1)
    s_ylo = surf("py", [lo], pscale=1)
    s_yhi = surf("py", [hi], pscale=1)
    s_zlo = surf("pz", [0.0], bc="vacuum")
    s_zhi = surf("pz", [height], bc="vacuum")
    s_cyl = surf("cz", [0.0, 0.0, r_outer], bc="vacuum")

    fuel_pin = {"type": "csg", "cells": [
        {"surfaces": [[s_fuel, -1]], "material": 0},
        {"surfaces": [[s_fuel, 1], [s_clad, -1]], "material": 1},
        {"surfaces": [[s_clad, 1]], "material": 2},
    ]}
    guide_pin = {"type": "csg", "cells": [
        {"surfaces": [[s_guide, -1]], "material": 3},
        {"surfaces": [[s_guide, 1]], "material": 2},
    ]}
    half_h = height / 2.0
    assembly = {"type": "rect", "grid": [grid_a, list(grid_a), [-half_h, half_h]],
                "fill": [1 if e in guides else 0 for e in range(n_pins)], "pscale": 1}
    core = {"type": "rect", "grid": [grid_c, list(grid_c), [0.0, height]],
            "fill": [2] * (n_core * n_core), "pscale": 1}
    zs = [[s_zlo, 1], [s_zhi, -1], [s_cyl, -1]]
    root = {"type": "csg", "cells": [
        {"surfaces": [[s_xlo, 1], [s_xhi, -1], [s_ylo, 1], [s_yhi, -1]] + zs,
         "fill": 3, "translation": [0.0, 0.0, 0.0]},
        {"surfaces": [[s_xhi, 1]] + zs, "material": 2},
        {"surfaces": [[s_xlo, -1]] + zs, "material": 2},
        {"surfaces": [[s_xlo, 1], [s_xhi, -1], [s_yhi, 1]] + zs, "material": 2},
        {"surfaces": [[s_xlo, 1], [s_xhi, -1], [s_ylo, -1]] + zs, "material": 2},
    ]}
    return {
        "format": FORMAT, "name": f"core_{n_core}x{n_core}_of_{n_assm}x{n_assm}",
        "geometry_id": geometry_id, "sigma": [float(s) for s in sigma], "surfaces": S,
        "universes": [fuel_pin, guide_pin, assembly, core, root], "root": 4,
        "source_box": [-r_outer, -r_outer, 0.0, r_outer, r_outer, height],
        "params": {"r_fuel": r_fuel, "r_clad": r_clad, "r_guide": r_guide, "pitch": pitch},
    }


# ---------------------------------------------------------------------------
# Config 3: hexagonal core of hexagonal assemblies
# ---------------------------------------------------------------------------

def config3(core_rings=6, assm_rings=6, pin_rings=5, assm_pitch=10.0, pin_pitch=1.0,
            r_pin=0.45, height=200.0, sigma=None, seed=1, geometry_id=0) -> dict:
    """Hex core (rings 0..6, 127 assemblies) of hex assemblies of 91 pins.

    The pin lattice is turned by 30 degrees against the assembly hexagon so
    that pins of rings 0..5 fit inside it; ring-6 elements hold a fill
    universe (material 4) that the assembly hexagon (parent level) clips.
    Pin interiors are material 0/1/2 in Empire-like proportions; the pin
    exterior is material 3.
    """
    if sigma is None:
        sigma = np.random.default_rng(seed).uniform(0.05, 1.2, size=5)
    S = [{"type": "cz", "coef": [0.0, 0.0, r_pin]}]
    U = []
    for m in range(3):
        U.append({"type": "csg", "cells": [
            {"surfaces": [[0, -1]], "material": m},
            {"surfaces": [[0, 1]], "material": 3}]})
    U.append({"type": "csg", "cells": [{"surfaces": [], "material": 4}]})  # fill, uid 3
    elems = hex_elements(assm_rings)
    pin_slots = [e for e, (q, r) in enumerate(elems) if hex_ring(q, r) <= pin_rings]
    n_pin = len(pin_slots)
    n0 = int(round(n_pin * 60 / 217))
    n1 = int(round(n_pin * 96 / 217))
    kinds = np.array([0] * n0 + [1] * n1 + [2] * (n_pin - n0 - n1))
    kinds = kinds[np.random.default_rng(seed).permutation(n_pin)]
    fill = [3] * len(elems)
    for slot, k in zip(pin_slots, kinds):
        fill[slot] = int(k)
    a1, a2, nrm = _hex_frame(pin_pitch, rot30=True)
    half_h = height / 2.0
    U.append({"type": "hex", "rings": assm_rings, "a1": a1, "a2": a2, "normals": nrm,
              "half_pitch": pin_pitch / 2.0, "z": [-half_h, half_h], "fill": fill})
    assm_uid = len(U) - 1
    a1c, a2c, nrmc = _hex_frame(assm_pitch, rot30=False)
    n_core = len(hex_elements(core_rings))
    U.append({"type": "hex", "rings": core_rings, "a1": a1c, "a2": a2c, "normals": nrmc,
              "half_pitch": assm_pitch / 2.0, "z": [0.0, height], "fill": [assm_uid] * n_core,
              "bc": ["vacuum", "vacuum", "vacuum"]})
    # bounding box of the union of hexagons (pointy along y for the unrotated core)
    apo = assm_pitch / 2.0
    circ = apo / SQRT3_2
    xs, ys = [], []
    for (q, r) in hex_elements(core_rings):
        cx = q * a1c[0] + r * a2c[0]
        cy = q * a1c[1] + r * a2c[1]
        xs += [cx - apo, cx + apo]
        ys += [cy - circ, cy + circ]
    return {
        "format": FORMAT, "name": f"hex_core_r{core_rings}_of_r{assm_rings}",
        "geometry_id": geometry_id, "sigma": [float(s) for s in sigma], "surfaces": S,
        "universes": U, "root": len(U) - 1,
        "source_box": [min(xs), min(ys), 0.0, max(xs), max(ys), height],
    }


# ---------------------------------------------------------------------------
# Config 4: batch of independent small geometries
# ---------------------------------------------------------------------------

def config4_member(i: int, height=100.0) -> tuple[dict, int]:
    """Geometry i of the batch (generator seed 1000+i) and its particle count.

    n ~ U{3..17}; rect or hex 50/50 (hex rings = ceil((n-1)/2)); levels ~ U{2,3};
    particles N = floor(10**U[4,6]); vacuum root.  Three-level members are a
    3x3 (rect) or ring-1 (hex) core of n x n (rings) assemblies.
    """
    rng = np.random.default_rng(1000 + i)
    n = int(rng.integers(3, 18))
    is_hex = bool(rng.integers(0, 2))
    levels = int(rng.integers(2, 4))
    npart = int(math.floor(10.0 ** rng.uniform(4.0, 6.0)))
    sigma = [float(s) for s in rng.uniform(0.05, 1.0, size=3)]
    S = [{"type": "cz", "coef": [0.0, 0.0, 0.41]}, {"type": "cz", "coef": [0.0, 0.0, 0.475]}]
    pin = {"type": "csg", "cells": [
        {"surfaces": [[0, -1]], "material": 0},
        {"surfaces": [[0, 1], [1, -1]], "material": 1},
        {"surfaces": [[1, 1]], "material": 2}]}
    U = [pin]
    vac = "vacuum"
    if not is_hex:
        p = 1.26
        grid = [(j - n / 2.0) * p for j in range(n + 1)]
        if levels == 2:
            U.append({"type": "rect", "grid": [grid, list(grid), [0.0, height]],
                      "fill": [0] * (n * n), "bc": [vac] * 6})
            ext = grid[-1]
        else:
            U.append({"type": "rect", "grid": [grid, list(grid), [-height / 2, height / 2]],
                      "fill": [0] * (n * n)})
            ap = n * p
            gc = [(i - 1.5) * ap for i in range(4)]
            U.append({"type": "rect", "grid": [gc, list(gc), [0.0, height]],
                      "fill": [1] * 9, "bc": [vac] * 6})
            ext = gc[-1]
        box = [-ext, -ext, 0.0, ext, ext, height]
    else:
        rings = int(math.ceil((n - 1) / 2.0))
        a1, a2, nrm = _hex_frame(1.0, rot30=False)
        ne = len(hex_elements(rings))
        if levels == 2:
            U.append({"type": "hex", "rings": rings, "a1": a1, "a2": a2, "normals": nrm,
                      "half_pitch": 0.5, "z": [0.0, height], "fill": [0] * ne,
                      "bc": [vac, vac, vac]})
            cp = 1.0
            cr = rings
        else:
            U.append({"type": "hex", "rings": rings, "a1": a1, "a2": a2, "normals": nrm,
                      "half_pitch": 0.5, "z": [-height / 2, height / 2], "fill": [0] * ne})
            cp = float(2 * rings + 1)
            a1c, a2c, nrmc = _hex_frame(cp, rot30=False)
            U.append({"type": "hex", "rings": 1, "a1": a1c, "a2": a2c, "normals": nrmc,
                      "half_pitch": cp / 2.0, "z": [0.0, height], "fill": [1] * 7,
                      "bc": [vac, vac, vac]})
            cr = 1
        ext = (cr + 0.5) * cp / SQRT3_2 + 1e-9
        box = [-ext, -ext, 0.0, ext, ext, height]
    desc = {"format": FORMAT, "name": f"batch_{i}", "geometry_id": i, "sigma": sigma,
            "surfaces": S, "universes": U, "root": len(U) - 1, "source_box": box,
            "meta": {"n": n, "hex": is_hex, "levels": levels}}
    return desc, npart


def config4(count=64):
    return [config4_member(i) for i in range(count)]


# ---------------------------------------------------------------------------
# Config 5: deterministic rays entering the config-2 geometry
# ---------------------------------------------------------------------------

@dataclass
class RaySet:
    origin: np.ndarray     # (n, 3) float64
    direction: np.ndarray  # (n, 3) float64

    def packed(self) -> np.ndarray:
        """(n, 6) row-major x,y,z,u,v,w."""
        return np.ascontiguousarray(np.concatenate([self.origin, self.direction], axis=1))


def boundary_rays(n: int, r_outer=170.0, height=366.0, seed=5, inset=1e-9,
                  cosine=False) -> RaySet:
    """Rays from the surface of the cylinder r<R, 0<z<H, pointing inward.

    Origins are uniform by area over the lateral face and both caps, set
    `inset` cm inside the surface so the birth point lies in a cell.  The
    direction is isotropic and flipped into the inward hemisphere (cosine-law
    weighted instead when `cosine` is set, as for the mean-chord test).
    """
    rng = np.random.default_rng(seed)
    a_lat = 2.0 * math.pi * r_outer * height
    a_cap = math.pi * r_outer * r_outer
    part = rng.choice(3, size=n, p=np.array([a_lat, a_cap, a_cap]) / (a_lat + 2 * a_cap))
    o = np.empty((n, 3))
    nrm = np.empty((n, 3))  # outward normal
    phi = rng.uniform(0.0, 2 * math.pi, size=n)
    zz = rng.uniform(0.0, height, size=n)
    rad = (r_outer - inset) * np.sqrt(rng.uniform(0.0, 1.0, size=n))
    lat = part == 0
    o[lat, 0] = (r_outer - inset) * np.cos(phi[lat])
    o[lat, 1] = (r_outer - inset) * np.sin(phi[lat])
    o[lat, 2] = zz[lat]
    nrm[lat] = np.stack([np.cos(phi[lat]), np.sin(phi[lat]), np.zeros(lat.sum())], 1)
    for k, zc, nz in ((1, inset, -1.0), (2, height - inset, 1.0)):
        m = part == k
        o[m, 0] = rad[m] * np.cos(phi[m])
        o[m, 1] = rad[m] * np.sin(phi[m])
        o[m, 2] = zc
        nrm[m] = np.array([0.0, 0.0, nz])
    d = _directions(rng, n, cosine, nrm)
    return RaySet(o, d)


def box_rays(n: int, lo, hi, seed=7, inset=1e-9, cosine=True) -> RaySet:
    """Rays entering an axis-aligned box from its faces (uniform by area)."""
    rng = np.random.default_rng(seed)
    lo = np.asarray(lo, float)
    hi = np.asarray(hi, float)
    ext = hi - lo
    areas = np.array([ext[1] * ext[2], ext[1] * ext[2], ext[0] * ext[2], ext[0] * ext[2],
                      ext[0] * ext[1], ext[0] * ext[1]])
    face = rng.choice(6, size=n, p=areas / areas.sum())
    o = lo + rng.uniform(0.0, 1.0, size=(n, 3)) * ext
    nrm = np.zeros((n, 3))
    for f in range(6):
        m = face == f
        ax, side = f // 2, f % 2
        o[m, ax] = (hi[ax] - inset) if side else (lo[ax] + inset)
        nrm[m, ax] = 1.0 if side else -1.0
    return RaySet(o, _directions(rng, n, cosine, nrm))


def cylinder_rays(n: int, radius: float, z0: float, z1: float, seed=9, inset=1e-9) -> RaySet:
    """Cosine-law rays entering a finite z-cylinder (lateral face and caps)."""
    rs = boundary_rays(n, r_outer=radius, height=z1 - z0, seed=seed, inset=inset, cosine=True)
    rs.origin[:, 2] += z0
    return rs


def _directions(rng, n, cosine, nrm_out):
    if cosine:
        # cosine-law about the inward normal: mu = sqrt(xi)
        mu = np.sqrt(rng.uniform(0.0, 1.0, size=n))
        ph = rng.uniform(0.0, 2 * math.pi, size=n)
        s = np.sqrt(1.0 - mu * mu)
        inward = -nrm_out
        # orthonormal frame about the inward normal
        t1 = np.where(np.abs(inward[:, 2:3]) < 0.9, np.array([[0.0, 0.0, 1.0]]),
                      np.array([[1.0, 0.0, 0.0]]))
        b1 = np.cross(inward, t1)
        b1 /= np.linalg.norm(b1, axis=1, keepdims=True)
        b2 = np.cross(inward, b1)
        d = mu[:, None] * inward + (s * np.cos(ph))[:, None] * b1 + (s * np.sin(ph))[:, None] * b2
    else:
        d = rng.normal(size=(n, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        flip = np.sum(d * nrm_out, axis=1) > 0
        d[flip] *= -1.0
    return d


def config5(n_rays=1 << 20, seed=5, **geom_kw):
    """Transmission workload: the config-2 geometry and 2^20 inward boundary rays."""
    desc = config2(**geom_kw)
    rays = boundary_rays(n_rays, seed=seed)
    return desc, rays


# ---------------------------------------------------------------------------
# Tiny geometries for pins and edge cases
# ---------------------------------------------------------------------------

def single_pin(pitch=1.26, r=(0.41, 0.475), height=10.0, bc="vacuum", sigma=(0.5, 0.4, 0.3)):
    """A 1x1 root lattice holding one pin of len(r) concentric cylinders."""
    S = [{"type": "cz", "coef": [0.0, 0.0, float(x)]} for x in r]
    cells = [{"surfaces": [[0, -1]], "material": 0}]
    for k in range(1, len(r)):
        cells.append({"surfaces": [[k - 1, 1], [k, -1]], "material": k})
    cells.append({"surfaces": [[len(r) - 1, 1]], "material": len(r)})
    h = pitch / 2.0
    root = {"type": "rect", "grid": [[-h, h], [-h, h], [0.0, height]], "fill": [0],
            "bc": [bc] * 6}
    return {"format": FORMAT, "name": "single_pin", "geometry_id": 0,
            "sigma": [float(sigma[k % len(sigma)]) for k in range(len(r) + 1)],
            "surfaces": S, "universes": [{"type": "csg", "cells": cells}, root],
            "root": 1, "source_box": [-h, -h, 0.0, h, h, height]}


def bare_cylinder(radius=0.41, z0=0.0, z1=10.0, sigma=0.0):
    """A single finite cylinder (root CSG, vacuum outside) for chord tests."""
    S = [{"type": "cz", "coef": [0.0, 0.0, radius], "bc": "vacuum"},
         {"type": "pz", "coef": [z0], "bc": "vacuum"},
         {"type": "pz", "coef": [z1], "bc": "vacuum"}]
    root = {"type": "csg", "cells": [
        {"surfaces": [[0, -1], [1, 1], [2, -1]], "material": 0}]}
    return {"format": FORMAT, "name": "bare_cylinder", "geometry_id": 0, "sigma": [sigma],
            "surfaces": S, "universes": [root], "root": 0,
            "source_box": [-radius, -radius, z0, radius, radius, z1]}


def random_tiny(seed: int) -> dict:
    """Small random nested geometry (1-3 cylinders per pin, 1x1..3x3x2 lattices)."""
    rng = np.random.default_rng(seed)
    ncyl = int(rng.integers(1, 4))
    pitch = float(rng.uniform(1.0, 2.0))
    radii = np.sort(rng.uniform(0.05, 0.49, size=ncyl)) * pitch
    S = [{"type": "cz", "coef": [float(rng.uniform(-0.02, 0.02)), float(rng.uniform(-0.02, 0.02)),
                                  float(x)]} for x in radii]
    cells = [{"surfaces": [[0, -1]], "material": 0}]
    for k in range(1, ncyl):
        cells.append({"surfaces": [[k - 1, 1], [k, -1]], "material": k % 3})
    cells.append({"surfaces": [[ncyl - 1, 1]], "material": 3})
    pin = {"type": "csg", "cells": cells}
    nx, ny, nz = (int(rng.integers(1, 4)), int(rng.integers(1, 4)), int(rng.integers(1, 3)))
    gx = [(i - nx / 2.0) * pitch for i in range(nx + 1)]
    gy = [(j - ny / 2.0) * pitch for j in range(ny + 1)]
    gz = [k * 3.0 for k in range(nz + 1)]
    bc = ["reflect" if rng.uniform() < 0.5 else "vacuum" for _ in range(6)]
    root = {"type": "rect", "grid": [gx, gy, gz], "fill": [0] * (nx * ny * nz), "bc": bc}
    sigma = [float(s) for s in rng.uniform(0.1, 1.5, size=4)]
    return {"format": FORMAT, "name": f"tiny_{seed}", "geometry_id": seed % 7, "sigma": sigma,
            "surfaces": S, "universes": [pin, root], "root": 1,
            "source_box": [gx[0], gy[0], gz[0], gx[-1], gy[-1], gz[-1]]}


def small_hex(rings=2, pitch=1.0, r_pin=0.4, height=5.0, rot30=False, bc="vacuum",
              sigma=(0.6, 0.2)):
    """Root hex lattice of 2-cell pins."""
    a1, a2, nrm = _hex_frame(pitch, rot30=rot30)
    S = [{"type": "cz", "coef": [0.0, 0.0, r_pin]}]
    pin = {"type": "csg", "cells": [{"surfaces": [[0, -1]], "material": 0},
                                    {"surfaces": [[0, 1]], "material": 1}]}
    ne = len(hex_elements(rings))
    U = [pin, {"type": "hex", "rings": rings, "a1": a1, "a2": a2, "normals": nrm,
               "half_pitch": pitch / 2.0, "z": [0.0, height], "fill": [0] * ne,
               "bc": [bc, bc, bc]}]
    ext = (rings + 1) * pitch
    return {"format": FORMAT, "name": f"hex_r{rings}", "geometry_id": 3, "sigma": list(sigma),
            "surfaces": S, "universes": U, "root": 1,
            "source_box": [-ext, -ext, 0.0, ext, ext, height]}


def small_core(n_core=3, n_assm=5, **kw) -> dict:
    """A reduced config-2 core (same structure, fewer assemblies and pins)."""
    pitch = kw.pop("pitch", 1.26)
    r_outer = kw.pop("r_outer", 0.5 * n_core * n_assm * pitch * 1.2)
    height = kw.pop("height", 40.0)
    return config2(n_core=n_core, n_assm=n_assm, pitch=pitch, r_outer=r_outer, height=height,
                   **kw)


def small_hex_core(core_rings=1, assm_rings=3, pin_rings=2, **kw) -> dict:
    """A reduced config-3 core (same structure, fewer rings)."""
    return config3(core_rings=core_rings, assm_rings=assm_rings, pin_rings=pin_rings,
                   assm_pitch=kw.pop("assm_pitch", 2.0 * pin_rings + 2.0), **kw)


CONFIGS = {
    "c1": config1,
    "c2": config2,
    "c3": config3,
}


# ---------------------------------------------------------------------------
# Superimposed mesh for the track-length tally
# ---------------------------------------------------------------------------

def with_mesh(desc: dict, nx: int, ny: int, nz: int, box=None) -> dict:
    """A copy of `desc` with a superimposed rectilinear mesh of nx x ny x nz
    equal bins over `box` (default: the source box); plane i of an axis is
    lo + (hi - lo) * i / n in FP64, written out explicitly."""
    d = dict(desc)
    lo = list((box or desc["source_box"])[:3])
    hi = list((box or desc["source_box"])[3:])
    grid = []
    for a, n in enumerate((nx, ny, nz)):
        g = [lo[a] + (hi[a] - lo[a]) * i / n for i in range(n)] + [hi[a]]
        grid.append([float(v) for v in g])
    d["mesh"] = {"grid": grid}
    return d


def with_nu(desc: dict, nu) -> dict:
    """A copy of `desc` with per-material fission yields nu (0: no fission),
    for the power iteration."""
    d = dict(desc)
    d["nu"] = [float(v) for v in nu]
    return d
