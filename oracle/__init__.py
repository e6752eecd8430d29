"""CPU FP64 oracle for nested-universe particle tracking (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path never does: the
library in ``paper_2406_13849_gb300`` fails loudly if its CUDA extension is
missing instead of falling back here.

``build()`` compiles ``oracle.cpp`` (plain C++17, ``-ffp-contract=off`` so no
multiply-add is fused) into ``_build/liboracle.so`` and, with
``-DORACLE_COUNT_FLOPS``, into ``_build/liboracle_count.so`` (same code on a
counting scalar type, for the algorithmic FP64 operation count per segment).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SRC = os.path.join(_HERE, "oracle.cpp")
_LOCK = threading.Lock()
_LIBS: dict = {}

MODE_RECT = 0   # rect arrays tracked by index (Alg. 5/6); hex arrays as pseudo-arrays
MODE_CSG = 1    # every universe a CSG universe; arrays become pseudo-arrays (Sec. 4.3)

# counters (same meaning as the library's device counters)
K_SEGMENTS, K_CROSSINGS, K_COLLISIONS, K_ABSORBED, K_ESCAPED, K_REFLECTIONS, K_LOST, \
    K_MAXSEG, K_CUTOFF, K_SOURCE = range(10)
N_COUNTERS = 16

P_ALIVE, P_ABSORBED, P_ESCAPED, P_CUTOFF, P_LOST, P_MAXSEG, P_SOURCE = 0, 1, 2, 3, -5, -6, -9
NPARAM = 4


def build(force: bool = False) -> None:
    """Compile both oracle libraries (in parallel) if missing or stale."""
    jobs = []
    for name, extra in (("liboracle.so", []), ("liboracle_count.so", ["-DORACLE_COUNT_FLOPS"])):
        out = os.path.join(_BUILD, name)
        if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
            jobs.append((out, extra))
    if not jobs:
        return
    os.makedirs(_BUILD, exist_ok=True)
    procs = []
    for out, extra in jobs:
        tmp = out + ".tmp"
        cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp,
               _SRC, "-lpthread"] + extra
        procs.append((subprocess.Popen(cmd), tmp, out))
    for p, tmp, out in procs:
        if p.wait() != 0:
            raise RuntimeError(f"oracle build failed: {out}")
        os.replace(tmp, out)


_D = ctypes.c_double
_LL = ctypes.c_longlong
_ULL = ctypes.c_ulonglong
_P = ctypes.c_void_p
_I = ctypes.c_int
_U = ctypes.c_uint


def _lib(counting: bool = False):
    key = "count" if counting else "plain"
    with _LOCK:
        if key in _LIBS:
            return _LIBS[key]
        build()
        lib = ctypes.CDLL(os.path.join(_BUILD, "liboracle_count.so" if counting else "liboracle.so"))
        lib.orc_geometry_load.restype = _P
        lib.orc_geometry_load.argtypes = [ctypes.c_char_p, _LL, _I, ctypes.c_char_p, _I]
        lib.orc_geometry_free.argtypes = [_P]
        lib.orc_n_instances.restype = _LL
        lib.orc_n_instances.argtypes = [_P]
        lib.orc_n_materials.argtypes = [_P]
        lib.orc_max_depth.argtypes = [_P]
        lib.orc_source.argtypes = [_P, _LL, _LL, _ULL, _P, _P]
        lib.orc_run.argtypes = [_P, _LL, _LL, _ULL, _D, _LL, _D, _I, _P, _P, _P, _P, _P, _P]
        lib.orc_trace.restype = _LL
        lib.orc_trace.argtypes = [_P, _LL, _ULL, _D, _LL, _LL, _P, _P, _P, _P, _P]
        lib.orc_clearance.argtypes = [_P, _LL, _P, _P, _P, _P]
        lib.orc_trace_from_site.restype = _LL
        lib.orc_trace_from_site.argtypes = [_P, _LL, _ULL, _D, _D, _P, _LL, _P, _P, _P, _P]
        lib.orc_find_cell.argtypes = [_P, _LL, _P, _P]
        lib.orc_find_cell_brute.argtypes = [_P, _LL, _P, _P, _P, _P]
        lib.orc_distance.argtypes = [_P, _LL, _P, _P, _P, _P, _P]
        lib.orc_transmission.argtypes = [_P, _LL, _P, _P, _D, _P, _P, _P, _P, _P, _I]
        lib.orc_philox4x32_10.argtypes = [_P, _P, _P]
        lib.orc_uniform2.argtypes = [_U, _U, _U, _U, _U, _U, _P]
        lib.orc_log.restype = _D
        lib.orc_log.argtypes = [_D]
        lib.orc_isotropic.argtypes = [_U, _U, _U, _U, _P]
        lib.orc_flop_counts.argtypes = [_P, _I]
        lib.orc_run_mesh.argtypes = [_P, _LL, _LL, _ULL, _D, _I, _P, _P, _P]
        lib.orc_mesh_segment.argtypes = [_P, _P, _P, _D, _P]
        lib.orc_power.argtypes = [_P, _LL, _LL, _ULL, _D, _I, _I, _I, _P, _P, _P, _P]
        lib.orc_mesh_bins.restype = _LL
        lib.orc_mesh_bins.argtypes = [_P]
        _LIBS[key] = lib
        return lib


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(_P)


class Geometry:
    """A description loaded into the oracle in one tracking mode."""

    def __init__(self, desc_json: str, mode: int = MODE_RECT, counting: bool = False):
        self.lib = _lib(counting)
        raw = desc_json.encode() if isinstance(desc_json, str) else desc_json
        err = ctypes.create_string_buffer(512)
        h = self.lib.orc_geometry_load(raw, len(raw), mode, err, 512)
        if not h:
            raise ValueError(err.value.decode())
        self.h = h
        self.mode = mode
        self.n_inst = int(self.lib.orc_n_instances(h))
        self.n_mat = int(self.lib.orc_n_materials(h))
        self.depth = int(self.lib.orc_max_depth(h))
        self.mesh_bins = int(self.lib.orc_mesh_bins(h))

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.lib.orc_geometry_free(h)
            self.h = None

    def run_mesh(self, n: int, seed: int, p_absorb: float, first_id: int = 0, threads: int = 1):
        """run() with the superimposed mesh's track-length tally (uint64 per
        bin, x fastest); the description must carry a mesh."""
        if not self.mesh_bins:
            raise ValueError("description has no mesh")
        tally = np.zeros(self.n_inst, np.uint64)
        cnt = np.zeros(N_COUNTERS, np.uint64)
        mesh = np.zeros(self.mesh_bins, np.uint64)
        self.lib.orc_run_mesh(self.h, n, first_id, seed, p_absorb, threads, _ptr(tally), _ptr(cnt), _ptr(mesh))
        return {"tally": tally, "counters": cnt, "mesh": mesh}

    def power(self, n: int, seed: int, p_absorb: float, inactive: int, cycles: int, first_id: int = 0,
              threads: int = 1):
        """Power iteration: k per cycle, sites banked per cycle, tally and
        counters of the active cycles."""
        k = np.zeros(cycles, np.float64)
        bank = np.zeros(cycles, np.int64)
        tally = np.zeros(self.n_inst, np.uint64)
        cnt = np.zeros(N_COUNTERS, np.uint64)
        rc = self.lib.orc_power(self.h, n, first_id, seed, p_absorb, inactive, cycles, threads, _ptr(k), _ptr(bank),
                                _ptr(tally), _ptr(cnt))
        return {"k": k, "bank": bank, "tally": tally, "counters": cnt, "ok": rc == 0}

    def mesh_segment(self, r, d, length: float) -> np.ndarray:
        """Mesh tally of one segment (start r, direction d, length)."""
        mesh = np.zeros(self.mesh_bins, np.uint64)
        self.lib.orc_mesh_segment(self.h, _ptr(np.ascontiguousarray(r, np.float64)),
                                  _ptr(np.ascontiguousarray(d, np.float64)), float(length), _ptr(mesh))
        return mesh

    def source(self, n: int, seed: int, first_id: int = 0):
        out = np.zeros((n, 7), np.float64)
        st = np.zeros(n, np.int32)
        self.lib.orc_source(self.h, n, first_id, seed, _ptr(out), _ptr(st))
        return out, st

    def run(self, n: int, seed: int, p_absorb: float, first_id: int = 0, max_segments: int = 1_000_000,
            max_path: float = float("inf"), threads: int = 1, records: bool = True):
        tally = np.zeros(self.n_inst, np.uint64)
        cnt = np.zeros(N_COUNTERS, np.uint64)
        rh = np.zeros(n, np.uint64) if records else None
        rn = np.zeros(n, np.int64) if records else None
        rs = np.zeros(n, np.int32) if records else None
        rf = np.zeros((n, 3), np.float64) if records else None
        self.lib.orc_run(self.h, n, first_id, seed, p_absorb, max_segments, max_path, threads,
                         _ptr(tally), _ptr(cnt), _ptr(rh), _ptr(rn), _ptr(rs), _ptr(rf))
        return {"tally": tally, "counters": cnt, "hash": rh, "nseg": rn, "status": rs, "final": rf}

    def trace(self, pid: int, seed: int, p_absorb: float, cap: int = 100_000, max_segments: int = 1_000_000,
              geometry: bool = False):
        """One history's segments: (leaf instance, length, kind, status), kind
        0 crossing, 1 collision, 2 cut; with geometry=True also each segment's
        start position, direction and material cross section, an (n, 7)
        array."""
        inst = np.zeros(cap, np.int64)
        ln = np.zeros(cap, np.float64)
        kind = np.zeros(cap, np.int32)
        st = np.zeros(1, np.int32)
        geo = np.zeros((cap, 7), np.float64) if geometry else None
        k = int(self.lib.orc_trace(self.h, pid, seed, p_absorb, max_segments, cap, _ptr(inst), _ptr(ln),
                                   _ptr(kind), _ptr(st), _ptr(geo)))
        k = min(k, cap)
        if geometry:
            return inst[:k], ln[:k], kind[:k], int(st[0]), geo[:k]
        return inst[:k], ln[:k], kind[:k], int(st[0])

    def clearance(self, xyz: np.ndarray, dirs: np.ndarray, lens) -> np.ndarray:
        """Distances of segments from the geometry's surfaces (global frame):
        per segment (start xyz, unit direction, length) the smallest distance
        from the start point to a surface and the smallest to any other
        surface, the same two at the end point, the tangency |b - r| over the
        cylinders whose axis is closest to the segment's line inside the
        segment (inf if none), and the unit normal (sign arbitrary) of the
        surface nearest to the end point: an (n, 8) array."""
        xyz = np.ascontiguousarray(xyz, np.float64).reshape(-1, 3)
        dirs = np.ascontiguousarray(dirs, np.float64).reshape(-1, 3)
        lens = np.ascontiguousarray(lens, np.float64).reshape(-1)
        out = np.zeros((len(xyz), 8), np.float64)
        self.lib.orc_clearance(self.h, len(xyz), _ptr(xyz), _ptr(dirs), _ptr(lens), _ptr(out))
        return out

    def trace_from_site(self, pid: int, seed: int, p_absorb: float, knorm: float, site, cap: int = 100_000):
        """One history born at `site` as the power iteration births its later
        cycles (direction and tau from the particle's source counters)."""
        inst = np.zeros(cap, np.int64)
        ln = np.zeros(cap, np.float64)
        kind = np.zeros(cap, np.int32)
        st = np.zeros(1, np.int32)
        site = np.ascontiguousarray(site, np.float64)
        k = int(self.lib.orc_trace_from_site(self.h, pid, seed, p_absorb, knorm, _ptr(site), cap, _ptr(inst),
                                             _ptr(ln), _ptr(kind), _ptr(st)))
        k = min(k, cap)
        return inst[:k], ln[:k], kind[:k], int(st[0])

    def find_cell(self, xyz: np.ndarray) -> np.ndarray:
        xyz = np.ascontiguousarray(xyz, np.float64)
        out = np.zeros(len(xyz), np.int64)
        self.lib.orc_find_cell(self.h, len(xyz), _ptr(xyz), _ptr(out))
        return out

    def distance(self, xyz: np.ndarray, dirs: np.ndarray):
        """distance_to_surface from points with directions: (distance,
        level of the winning surface, leaf instance); NaN / -1 outside."""
        xyz = np.ascontiguousarray(xyz, np.float64)
        dirs = np.ascontiguousarray(dirs, np.float64)
        n = len(xyz)
        d = np.zeros(n, np.float64)
        lev = np.zeros(n, np.int32)
        inst = np.zeros(n, np.int64)
        self.lib.orc_distance(self.h, n, _ptr(xyz), _ptr(dirs), _ptr(d), _ptr(lev), _ptr(inst))
        return d, lev, inst

    def find_cell_brute(self, xyz: np.ndarray):
        xyz = np.ascontiguousarray(xyz, np.float64)
        inst = np.zeros(len(xyz), np.int64)
        cnt = np.zeros(len(xyz), np.int32)
        near = np.zeros(len(xyz), np.float64)
        nleaf = self.lib.orc_find_cell_brute(self.h, len(xyz), _ptr(xyz), _ptr(inst), _ptr(cnt), _ptr(near))
        return inst, cnt, near, nleaf

    def transmission(self, rays: np.ndarray, sigma, pitch: float = 0.0, grad: bool = True, threads: int = 1):
        rays = np.ascontiguousarray(rays, np.float64)
        n = len(rays)
        sigma = np.ascontiguousarray(sigma, np.float64)
        T = np.zeros(n)
        lens = np.zeros((n, self.n_mat))
        dT = np.zeros((n, self.n_mat + NPARAM)) if grad else None
        hs = np.zeros(n, np.uint64)
        st = np.zeros(n, np.int32)
        self.lib.orc_transmission(self.h, n, _ptr(rays), _ptr(sigma), pitch, _ptr(T), _ptr(lens), _ptr(dT),
                                  _ptr(hs), _ptr(st), threads)
        return {"T": T, "lens": lens, "dT": dT, "hash": hs, "status": st}

    def flop_counts(self, reset: bool = True) -> dict:
        out = np.zeros(5, np.uint64)
        self.lib.orc_flop_counts(_ptr(out), 1 if reset else 0)
        return dict(zip(("add", "mul", "div", "sqrt", "cmp"), (int(x) for x in out)))


def philox4x32_10(ctr, key) -> np.ndarray:
    lib = _lib()
    c = np.ascontiguousarray(ctr, np.uint32)
    k = np.ascontiguousarray(key, np.uint32)
    o = np.zeros(4, np.uint32)
    lib.orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(o))
    return o


def uniform2(pid, event, tag, k, seed_lo, gid):
    o = np.zeros(2)
    _lib().orc_uniform2(pid, event, tag, k, seed_lo, gid, _ptr(o))
    return o


def own_log(x: float) -> float:
    return float(_lib().orc_log(float(x)))


def isotropic(pid, event, seed_lo, gid):
    o = np.zeros(3)
    ok = _lib().orc_isotropic(pid, event, seed_lo, gid, _ptr(o))
    return o, bool(ok)
