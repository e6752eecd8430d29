"""Thin Python binding of the C-ABI in include/trk.h (argument marshalling only).

Every step of the tracking path runs in the library's CUDA kernels; PyTorch
supplies device memory and streams.  The functions keep the ABI's names:
``geometry_build``, ``source_init``, ``run_histories``, ``tally_read``,
``trk_find_cell``, ``trk_trace``, ``transmission_fwd``, ``transmission_bwd``.

There is no CPU fallback: if the compiled library is missing, loading raises.
"""
from __future__ import annotations

import ctypes
import math
import os
import threading

import numpy as np
import torch

from . import build as _build

TRK_OK = 0
STATUS = {0: "TRK_OK", -1: "TRK_E_INVALID", -2: "TRK_E_DESC", -3: "TRK_E_CUDA", -4: "TRK_E_NOMEM",
          -5: "TRK_E_LOST", -6: "TRK_E_MAX_SEGMENTS", -7: "TRK_E_TIMEOUT", -8: "TRK_E_UNSUPPORTED",
          -9: "TRK_E_SOURCE"}
TRACKER_RECT, TRACKER_CSG, TRACKER_AUTO, TRACKER_DP = 0, 1, 2, 3
MODE_HISTORY, MODE_EVENT = 0, 1
FP64, FP32_LOCAL = 0, 1
NCOUNTERS = 16
K = dict(segments=0, crossings=1, collisions=2, absorbed=3, escaped=4, reflections=5, lost=6,
         maxseg=7, cutoff=8, source=9, close_calls=10, status=15)
NGEOM_PARAMS = 4


class TrkError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class RunOpts(ctypes.Structure):
    _fields_ = [("tracker", ctypes.c_int), ("mode", ctypes.c_int), ("precision", ctypes.c_int),
                ("block", ctypes.c_int), ("grid", ctypes.c_int), ("queue_depth", ctypes.c_int),
                ("sort_interval", ctypes.c_int), ("max_rounds", ctypes.c_int),
                ("seed", ctypes.c_uint64), ("first_id", ctypes.c_uint64),
                ("max_segments", ctypes.c_uint64), ("p_absorb", ctypes.c_double),
                ("max_path", ctypes.c_double), ("mesh_tally", ctypes.c_void_p)]


_P = ctypes.c_void_p
_LIBS: dict = {}
_LOCK = threading.Lock()


def library(exact: bool = False):
    """Load libtrk.so (or libtrk_exact.so), building it first if it is stale."""
    key = "exact" if exact else "fast"
    with _LOCK:
        if key in _LIBS:
            return _LIBS[key]
        path = _build.outputs()[key]
        if not os.path.exists(path):
            _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA tracking library missing: {path} (run paper_2406_13849_gb300.build)")
        lib = ctypes.CDLL(path)
        i64, u64, sz = ctypes.c_int64, ctypes.c_uint64, ctypes.c_size_t
        pi64, pi32, psz = ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(sz)
        sig = {
            "trk_last_error": (ctypes.c_char_p, []),
            "trk_exact_build": (ctypes.c_int, []),
            "trk_default_opts": (None, [ctypes.POINTER(RunOpts)]),
            "geometry_build": (ctypes.c_int, [ctypes.c_char_p, sz, _P, psz, _P, ctypes.POINTER(_P)]),
            "geometry_destroy": (ctypes.c_int, [_P]),
            "geometry_info": (ctypes.c_int, [_P, pi64, pi32, pi32, pi32]),
            "geometry_mesh_bins": (ctypes.c_int, [_P, pi64]),
            "power_iteration_work_bytes": (ctypes.c_int, [_P, i64, ctypes.POINTER(RunOpts), psz]),
            "power_iteration": (ctypes.c_int, [_P, i64, ctypes.c_int, ctypes.c_int, _P, _P, _P, _P, _P, sz,
                                               ctypes.POINTER(RunOpts), _P]),
            "source_init": (ctypes.c_int, [_P, i64, u64, u64, _P, psz, _P]),
            "run_histories_work_bytes": (ctypes.c_int, [_P, i64, ctypes.POINTER(RunOpts), psz]),
            "run_histories": (ctypes.c_int, [_P, _P, i64, _P, _P, _P, _P, sz, ctypes.POINTER(RunOpts), _P]),
            "tally_read": (ctypes.c_int, [_P, _P, _P, i64, _P, _P]),
            "trk_find_cell": (ctypes.c_int, [_P, ctypes.c_int, i64, _P, _P, _P]),
            "trk_distance_to_surface": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, i64, _P, _P, _P, _P, _P, _P,
                                                       _P]),
            "trk_sync_status": (ctypes.c_int, [_P, _P]),
            "trk_trace": (ctypes.c_int, [_P, _P, i64, ctypes.c_int32, _P, _P, _P, _P, _P, sz,
                                         ctypes.POINTER(RunOpts), _P]),
            "transmission_fwd": (ctypes.c_int, [_P, ctypes.c_int, i64, _P, _P, _P, _P, _P]),
            "transmission_bwd_work_bytes": (ctypes.c_int, [_P, i64, psz]),
            "transmission_bwd": (ctypes.c_int, [_P, ctypes.c_int, i64, _P, _P, ctypes.c_double, _P, _P,
                                                _P, sz, _P]),
            "batch_create": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P, _P, _P, ctypes.c_int, ctypes.POINTER(_P)]),
            "batch_destroy": (ctypes.c_int, [_P]),
            "batch_work_bytes": (ctypes.c_int, [_P, psz]),
            "batch_upload": (ctypes.c_int, [_P, _P, sz, ctypes.c_int, _P]),
            "run_batched": (ctypes.c_int, [_P, _P, ctypes.POINTER(RunOpts), _P]),
            "batch_autotune": (ctypes.c_int, [_P, _P, sz, ctypes.POINTER(RunOpts), ctypes.POINTER(ctypes.c_int),
                                              ctypes.c_int, ctypes.POINTER(ctypes.c_double), _P]),
            "transmission_bwd_noalloc": (ctypes.c_int, [_P, ctypes.c_int, i64, _P, _P, ctypes.c_double, _P, _P,
                                                        _P]),
            "trk_peak_kernel": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, sz,
                                               ctypes.POINTER(ctypes.c_double), _P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _LIBS[key] = lib
        return lib


def _check(lib, code):
    if code != TRK_OK:
        raise TrkError(code, lib.trk_last_error().decode())


def _ptr(t):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


_I64 = tuple(d for d in (torch.int64, getattr(torch, "uint64", None)) if d is not None)
_F64 = (torch.float64,)


def _need(t, what: str, device, nbytes: int = 0, dtypes=None, cols: int = 0):
    """Checks a tensor before its pointer goes to a kernel: on a CUDA device
    (the geometry's, when that has an index), contiguous, of one of `dtypes`,
    shaped (n, cols) when cols > 0, and holding at least nbytes bytes.  The C
    ABI sees only a raw device pointer, so these are caught here, before any
    launch, as TrkError(TRK_E_INVALID)."""
    if not isinstance(t, torch.Tensor):
        raise TrkError(-1, f"{what}: expected a torch tensor, got {type(t).__name__}")
    if dtypes is not None and t.dtype not in dtypes:
        raise TrkError(-1, f"{what}: dtype {t.dtype}, expected {' or '.join(str(d) for d in dtypes)}")
    if cols and (t.dim() != 2 or t.shape[1] != cols):
        raise TrkError(-1, f"{what}: shape {tuple(t.shape)}, expected (n, {cols})")
    have = t.numel() * t.element_size()
    if have < nbytes:
        raise TrkError(-1, f"{what}: {have} bytes, need {nbytes}")
    if not t.is_contiguous():
        raise TrkError(-1, f"{what}: tensor is not contiguous")
    if t.device.type != "cuda" or (device is not None and device.index is not None and
                                   t.device.index != device.index):
        raise TrkError(-1, f"{what}: tensor on {t.device}, expected {device or 'cuda'}")
    return t


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def default_opts(**kw) -> RunOpts:
    o = RunOpts()
    library().trk_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, v)
    return o


class Geometry:
    """A description flattened into device memory (geometry_build)."""

    def __init__(self, desc_json: str, device=None, exact: bool = False, stream=None):
        self.lib = library(exact)
        self.exact = exact
        raw = desc_json.encode() if isinstance(desc_json, str) else bytes(desc_json)
        self.device = torch.device(device if device is not None else "cuda")
        nbytes = ctypes.c_size_t(0)
        _check(self.lib, self.lib.geometry_build(raw, len(raw), None, ctypes.byref(nbytes), None, None))
        # 256-byte aligned device buffer owned by this object
        self.buf = torch.empty(nbytes.value + 256, dtype=torch.uint8, device=self.device)
        off = (-self.buf.data_ptr()) % 256
        self._base = self.buf.data_ptr() + off
        h = ctypes.c_void_p()
        cap = ctypes.c_size_t(nbytes.value)
        _check(self.lib, self.lib.geometry_build(raw, len(raw), ctypes.c_void_p(self._base), ctypes.byref(cap),
                                                 _stream(stream), ctypes.byref(h)))
        self.h = h
        ni, nm, dp, ro = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(self.lib, self.lib.geometry_info(h, ctypes.byref(ni), ctypes.byref(nm), ctypes.byref(dp),
                                                ctypes.byref(ro)))
        self.n_inst, self.n_mat, self.depth, self.rect_ok = ni.value, nm.value, dp.value, bool(ro.value)
        mb = ctypes.c_int64()
        _check(self.lib, self.lib.geometry_mesh_bins(h, ctypes.byref(mb)))
        self.mesh_bins = mb.value
        self.device_bytes = nbytes.value

    def close(self):
        if getattr(self, "h", None):
            self.lib.geometry_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- source_init -------------------------------------------------------
    def particle_bytes(self, n: int) -> int:
        b = ctypes.c_size_t(0)
        _check(self.lib, self.lib.source_init(self.h, n, 0, 0, None, ctypes.byref(b), None))
        return b.value

    def source_init(self, n: int, seed: int = 1, first_id: int = 0, out=None, stream=None):
        need = self.particle_bytes(n)
        if out is None:
            out = torch.empty(max(need, 8), dtype=torch.uint8, device=self.device)
        _need(out, "source_init out", self.device, need)
        b = ctypes.c_size_t(out.numel() * out.element_size())
        _check(self.lib, self.lib.source_init(self.h, n, first_id, seed, _ptr(out), ctypes.byref(b),
                                              _stream(stream)))
        return out

    @staticmethod
    def particles_as_arrays(buf, n):
        d = buf[: n * 56].view(torch.float64).view(7, n)
        st = buf[n * 56: n * 60].view(torch.int32)
        return d, st

    # -- run_histories -----------------------------------------------------
    def work_bytes(self, n: int, opts: RunOpts) -> int:
        b = ctypes.c_size_t(0)
        _check(self.lib, self.lib.run_histories_work_bytes(self.h, n, ctypes.byref(opts), ctypes.byref(b)))
        return b.value

    def run_histories(self, particles, n: int, tally=None, counters=None, records: bool = False,
                      work=None, opts: RunOpts | None = None, stream=None, mesh=None, **kw):
        """mesh: an int64 device tensor of mesh_bins to add the superimposed
        mesh tally to (sets opts.mesh_tally)."""
        opts = opts if opts is not None else default_opts(**kw)
        if mesh is not None:
            opts = RunOpts.from_buffer_copy(opts)
            opts.mesh_tally = mesh.data_ptr()
        if tally is None:
            tally = torch.zeros(self.n_inst, dtype=torch.int64, device=self.device)
        if counters is None:
            counters = torch.zeros(NCOUNTERS, dtype=torch.int64, device=self.device)
        rec = torch.zeros(2 * n, dtype=torch.int64, device=self.device) if records else None
        self._check_run(particles, n, tally, counters, mesh, "run_histories")
        wb = self.work_bytes(n, opts)
        if work is None and wb:
            work = torch.empty(wb + 256, dtype=torch.uint8, device=self.device)
        wp, wlen = None, 0
        if work is not None:
            _need(work, "run_histories work", self.device)
            off = (-work.data_ptr()) % 256
            wp = ctypes.c_void_p(work.data_ptr() + off)
            wlen = work.numel() * work.element_size() - off
        _check(self.lib, self.lib.run_histories(self.h, _ptr(particles), n, _ptr(tally), _ptr(counters), _ptr(rec),
                                                wp, wlen, ctypes.byref(opts), _stream(stream)))
        return tally, counters, rec

    def _check_run(self, particles, n, tally, counters, mesh, what):
        if n > 0 and particles is not None:
            _need(particles, f"{what} particles", self.device, self.particle_bytes(n))
        _need(tally, f"{what} tally", self.device, 8 * self.n_inst, _I64)
        _need(counters, f"{what} counters", self.device, 8 * NCOUNTERS, _I64)
        if mesh is not None:
            _need(mesh, f"{what} mesh", self.device, 8 * self.mesh_bins, _I64)

    def power_iteration_work_bytes(self, n: int, opts: RunOpts | None = None, **kw) -> int:
        opts = opts if opts is not None else default_opts(**kw)
        b = ctypes.c_size_t(0)
        _check(self.lib, self.lib.power_iteration_work_bytes(self.h, n, ctypes.byref(opts), ctypes.byref(b)))
        return b.value

    def power_iteration(self, n: int, inactive: int, cycles: int, tally=None, counters=None, mesh=None,
                        opts: RunOpts | None = None, stream=None, work=None, **kw):
        """Alg. 1 with the synthetic fission source ("nu" in the description):
        returns (k per cycle, sites banked per cycle) as device tensors, and
        the tally and counters of the active cycles.  work: a caller device
        buffer of power_iteration_work_bytes (+256 for alignment) reused
        across calls; allocated per call when None."""
        opts = RunOpts.from_buffer_copy(opts) if opts is not None else default_opts(**kw)
        if mesh is not None:
            opts.mesh_tally = mesh.data_ptr()
        if tally is None:
            tally = torch.zeros(self.n_inst, dtype=torch.int64, device=self.device)
        if counters is None:
            counters = torch.zeros(NCOUNTERS, dtype=torch.int64, device=self.device)
        self._check_run(None, n, tally, counters, mesh, "power_iteration")
        k = torch.zeros(cycles, dtype=torch.float64, device=self.device)
        bank = torch.zeros(cycles, dtype=torch.int64, device=self.device)
        wp, wlen = self._work_arg(work, self.power_iteration_work_bytes(n, opts), "power_iteration work")
        _check(self.lib, self.lib.power_iteration(self.h, n, inactive, cycles, _ptr(k), _ptr(bank), _ptr(tally),
                                                  _ptr(counters), wp, wlen, ctypes.byref(opts), _stream(stream)))
        return k, bank, tally, counters

    def tally_read(self, tally, counters=None, stream=None) -> np.ndarray:
        _need(tally, "tally_read tally", self.device, 8 * self.n_inst, _I64)
        if counters is not None:
            _need(counters, "tally_read counters", self.device, 8 * NCOUNTERS, _I64)
        out = np.zeros(self.n_inst, np.float64)
        _check(self.lib, self.lib.tally_read(self.h, _ptr(tally), out.ctypes.data_as(_P), self.n_inst,
                                             _ptr(counters), _stream(stream)))
        return out

    # -- diagnostics ---------------------------------------------------------
    def find_cell(self, xyz, tracker=TRACKER_AUTO, stream=None):
        xyz = _need(xyz.contiguous(), "find_cell xyz", self.device, 0, _F64, cols=3)
        out = torch.empty(xyz.shape[0], dtype=torch.int64, device=self.device)
        _check(self.lib, self.lib.trk_find_cell(self.h, tracker, xyz.shape[0], _ptr(xyz), _ptr(out),
                                                _stream(stream)))
        return out

    def distance_to_surface(self, xyz, dirs, tracker=TRACKER_AUTO, stream=None, precision=FP64,
                            with_close=False):
        """(distance, level, leaf instance) per point: find_cell from the
        root, then distance_to_surface over the levels; precision=FP32_LOCAL
        gives the FP32-local flight's distance, and with_close=True adds the
        per-point flag of distances redone in FP64."""
        xyz = _need(xyz.contiguous(), "distance_to_surface xyz", self.device, 0, _F64, cols=3)
        n = xyz.shape[0]
        dirs = _need(dirs.contiguous(), "distance_to_surface dirs", self.device, 24 * n, _F64, cols=3)
        d = torch.empty(n, dtype=torch.float64, device=self.device)
        lev = torch.empty(n, dtype=torch.int32, device=self.device)
        inst = torch.empty(n, dtype=torch.int64, device=self.device)
        close = torch.empty(n, dtype=torch.int32, device=self.device) if with_close else None
        _check(self.lib, self.lib.trk_distance_to_surface(self.h, tracker, precision, n, _ptr(xyz), _ptr(dirs),
                                                          _ptr(d), _ptr(lev), _ptr(inst), _ptr(close),
                                                          _stream(stream)))
        if with_close:
            return d, lev, inst, close
        return d, lev, inst

    def trace(self, particles, n: int, cap: int, opts: RunOpts | None = None, stream=None, work=None, **kw):
        """Segment log per particle (trk_trace): (instances (n, cap) int32,
        lengths (n, cap), tally, counters).  opts.mode picks the history or
        the event kernel; an event-mode work buffer is allocated unless given."""
        opts = opts if opts is not None else default_opts(**kw)
        if n > 0:
            _need(particles, "trace particles", self.device, self.particle_bytes(n))
        inst = torch.empty(n * cap, dtype=torch.int32, device=self.device)
        ln = torch.empty(n * cap, dtype=torch.float64, device=self.device)
        tally = torch.zeros(self.n_inst, dtype=torch.int64, device=self.device)
        cnt = torch.zeros(NCOUNTERS, dtype=torch.int64, device=self.device)
        wp, wlen = self._work_arg(work, self.work_bytes(n, opts), "trace work")
        _check(self.lib, self.lib.trk_trace(self.h, _ptr(particles), n, cap, _ptr(inst), _ptr(ln), _ptr(tally),
                                            _ptr(cnt), wp, wlen, ctypes.byref(opts), _stream(stream)))
        return inst.view(n, cap), ln.view(n, cap), tally, cnt

    def _work_arg(self, work, need: int, what: str):
        """(256-byte aligned pointer, usable bytes) of a caller work tensor,
        allocating one of `need` bytes when none is given and need > 0."""
        if work is None:
            if not need:
                return None, 0
            work = torch.empty(need + 256, dtype=torch.uint8, device=self.device)
        _need(work, what, self.device)
        off = (-work.data_ptr()) % 256
        have = work.numel() * work.element_size() - off
        if have < need:
            raise TrkError(-4, f"{what}: {have} usable bytes after 256-byte alignment, need {need}")
        # keep the buffer alive for the asynchronous launch
        self._last_work = work
        return ctypes.c_void_p(work.data_ptr() + off), have

    # -- transmission --------------------------------------------------------
    def transmission_fwd(self, rays, sigma, tracker=TRACKER_AUTO, lens: bool = True, stream=None):
        rays = _need(rays.contiguous(), "transmission_fwd rays", self.device, 0, _F64, cols=6)
        n = rays.shape[0]
        sigma = _need(sigma.contiguous(), "transmission_fwd sigma", self.device, 8 * self.n_mat, _F64)
        T = torch.empty(n, dtype=torch.float64, device=self.device)
        L = torch.empty(n, self.n_mat, dtype=torch.float64, device=self.device) if lens else None
        _check(self.lib, self.lib.transmission_fwd(self.h, tracker, n, _ptr(rays), _ptr(sigma),
                                                   _ptr(T), _ptr(L), _stream(stream)))
        return T, L

    def transmission_bwd_work_bytes(self, n: int) -> int:
        b = ctypes.c_size_t(0)
        _check(self.lib, self.lib.transmission_bwd_work_bytes(self.h, n, ctypes.byref(b)))
        return b.value

    def transmission_bwd(self, rays, sigma, pitch: float, gT, tracker=TRACKER_AUTO, stream=None, work=None,
                         grad=None):
        """dL/dtheta (n_materials + 4) from dL/dT per ray.  work: a caller
        device buffer of transmission_bwd_work_bytes bytes reused across
        calls (allocated per call when None); grad: the output tensor."""
        rays = _need(rays.contiguous(), "transmission_bwd rays", self.device, 0, _F64, cols=6)
        n = rays.shape[0]
        sigma = _need(sigma.contiguous(), "transmission_bwd sigma", self.device, 8 * self.n_mat, _F64)
        gT = _need(gT.contiguous(), "transmission_bwd gT", self.device, 8 * n, _F64)
        need = max(self.transmission_bwd_work_bytes(n), 8)
        if work is None:
            work = torch.empty(need, dtype=torch.uint8, device=self.device)
        _need(work, "transmission_bwd work", self.device, need)
        if grad is None:
            grad = torch.empty(self.n_mat + NGEOM_PARAMS, dtype=torch.float64, device=self.device)
        _need(grad, "transmission_bwd grad", self.device, 8 * (self.n_mat + NGEOM_PARAMS), _F64)
        _check(self.lib, self.lib.transmission_bwd(self.h, tracker, n, _ptr(rays), _ptr(sigma),
                                                   float(pitch), _ptr(gT), _ptr(grad), _ptr(work),
                                                   work.numel() * work.element_size(), _stream(stream)))
        return grad


class Batch:
    """Many geometries and particle populations in one persistent launch.

    geoms: list of Geometry (same library flavour); particles: their
    source_init buffers; counts: particles per geometry.  Tallies, counters
    (one row of NCOUNTERS per geometry) and optional records are allocated
    here unless given.
    """

    def __init__(self, geoms, particles, counts, tracker=TRACKER_AUTO, records: bool = False):
        self.lib = geoms[0].lib
        self.geoms = list(geoms)
        self.counts = [int(c) for c in counts]
        self.particles = list(particles)
        if len(self.particles) != len(self.geoms) or len(self.counts) != len(self.geoms):
            raise TrkError(-1, "Batch: one particle buffer and one count per geometry")
        if any(g.lib is not self.lib for g in self.geoms):
            raise TrkError(-1, "Batch: every geometry must come from the same library build (exact or fast)")
        for k, (g, p, c) in enumerate(zip(self.geoms, self.particles, self.counts)):
            _need(p, f"Batch particles[{k}]", g.device, g.particle_bytes(c) if c > 0 else 0)
        dev = geoms[0].device
        self.tallies = [torch.zeros(g.n_inst, dtype=torch.int64, device=dev) for g in geoms]
        self.counters = torch.zeros(len(geoms) * NCOUNTERS, dtype=torch.int64, device=dev)
        self.records = [torch.zeros(2 * max(c, 1), dtype=torch.int64, device=dev) for c in self.counts] \
            if records else None
        n = len(geoms)
        arr = ctypes.c_void_p * n
        hg = arr(*[g.h.value if isinstance(g.h, ctypes.c_void_p) else g.h for g in geoms])
        hp = arr(*[p.data_ptr() for p in particles])
        ht = arr(*[t.data_ptr() for t in self.tallies])
        hr = arr(*[r.data_ptr() for r in self.records]) if records else None
        hc = (ctypes.c_int64 * n)(*self.counts)
        h = ctypes.c_void_p()
        _check(self.lib, self.lib.batch_create(ctypes.cast(hg, _P), n, ctypes.cast(hp, _P), ctypes.cast(hc, _P),
                                               ctypes.cast(ht, _P), _ptr(self.counters),
                                               ctypes.cast(hr, _P) if hr is not None else None, tracker,
                                               ctypes.byref(h)))
        self.h = h
        b = ctypes.c_size_t(0)
        _check(self.lib, self.lib.batch_work_bytes(h, ctypes.byref(b)))
        self.work = torch.empty(b.value + 256, dtype=torch.uint8, device=dev)
        off = (-self.work.data_ptr()) % 256
        self.work_ptr = ctypes.c_void_p(self.work.data_ptr() + off)
        self.work_bytes = b.value
        self.chunk = 0

    def upload(self, chunk: int = 512, stream=None):
        _check(self.lib, self.lib.batch_upload(self.h, self.work_ptr, self.work_bytes, chunk, _stream(stream)))
        self.chunk = chunk

    def run(self, opts: RunOpts | None = None, stream=None, **kw):
        opts = opts if opts is not None else default_opts(**kw)
        _check(self.lib, self.lib.run_batched(self.h, self.work_ptr, ctypes.byref(opts), _stream(stream)))

    def autotune(self, opts: RunOpts, reps: int = 2, stream=None):
        ch = ctypes.c_int(0)
        best = ctypes.c_double(0)
        _check(self.lib, self.lib.batch_autotune(self.h, self.work_ptr, self.work_bytes, ctypes.byref(opts),
                                                 ctypes.byref(ch), reps, ctypes.byref(best), _stream(stream)))
        self.chunk = ch.value
        self.zero()
        return opts, ch.value, best.value

    def zero(self):
        for t in self.tallies:
            t.zero_()
        self.counters.zero_()

    def close(self):
        if getattr(self, "h", None):
            self.lib.batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def transmission_bwd_noalloc(geom: "Geometry", rays, sigma, pitch: float, gT, grad_out, tracker=TRACKER_AUTO,
                             stream=None):
    """transmission_bwd without a work buffer (its scratch lives in the
    library's fixed device array); writes grad_out (n_materials + 4)."""
    rays = _need(rays, "transmission_bwd_noalloc rays", geom.device, 0, _F64, cols=6)
    _need(sigma, "transmission_bwd_noalloc sigma", geom.device, 8 * geom.n_mat, _F64)
    _need(gT, "transmission_bwd_noalloc gT", geom.device, 8 * rays.shape[0], _F64)
    _need(grad_out, "transmission_bwd_noalloc grad_out", geom.device, 8 * (geom.n_mat + NGEOM_PARAMS), _F64)
    # the fixed scratch array is looked up on the current device: make it the
    # geometry's
    with torch.cuda.device(rays.device):
        _check(geom.lib, geom.lib.transmission_bwd_noalloc(geom.h, tracker, rays.shape[0], _ptr(rays), _ptr(sigma),
                                                           float(pitch), _ptr(gT), _ptr(grad_out), _stream(stream)))
    return grad_out


def sync_status(counters, stream=None, exact: bool = False) -> None:
    """Synchronises the stream and raises TrkError if a kernel wrote a
    status to counters[status] (trk_sync_status)."""
    lib = library(exact)
    _need(counters, "sync_status counters", None, 8 * NCOUNTERS, _I64)
    _check(lib, lib.trk_sync_status(_ptr(counters), _stream(stream)))


def unpack_records(rec: torch.Tensor):
    """(hash uint64, segments, status) from run_histories records."""
    r = rec.view(-1, 2).cpu().numpy().view(np.uint64)
    h = r[:, 0]
    nseg = (r[:, 1] >> np.uint64(32)).astype(np.int64)
    st = (r[:, 1] & np.uint64(0xffffffff)).astype(np.uint32).view(np.int32)
    return h, nseg, st


def peak_kernel(kind: int, blocks: int, iters: int, nbins: int, scratch, stream=None) -> float:
    """Launch one microbenchmark (trk_peak_kernel); returns its operation count."""
    lib = library()
    _need(scratch, "peak_kernel scratch", None)
    ops = ctypes.c_double(0)
    _check(lib, lib.trk_peak_kernel(kind, blocks, iters, nbins, _ptr(scratch),
                                    scratch.numel() * scratch.element_size(), ctypes.byref(ops),
                                    _stream(stream)))
    return ops.value
