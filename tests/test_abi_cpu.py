"""C-ABI checks that need no GPU: the library builds, loads and exports every
entry point declared in include/*.h; host-side validation returns the
documented status codes (no compute calls)."""
import copy
import ctypes
import glob
import os
import random
import re

import pytest
import torch

from paper_2406_13849_gb300 import inputs as I
from paper_2406_13849_gb300 import native as N

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"^\s*(?:[A-Za-z_][\w\s\*]*?)\b([A-Za-z_]\w*)\s*\(", txt, flags=re.M):
            name = m.group(1)
            if name not in ("if", "for", "while", "return", "sizeof"):
                names.append(name)
    return sorted(set(names))


@pytest.mark.parametrize("exact", [False, True])
def test_library_exports_every_declared_symbol(exact):
    lib = N.library(exact)
    names = declared_functions()
    assert "geometry_build" in names and "run_histories" in names and "tally_read" in names
    assert "source_init" in names and "transmission_bwd" in names
    for n in names:
        assert hasattr(lib, n), n
    assert lib.trk_exact_build() == (1 if exact else 0)


def _size(desc_json):
    lib = N.library()
    raw = desc_json.encode()
    nb = ctypes.c_size_t(0)
    st = lib.geometry_build(raw, len(raw), None, ctypes.byref(nb), None, None)
    return st, nb.value, lib.trk_last_error().decode()


def test_size_query_for_every_config():
    for d in (I.config1(), I.config2(), I.config3(), I.small_hex_core(), I.config4_member(3)[0]):
        st, nb, err = _size(I.to_json(d))
        assert st == 0, err
        assert 0 < nb < 1 << 22


@pytest.mark.parametrize("mutate,code", [
    (lambda d: d.update(root=99), -2),
    (lambda d: d["universes"][1].update(fill=[0] * 3), -2),
    (lambda d: d["surfaces"][0].update(bc="reflect"), -2),
    (lambda d: d["surfaces"][0].update(coef=[0.0, 0.0]), -2),
    (lambda d: d["surfaces"][0].update(coef=[0.0, 0.0, -1.0]), -2),
    (lambda d: d["universes"][0]["cells"][0].update(material=7), -2),
    (lambda d: d["universes"][0]["cells"][0]["surfaces"][0].__setitem__(1, 0), -2),
    (lambda d: d["universes"][1]["grid"][0].reverse(), -2),
    (lambda d: d.update(sigma=[]), -2),
    (lambda d: d.update(source_box=[0, 0, 0, 0, 0, 0]), -2),
])
def test_bad_descriptions(mutate, code):
    d = I.config1()
    mutate(d)
    st, _, err = _size(I.to_json(d))
    assert st == code and err


def test_cyclic_and_too_deep():
    d = I.config1()
    d["universes"][0] = {"type": "csg", "cells": [{"surfaces": [], "fill": 1, "translation": [0, 0, 0]}]}
    st, _, err = _size(I.to_json(d))
    assert st == -2 and "itself" in err
    # five nested levels exceed the compiled depth of four
    d = I.config2()
    d["universes"].append({"type": "csg", "cells": [{"surfaces": [], "fill": 4, "translation": [0, 0, 0]}]})
    d["root"] = 5
    st, _, err = _size(I.to_json(d))
    assert st == -8


def test_null_arguments():
    lib = N.library()
    assert lib.geometry_build(None, 0, None, None, None, None) == -1
    assert lib.geometry_destroy(None) == -1
    assert lib.run_histories(None, None, 0, None, None, None, None, 0, None, None) == -1
    assert lib.tally_read(None, None, None, 0, None, None) == -1
    assert lib.source_init(None, 1, 0, 0, None, None, None) == -1
    st, _, err = _size("not json at all")
    assert st == -2 and "JSON" in err


def _unreachable(d):
    d["universes"].append(copy.deepcopy(d["universes"][0]))


@pytest.mark.parametrize("mutate,needle", [
    (_unreachable, "not reachable"),
    (lambda d: d["surfaces"][0].update(rparam=5), "rparam"),
    (lambda d: d["surfaces"][0].update(rparam=0.5), "rparam"),
    (lambda d: d["surfaces"][0].update(pscale=2), "pscale"),
    (lambda d: d["universes"][1].update(pscale=-1), "pscale"),
    (lambda d: d.update(geometry_id=1e30), "geometry_id"),
    (lambda d: d.update(geometry_id=-3), "geometry_id"),
    (lambda d: d["universes"][0]["cells"][0]["surfaces"][0].__setitem__(0, 1e30), "surface id"),
    (lambda d: d["universes"][0]["cells"][0]["surfaces"][0].__setitem__(1, 0.5), "sense"),
    (lambda d: d["universes"][1]["grid"][0].__setitem__(0, -1e999), "grid"),
    (lambda d: d.update(source_box=[0, 0, 0, 1e999, 1, 1]), "source_box"),
])
def test_rejects_out_of_range_fields(mutate, needle):
    """Fields the builder packs into integers or uses as coordinates are range-checked:
    each of these descriptions once reached undefined behaviour or an out-of-bounds read
    on the host (found by the fuzz test below)."""
    d = I.config1()
    mutate(d)
    st, _, err = _size(I.to_json(d).replace("Infinity", "1e999"))
    assert st == -2 and needle in err, err


def test_hex_fields_checked():
    d = I.small_hex()
    hx = next(u for u in d["universes"] if u["type"] == "hex")
    hx["rings"] = 1.5
    assert _size(I.to_json(d))[0] == -2
    d = I.small_hex()
    hx = next(u for u in d["universes"] if u["type"] == "hex")
    hx["normals"][1] = [0.0, 0.0]
    assert _size(I.to_json(d))[0] == -2


def test_deeply_nested_json_is_an_error_not_a_crash():
    st, _, err = _size("[" * 200000)
    assert st == -2 and "deep" in err
    st, _, err = _size('{"a":' * 100000)
    assert st == -2 and "deep" in err


_FUZZ_VALUES = [0, -1, 1, 2, 3, 0.5, -0.5, 1e308, -1e308, 1e30, 2**31, 2**31 - 1, -(2**31), 2**40, 7,
                64, 65, 1e-300, "x", "reflect", "vacuum", None, True, [], [0], [0, 0], [0, 0, 0], {},
                [[0, 1]]]


def _fuzz_paths(o, pre=()):
    yield pre
    if isinstance(o, dict):
        for k, v in o.items():
            yield from _fuzz_paths(v, pre + (k,))
    elif isinstance(o, list):
        for i, v in enumerate(o):
            yield from _fuzz_paths(v, pre + (i,))


def _fuzz_mutate(d, rng):
    path = rng.choice(list(_fuzz_paths(d))[1:])
    parent = d
    for k in path[:-1]:
        parent = parent[k]
    k = path[-1]
    r = rng.random()
    if r < 0.15:
        del parent[k]
    elif r < 0.3 and isinstance(parent, list):
        parent.insert(k, copy.deepcopy(parent[k]))
    else:
        parent[k] = copy.deepcopy(rng.choice(_FUZZ_VALUES))


def test_mutated_descriptions_never_crash_the_builder():
    """Seeded mutations of valid descriptions (deleted, duplicated or retyped members,
    extreme numbers, truncated text) through the host-only size query: every one is
    accepted or rejected with a status; the process must survive all of them."""
    rng = random.Random(2406)
    bases = [I.config1(), I.single_pin(), I.small_hex(), I.small_core(), I.small_hex_core(),
             I.with_mesh(I.single_pin(), 3, 3, 2), I.random_tiny(3), I.config4_member(5)[0],
             I.with_nu(I.single_pin(), [2.0, 0.0, 0.0])]
    seen = {}
    for _ in range(1500):
        d = copy.deepcopy(rng.choice(bases))
        for _ in range(rng.randint(1, 3)):
            _fuzz_mutate(d, rng)
        txt = I.to_json(d)
        if rng.random() < 0.05:
            txt = txt[: rng.randrange(len(txt))]
        st, nb, err = _size(txt)
        assert st in (0, -2, -8), (st, err)
        assert (st == 0) == (err == "") and (st != 0 or nb > 0)
        seen[st] = seen.get(st, 0) + 1
    assert seen.get(0, 0) > 20 and seen.get(-2, 0) > 1000


def _fake_geometry(n_inst=10, n_mat=3, mesh_bins=0):
    """A Geometry object without a device image: enough for the binding's
    checks, which run before any library call."""
    g = object.__new__(N.Geometry)
    g.lib, g.exact, g.h = N.library(), False, None
    g.device = torch.device("cuda")
    g.n_inst, g.n_mat, g.mesh_bins = n_inst, n_mat, mesh_bins
    g.particle_bytes = lambda n: 60 * n
    return g


def _code_and_message(fn):
    with pytest.raises(N.TrkError) as e:
        fn()
    return e.value.code, str(e.value)


def test_binding_checks_tensors_before_any_launch():
    """The C ABI sees raw device pointers, so the binding checks what a tensor
    can tell: dtype, shape, size, layout and device, in that order (a CPU
    tensor here is never on the GPU, so each case checks the first tensor a
    call hands over, and one that passes the other checks stops at the device)."""
    g = _fake_geometry()
    i64, f64 = torch.int64, torch.float64
    tally, cnt = torch.zeros(10, dtype=i64), torch.zeros(16, dtype=i64)
    parts = torch.zeros(600, dtype=torch.uint8)
    cases = [
        (lambda: g.run_histories(parts[:599], 10, tally=tally, counters=cnt), "bytes, need 600"),
        (lambda: g.run_histories(parts, 10, tally=tally, counters=cnt), "tensor on cpu"),
        (lambda: g.run_histories(None, 10, tally=torch.zeros(9, dtype=i64), counters=cnt), "need 80"),
        (lambda: g.run_histories(None, 10, tally=tally.double(), counters=cnt), "dtype"),
        (lambda: N.sync_status(cnt[:8]), "need 128"),
        (lambda: g.tally_read(torch.zeros(5, dtype=i64)), "need 80"),
        (lambda: g.tally_read(tally), "tensor on cpu"),
        (lambda: g.find_cell(torch.zeros(30, dtype=f64)), "expected (n, 3)"),
        (lambda: g.find_cell(torch.zeros(10, 3, dtype=torch.float32)), "dtype"),
        (lambda: g.distance_to_surface(torch.zeros(4, 2, dtype=f64), torch.zeros(4, 3, dtype=f64)), "expected (n, 3)"),
        (lambda: g.transmission_fwd(torch.zeros(4, 3, dtype=f64), torch.zeros(3, dtype=f64)), "expected (n, 6)"),
        (lambda: g.transmission_bwd(torch.zeros(4, 6, dtype=torch.float32), torch.zeros(3, dtype=f64), 1.26,
                                    torch.zeros(4, dtype=f64)), "dtype"),
        (lambda: g.source_init(10, out=torch.zeros(100, dtype=torch.uint8)), "need 600"),
        (lambda: N.sync_status(torch.zeros(16, dtype=torch.float64)), "dtype"),
        (lambda: N.transmission_bwd_noalloc(g, torch.zeros(4, 5, dtype=f64), torch.zeros(3, dtype=f64), 1.26,
                                            torch.zeros(4, dtype=f64), torch.zeros(7, dtype=f64)), "expected (n, 6)"),
    ]
    for fn, needle in cases:
        code, msg = _code_and_message(fn)
        assert code == -1 and needle in msg, (needle, msg)
    # a strided view is copied by .contiguous() where the binding owns the copy
    code, msg = _code_and_message(lambda: g.find_cell(torch.zeros(4, 6, dtype=f64)[:, ::2]))
    assert "tensor on cpu" in msg
    # output buffers are written in place, so a strided one is refused
    code, msg = _code_and_message(lambda: g.run_histories(None, 10, tally=torch.zeros(20, dtype=i64)[::2],
                                                          counters=cnt))
    assert "not contiguous" in msg


def test_batch_checks_its_members_before_any_call():
    fast, exact = _fake_geometry(), _fake_geometry()
    exact.lib, exact.exact = N.library(True), True
    parts = torch.zeros(600, dtype=torch.uint8)
    code, msg = _code_and_message(lambda: N.Batch([fast, exact], [parts, parts], [10, 10]))
    assert "same library build" in msg
    code, msg = _code_and_message(lambda: N.Batch([fast, fast], [parts], [10, 10]))
    assert "one particle buffer" in msg
    code, msg = _code_and_message(lambda: N.Batch([fast], [parts[:100]], [10]))
    assert "need 600" in msg


def test_every_entry_point_rejects_a_null_handle_on_the_host():
    """Each entry point that takes a handle or output pointer validates it on
    the host and returns TRK_E_INVALID (no launch, no device access): the
    ABI's "calls return a status and never throw" convention, for all of
    them.  Functions without arguments to validate are listed apart."""
    lib = N.library()
    o = N.default_opts()
    calls = {
        "geometry_build": (None, 0, None, None, None, None),
        "geometry_destroy": (None,),
        "geometry_info": (None, None, None, None, None),
        "geometry_mesh_bins": (None, None),
        "source_init": (None, 1, 0, 0, None, None, None),
        "run_histories_work_bytes": (None, 1, ctypes.byref(o), None),
        "run_histories": (None, None, 1, None, None, None, None, 0, ctypes.byref(o), None),
        "power_iteration_work_bytes": (None, 1, ctypes.byref(o), None),
        "power_iteration": (None, 1, 0, 1, None, None, None, None, None, 0, ctypes.byref(o), None),
        "tally_read": (None, None, None, 0, None, None),
        "trk_find_cell": (None, 0, 1, None, None, None),
        "trk_distance_to_surface": (None, 0, 0, 1, None, None, None, None, None, None, None),
        "trk_sync_status": (None, None),
        "trk_trace": (None, None, 1, 1, None, None, None, None, None, 0, ctypes.byref(o), None),
        "transmission_fwd": (None, 0, 1, None, None, None, None, None),
        "transmission_bwd_work_bytes": (None, 1, None),
        "transmission_bwd": (None, 0, 1, None, None, 1.26, None, None, None, 0, None),
        "transmission_bwd_noalloc": (None, 0, 1, None, None, 1.26, None, None, None),
        "batch_create": (None, 1, None, None, None, None, None, 0, None),
        "batch_destroy": (None,),
        "batch_work_bytes": (None, None),
        "batch_upload": (None, None, 0, 512, None),
        "run_batched": (None, None, ctypes.byref(o), None),
        "batch_autotune": (None, None, 0, ctypes.byref(o), None, 1, None, None),
        "trk_peak_kernel": (0, 1, 1, 0, None, 0, None, None),
    }
    no_arguments_to_check = {"trk_default_opts", "trk_last_error", "trk_exact_build"}
    assert set(calls) | no_arguments_to_check == set(declared_functions())
    for name, args in calls.items():
        st = getattr(lib, name)(*args)
        assert st == -1, (name, st)
        assert lib.trk_last_error().decode(), name


def test_last_error_is_per_thread():
    """trk_last_error is thread-local: threads failing at the same time for
    different reasons each read their own message (ctypes releases the GIL
    around the calls, so the calls overlap)."""
    import threading
    lib = N.library()
    bad = {"json": ("not json", "JSON"), "root": (None, "root")}
    d = I.config1()
    d["root"] = 99
    bad["root"] = (I.to_json(d), "root")
    seen, errors = [], []

    def worker(kind):
        txt, needle = bad[kind]
        raw = txt.encode()
        for _ in range(300):
            nb = ctypes.c_size_t(0)
            st = lib.geometry_build(raw, len(raw), None, ctypes.byref(nb), None, None)
            msg = lib.trk_last_error().decode()
            if st != -2 or needle not in msg:
                errors.append((kind, st, msg))
        seen.append(kind)

    threads = [threading.Thread(target=worker, args=(k,)) for k in ("json", "root") * 4]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert len(seen) == 8 and not errors, errors[:3]
