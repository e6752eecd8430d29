"""C-ABI checks that need no GPU: the library builds, loads and exports every
entry point declared in include/*.h; host-side validation returns the
documented status codes (no compute calls)."""
import ctypes
import glob
import os
import re

import pytest

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
