"""The dynamic-polymorphism tracker (the paper's DP method, Sec. 4.1): rect
array and CSG tracker objects behind one base class, each per-level find,
distance and crossing a virtual call.  Its per-level arithmetic is the array
tracker's, so its histories equal the oracle's rect mode bit for bit in the
--fmad=false build and equal the array tracker's in both builds."""
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
    "small_hex_core": (I.small_hex_core(), 0.25, 3_001),
    "hex_rot": (I.small_hex(rings=3, rot30=True), 0.3, 2_003),
}


def _u64(t):
    return t.cpu().numpy().view(np.uint64)


def _run(g, n, pa, tracker, **kw):
    parts = g.source_init(n, seed=SEED)
    tally, cnt, rec = g.run_histories(parts, n, records=True, tracker=tracker, p_absorb=pa, seed=SEED, **kw)
    torch.cuda.synchronize()
    return _u64(tally), _u64(cnt), rec


@pytest.mark.parametrize("name", list(CASES))
def test_dp_bit_exact_vs_oracle(name):
    desc, pa, n = CASES[name]
    o = O.Geometry(I.to_json(desc), O.MODE_RECT).run(n, SEED, pa, threads=8)
    g = N.Geometry(I.to_json(desc), exact=True)
    tally, cnt, rec = _run(g, n, pa, N.TRACKER_DP)
    h, nseg, st = N.unpack_records(rec)
    assert np.array_equal(st, o["status"]) and np.array_equal(nseg, o["nseg"]) and np.array_equal(h, o["hash"])
    assert np.array_equal(tally, o["tally"])
    assert np.array_equal(cnt[:10], o["counters"][:10]) and cnt[N.K["status"]] == 0


@pytest.mark.parametrize("exact", [True, False])
def test_dp_equals_array_tracker(exact):
    # same kernel arithmetic behind static and virtual dispatch: identical
    # histories in either build, on the full three-level core
    desc = I.config2()
    n, pa = 200_000, 0.25
    g = N.Geometry(I.to_json(desc), exact=exact)
    t_dp, c_dp, r_dp = _run(g, n, pa, N.TRACKER_DP)
    t_rt, c_rt, r_rt = _run(g, n, pa, N.TRACKER_RECT)
    assert np.array_equal(t_dp, t_rt) and np.array_equal(c_dp, c_rt)
    assert np.array_equal(_u64(r_dp), _u64(r_rt))


def test_dp_without_records_and_segment_cap():
    desc, pa, n = CASES["small_core"]
    g = N.Geometry(I.to_json(desc), exact=True)
    parts = g.source_init(n, seed=SEED)
    t1, c1, _ = g.run_histories(parts, n, tracker=N.TRACKER_DP, p_absorb=pa, seed=SEED)
    t2, c2, _ = g.run_histories(parts, n, tracker=N.TRACKER_RECT, p_absorb=pa, seed=SEED)
    torch.cuda.synchronize()
    assert np.array_equal(_u64(t1), _u64(t2)) and np.array_equal(_u64(c1), _u64(c2))
    o = O.Geometry(I.to_json(desc), O.MODE_RECT).run(n, SEED, pa, threads=8, max_segments=7)
    tally, cnt, rec = _run(g, n, pa, N.TRACKER_DP, max_segments=7)
    h, nseg, st = N.unpack_records(rec)
    assert np.array_equal(h, o["hash"]) and np.array_equal(st, o["status"]) and np.array_equal(tally, o["tally"])


def test_dp_unsupported_options():
    desc, pa, n = CASES["c1"]
    g = N.Geometry(I.to_json(desc), exact=False)
    parts = g.source_init(n, seed=SEED)
    for kw in (dict(mode=N.MODE_EVENT), dict(precision=N.FP32_LOCAL), dict(max_path=5.0)):
        with pytest.raises(N.TrkError):
            g.run_histories(parts, n, tracker=N.TRACKER_DP, p_absorb=pa, seed=SEED, **kw)
    with pytest.raises(N.TrkError):
        g.find_cell(torch.zeros(4, 3, dtype=torch.float64, device="cuda"), tracker=N.TRACKER_DP)
