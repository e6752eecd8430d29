"""The CSG tracker with the bounding interval hierarchy ("accel": "bih",
Sec. 4.3) instead of the BVH: the same histories as the oracle's linear
scans, bit for bit in the exact build."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2406_13849_gb300 import inputs as I
from paper_2406_13849_gb300 import native as N

pytestmark = pytest.mark.gpu
SEED = 1

CASES = {
    "c1": (I.config1(), 0.3, 6_001),
    "small_core": (I.small_core(), 0.25, 4_003),
    "tiny8": (I.random_tiny(8), 0.3, 3_001),
    "small_hex_core": (I.small_hex_core(), 0.25, 3_001),
    "c3": (I.config3(), 0.25, 1_201),
}


def _u64(t):
    return t.cpu().numpy().view(np.uint64)


def _bih(desc):
    return dict(desc, accel="bih")


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("mode", [N.MODE_HISTORY, N.MODE_EVENT])
def test_bih_histories_bit_exact(name, mode):
    desc, pa, n = CASES[name]
    ref = O.Geometry(I.to_json(desc), O.MODE_CSG).run(n, SEED, pa, threads=8)
    g = N.Geometry(I.to_json(_bih(desc)), exact=True)
    parts = g.source_init(n, seed=SEED)
    tally, cnt, rec = g.run_histories(parts, n, records=True, tracker=N.TRACKER_CSG, mode=mode, p_absorb=pa,
                                      seed=SEED)
    h, nseg, st = N.unpack_records(rec)
    assert np.array_equal(h, ref["hash"]) and np.array_equal(nseg, ref["nseg"])
    assert np.array_equal(_u64(tally), ref["tally"])
    assert np.array_equal(_u64(cnt)[:10], ref["counters"][:10])


@pytest.mark.parametrize("name", list(CASES))
def test_bih_find_cell(name):
    desc, _, _ = CASES[name]
    lo, hi = np.array(desc["source_box"][:3]), np.array(desc["source_box"][3:])
    pts = lo + np.random.default_rng(5).uniform(0, 1, (20_000, 3)) * (hi - lo)
    ref = O.Geometry(I.to_json(desc), O.MODE_CSG).find_cell(pts)
    g = N.Geometry(I.to_json(_bih(desc)), exact=True)
    got = g.find_cell(torch.from_numpy(pts).cuda(), tracker=N.TRACKER_CSG).cpu().numpy()
    assert np.array_equal(got, ref)


def test_bih_full_size_sampled():
    # the three-level core with the BIH, event kernel, fast build, equal to
    # the same geometry with the BVH (the search finds the same unique cell)
    desc = I.config2()
    n = 300_000
    res = []
    for d in (desc, _bih(desc)):
        g = N.Geometry(I.to_json(d), exact=False)
        parts = g.source_init(n, seed=SEED)
        t, c, r = g.run_histories(parts, n, records=True, tracker=N.TRACKER_CSG, mode=N.MODE_EVENT, p_absorb=0.25,
                                  seed=SEED, queue_depth=512)
        res.append((_u64(t), _u64(r)))
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])


def test_accel_key_validated():
    with pytest.raises(N.TrkError):
        N.Geometry(I.to_json(dict(I.config1(), accel="kd")), exact=False)
