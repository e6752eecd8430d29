"""Superimposed mesh track-length tally: the CUDA path against the oracle's
walk over the mesh planes (bit for bit in the exact build)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2406_13849_gb300 import inputs as I
from paper_2406_13849_gb300 import native as N

pytestmark = pytest.mark.gpu
SEED = 1

CASES = {
    "c1": (I.with_mesh(I.config1(), 17, 17, 10), 0.3, 6_001),
    "small_core": (I.with_mesh(I.small_core(), 13, 11, 7), 0.25, 4_003),
    # a mesh smaller than the geometry: segments enter and leave it
    "c1_partial": (I.with_mesh(I.config1(), 5, 6, 4, box=[-4.0, -6.0, 20.0, 7.0, 3.5, 70.0]), 0.3, 6_001),
}


def _u64(t):
    return t.cpu().numpy().view(np.uint64)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("tracker,mode", [(N.TRACKER_RECT, N.MODE_HISTORY), (N.TRACKER_CSG, N.MODE_EVENT),
                                          (N.TRACKER_RECT, N.MODE_EVENT)])
def test_mesh_tally_bit_exact(name, tracker, mode):
    desc, pa, n = CASES[name]
    omode = O.MODE_RECT if tracker == N.TRACKER_RECT else O.MODE_CSG
    ref = O.Geometry(I.to_json(desc), omode).run_mesh(n, SEED, pa, threads=8)
    g = N.Geometry(I.to_json(desc), exact=True)
    assert g.mesh_bins == len(ref["mesh"])
    parts = g.source_init(n, seed=SEED)
    mesh = torch.zeros(g.mesh_bins, dtype=torch.int64, device="cuda")
    tally, cnt, rec = g.run_histories(parts, n, tracker=tracker, mode=mode, p_absorb=pa, seed=SEED, mesh=mesh,
                                      records=True)
    torch.cuda.synchronize()
    assert np.array_equal(_u64(mesh), ref["mesh"])
    assert np.array_equal(_u64(tally), ref["tally"])
    assert np.array_equal(_u64(cnt)[:10], ref["counters"][:10])


def test_mesh_tally_fast_build_and_totals():
    desc, pa, n = CASES["small_core"]
    ref = O.Geometry(I.to_json(desc), O.MODE_RECT).run_mesh(n, SEED, pa, threads=8)
    g = N.Geometry(I.to_json(desc), exact=False)
    parts = g.source_init(n, seed=SEED)
    mesh = torch.zeros(g.mesh_bins, dtype=torch.int64, device="cuda")
    tally, _, _ = g.run_histories(parts, n, mode=N.MODE_EVENT, p_absorb=pa, seed=SEED, mesh=mesh)
    torch.cuda.synchronize()
    got = _u64(mesh).astype(np.float64) / 2**32
    exp = ref["mesh"].astype(np.float64) / 2**32
    # contraction moves segment ends by ~1e-15 cm (rarely ~1e-8, near-tangent
    # hits): bins agree to 1e-9 relative plus 1e-6 cm
    assert np.all(np.abs(got - exp) <= 1e-9 * exp + 1e-6)
    # the mesh covers the geometry: its total is the cell tally's total up to
    # each piece's rounding to 2^-32 cm
    t = _u64(tally).astype(np.float64).sum() / 2**32
    assert abs(got.sum() - t) <= 1e-9 * t


def test_mesh_tally_full_size_sampled():
    # the benchmark's mesh (119 x 119 x 30 over the core's box) on the
    # three-level core, event kernel, BVH-CSG: a 200k-particle sample
    desc = I.with_mesh(I.config2(), 119, 119, 30)
    n = 200_000
    ref = O.Geometry(I.to_json(desc), O.MODE_CSG).run_mesh(n, SEED, 0.25, threads=16)
    g = N.Geometry(I.to_json(desc), exact=True)
    parts = g.source_init(n, seed=SEED)
    mesh = torch.zeros(g.mesh_bins, dtype=torch.int64, device="cuda")
    g.run_histories(parts, n, tracker=N.TRACKER_CSG, mode=N.MODE_EVENT, p_absorb=0.25, seed=SEED, mesh=mesh,
                    queue_depth=512)
    torch.cuda.synchronize()
    assert g.mesh_bins == 119 * 119 * 30
    assert np.array_equal(_u64(mesh), ref["mesh"])


def test_mesh_tally_errors():
    g = N.Geometry(I.to_json(I.config1()), exact=False)
    parts = g.source_init(100, seed=SEED)
    assert g.mesh_bins == 0
    mesh = torch.zeros(8, dtype=torch.int64, device="cuda")
    with pytest.raises(N.TrkError) as e:
        g.run_histories(parts, 100, mesh=mesh)
    assert e.value.code == -1
    gm = N.Geometry(I.to_json(I.with_mesh(I.config1(), 2, 2, 2)), exact=False)
    pm = gm.source_init(100, seed=SEED)
    with pytest.raises(N.TrkError) as e:
        gm.run_histories(pm, 100, mesh=mesh, precision=N.FP32_LOCAL)
    assert e.value.code == -8
    with pytest.raises(N.TrkError) as e:
        gm.run_histories(pm, 100, mesh=mesh, max_path=10.0)
    assert e.value.code == -8
