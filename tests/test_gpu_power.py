"""Power iteration (Alg. 1) with the synthetic fission source: the CUDA
cycles against the oracle's, bit for bit in the exact build (k per cycle,
sites banked, tallies and counters of the active cycles)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2406_13849_gb300 import inputs as I
from paper_2406_13849_gb300 import native as N

pytestmark = pytest.mark.gpu
SEED = 1


def _u64(t):
    return t.cpu().numpy().view(np.uint64)


CASES = {
    "small_core": (I.with_nu(I.small_core(), (2.4, 0.0, 0.0, 0.0)), 0.25, 4_001),
    "c1_mixed": (I.with_nu(I.config1(), (2.1, 0.0, 0.3)), 0.3, 5_003),
    "hex": (I.with_nu(I.small_hex_core(), (2.3, 2.0, 1.5, 0.0, 0.0)), 0.25, 3_001),
}


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("tracker,mode", [(N.TRACKER_RECT, N.MODE_HISTORY), (N.TRACKER_CSG, N.MODE_EVENT),
                                          (N.TRACKER_RECT, N.MODE_EVENT)])
def test_power_iteration_bit_exact(name, tracker, mode):
    desc, pa, n = CASES[name]
    omode = O.MODE_RECT if tracker == N.TRACKER_RECT else O.MODE_CSG
    ref = O.Geometry(I.to_json(desc), omode).power(n, SEED, pa, 2, 5, threads=8)
    assert ref["ok"]
    g = N.Geometry(I.to_json(desc), exact=True)
    k, bank, tally, cnt = g.power_iteration(n, 2, 5, tracker=tracker, mode=mode, p_absorb=pa, seed=SEED,
                                            queue_depth=128)
    torch.cuda.synchronize()
    assert np.array_equal(k.cpu().numpy(), ref["k"])
    assert np.array_equal(bank.cpu().numpy(), ref["bank"])
    assert np.array_equal(_u64(tally), ref["tally"])
    assert np.array_equal(_u64(cnt)[:10], ref["counters"][:10])
    assert _u64(cnt)[N.K["status"]] == 0


def test_power_infinite_medium_k_is_nu():
    d = I.with_nu(I.config1(sigma=(0.5, 0.5, 0.5)), (2.5, 2.5, 2.5))
    g = N.Geometry(I.to_json(d), exact=False)
    n = 20_000
    k, bank, _, _ = g.power_iteration(n, 1, 4, mode=N.MODE_EVENT, p_absorb=0.3, seed=SEED)
    assert np.all(k.cpu().numpy() == 2.5)
    assert np.all(bank.cpu().numpy()[1:] == n)


def test_power_iteration_graph_replay_and_mesh():
    # the whole iteration is one stream of launches: capture it, replay it
    # twice, and the active-cycle tallies (cell and mesh) double
    d = I.with_mesh(I.with_nu(I.small_core(), (2.4, 0.0, 0.0, 0.0)), 9, 7, 5)
    g = N.Geometry(I.to_json(d), exact=False)
    n = 20_000
    tally = torch.zeros(g.n_inst, dtype=torch.int64, device="cuda")
    cnt = torch.zeros(N.NCOUNTERS, dtype=torch.int64, device="cuda")
    mesh = torch.zeros(g.mesh_bins, dtype=torch.int64, device="cuda")
    opts = N.default_opts(mode=N.MODE_EVENT, p_absorb=0.25, seed=SEED, queue_depth=128)
    k1, b1, _, _ = g.power_iteration(n, 1, 3, tally=tally, counters=cnt, mesh=mesh, opts=opts)
    torch.cuda.synchronize()
    t1, m1 = _u64(tally).copy(), _u64(mesh).copy()
    assert abs(float(m1.sum()) - float(t1.sum())) <= 1e-9 * float(t1.sum())
    tally.zero_(); cnt.zero_(); mesh.zero_()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        g.power_iteration(n, 1, 3, tally=tally, counters=cnt, mesh=mesh, opts=opts, stream=s)
    graph.replay()
    graph.replay()
    torch.cuda.synchronize()
    assert np.array_equal(_u64(tally), 2 * t1) and np.array_equal(_u64(mesh), 2 * m1)


def test_power_iteration_errors_and_no_fission():
    g = N.Geometry(I.to_json(I.config1()), exact=False)
    k, bank, _, cnt = g.power_iteration(1000, 0, 2, p_absorb=0.3, seed=SEED)
    torch.cuda.synchronize()
    assert k.cpu().numpy()[0] == 0.0 and bank.cpu().numpy()[0] == 0
    assert _u64(cnt)[N.K["status"]].view(np.int64) == -9          # TRK_E_SOURCE
    gd = N.Geometry(I.to_json(I.with_nu(I.config1(), (2.0, 0.0, 0.0))), exact=False)
    with pytest.raises(N.TrkError) as e:
        gd.power_iteration(1000, 0, 2, precision=N.FP32_LOCAL)
    assert e.value.code == -8
    with pytest.raises(N.TrkError) as e:
        gd.power_iteration(1000, 3, 2)
    assert e.value.code == -1
