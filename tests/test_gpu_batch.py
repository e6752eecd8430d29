"""Batched tracking (many geometries in one persistent launch) against the
per-geometry run_histories path and the oracle."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2406_13849_gb300 import inputs as I
from paper_2406_13849_gb300 import native as N

pytestmark = pytest.mark.gpu
SEED = 1
PA = 0.3


def _u64(t):
    return t.cpu().numpy().view(np.uint64)


def _members(k, cap):
    out = []
    for i in range(k):
        d, n = I.config4_member(i)
        out.append((d, min(n, cap) if cap else n))
    return out


def _build(members, exact):
    geoms = [N.Geometry(I.to_json(d), exact=exact) for d, _ in members]
    parts = [g.source_init(n, seed=SEED) for g, (_, n) in zip(geoms, members)]
    return geoms, parts


def test_batch_mix_of_trackers_and_levels():
    m = _members(64, 0)
    kinds = {(d["meta"]["hex"], d["meta"]["levels"]) for d, _ in m}
    assert kinds == {(False, 2), (False, 3), (True, 2), (True, 3)}
    n = [c for _, c in m]
    assert min(n) >= 10_000 and max(n) <= 1_000_000


@pytest.mark.parametrize("chunk", [32, 128, 1000])
def test_batched_bit_exact_vs_per_geometry(chunk):
    members = _members(12, 2_500)
    geoms, parts = _build(members, exact=True)
    b = N.Batch(geoms, parts, [n for _, n in members], records=True)
    b.upload(chunk)
    b.run(p_absorb=PA, seed=SEED)
    torch.cuda.synchronize()
    for k, (g, p, (_, n)) in enumerate(zip(geoms, parts, members)):
        t, c, r = g.run_histories(p, n, records=True, p_absorb=PA, seed=SEED)
        torch.cuda.synchronize()
        assert np.array_equal(_u64(b.tallies[k]), _u64(t)), k
        assert np.array_equal(_u64(b.counters)[16 * k:16 * k + 11], _u64(c)[:11]), k
        assert np.array_equal(_u64(b.records[k])[:2 * n], _u64(r)), k


def test_batched_against_oracle():
    members = _members(6, 800)
    geoms, parts = _build(members, exact=True)
    b = N.Batch(geoms, parts, [n for _, n in members], records=True)
    b.upload(128)
    b.run(p_absorb=PA, seed=SEED)
    torch.cuda.synchronize()
    for k, ((d, n), g) in enumerate(zip(members, geoms)):
        mode = O.MODE_RECT if g.rect_ok else O.MODE_CSG
        ref = O.Geometry(I.to_json(d), mode).run(n, SEED, PA, threads=8)
        h, nseg, st = N.unpack_records(b.records[k][:2 * n])
        assert np.array_equal(h, ref["hash"]) and np.array_equal(_u64(b.tallies[k]), ref["tally"]), k


def test_batched_graph_replay():
    members = _members(8, 4_000)
    geoms, parts = _build(members, exact=False)
    b = N.Batch(geoms, parts, [n for _, n in members])
    b.upload(256)
    opts = N.default_opts(p_absorb=PA, seed=SEED, precision=N.FP32_LOCAL)
    b.run(opts)
    torch.cuda.synchronize()
    once = [_u64(t).copy() for t in b.tallies]
    once_c = _u64(b.counters).copy()
    b.zero()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        b.run(opts)
    graph.replay()
    graph.replay()
    torch.cuda.synchronize()
    for k in range(len(geoms)):
        assert np.array_equal(_u64(b.tallies[k]), 2 * once[k])
    assert np.array_equal(_u64(b.counters), 2 * once_c)


def test_batched_fp32_vs_fp64():
    members = _members(16, 20_000)
    geoms, parts = _build(members, exact=False)
    counts = [n for _, n in members]
    b64 = N.Batch(geoms, parts, counts, records=True)
    b64.upload(512)
    b64.run(p_absorb=PA, seed=SEED)
    b32 = N.Batch(geoms, parts, counts, records=True)
    b32.upload(512)
    b32.run(p_absorb=PA, seed=SEED, precision=N.FP32_LOCAL)
    torch.cuda.synchronize()
    same, tot = 0, 0
    for k, n in enumerate(counts):
        _, na, sa = N.unpack_records(b64.records[k][:2 * n])
        _, nb, sb = N.unpack_records(b32.records[k][:2 * n])
        same += int(((na == nb) & (sa == sb)).sum())
        tot += n
        ta, tb = _u64(b64.tallies[k]).astype(float), _u64(b32.tallies[k]).astype(float)
        assert abs(tb.sum() - ta.sum()) <= 1e-3 * ta.sum()
    assert same / tot > 0.995
    c = _u64(b32.counters).reshape(-1, 16)
    assert c[:, N.K["lost"]].sum() == 0 and c[:, N.K["status"]].sum() == 0


def test_autotune_then_exact_results():
    members = _members(10, 3_000)
    geoms, parts = _build(members, exact=True)
    counts = [n for _, n in members]
    b = N.Batch(geoms, parts, counts, records=True)
    opts, chunk, ms = b.autotune(N.default_opts(p_absorb=PA, seed=SEED), reps=1)
    assert opts.block in (64, 96, 128) and chunk in (128, 512, 2048) and ms > 0
    b.run(opts)
    torch.cuda.synchronize()
    for k, (g, p, n) in enumerate(zip(geoms, parts, counts)):
        t, _, r = g.run_histories(p, n, records=True, p_absorb=PA, seed=SEED)
        assert np.array_equal(_u64(b.tallies[k]), _u64(t))


def test_config4_full_batch_vs_loop():
    members = _members(64, 0)
    geoms, parts = _build(members, exact=True)
    counts = [n for _, n in members]
    b = N.Batch(geoms, parts, counts)
    b.upload(512)
    b.run(p_absorb=PA, seed=SEED)
    torch.cuda.synchronize()
    for k, (g, p, n) in enumerate(zip(geoms, parts, counts)):
        t, c, _ = g.run_histories(p, n, p_absorb=PA, seed=SEED)
        torch.cuda.synchronize()
        assert np.array_equal(_u64(b.tallies[k]), _u64(t)), k
    # sampled particles of a few members, one by one in the oracle
    for k in (0, 17, 42, 63):
        d, n = members[k]
        mode = O.MODE_RECT if geoms[k].rect_ok else O.MODE_CSG
        o = O.Geometry(I.to_json(d), mode)
        bb = N.Batch([geoms[k]], [parts[k]], [n], records=True)
        bb.upload(512)
        bb.run(p_absorb=PA, seed=SEED)
        h, nseg, st = N.unpack_records(bb.records[0][:2 * n])
        for i in np.random.default_rng(k).choice(n, 20, replace=False):
            r = o.run(1, SEED, PA, first_id=int(i))
            assert r["hash"][0] == h[i] and r["nseg"][0] == nseg[i]


@pytest.mark.parametrize("member", [17, 63, 5])
def test_hex_root_lattice_members_bit_exact(member):
    # root hex lattices: every history against the oracle (cell boxes of
    # the root pseudo-array come from polygon clipping)
    d, n = I.config4_member(member)
    n = min(n, 300_000)
    g = N.Geometry(I.to_json(d), exact=True)
    parts = g.source_init(n, seed=SEED)
    t, c, r = g.run_histories(parts, n, records=True, p_absorb=PA, seed=SEED)
    h, nseg, st = N.unpack_records(r)
    mode = O.MODE_RECT if g.rect_ok else O.MODE_CSG
    ref = O.Geometry(I.to_json(d), mode).run(n, SEED, PA, threads=16)
    assert np.array_equal(h, ref["hash"])
    assert np.array_equal(_u64(t), ref["tally"])
