"""Batched tracking in event mode (the event kernel's warp queues and slot
records over chunks of one geometry at a time) against the per-geometry
run_histories path and the oracle."""
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


def _members(k, cap, start=0):
    out = []
    for i in range(start, start + k):
        d, n = I.config4_member(i)
        out.append((d, min(n, cap) if cap else n))
    return out


def _build(members, exact):
    geoms = [N.Geometry(I.to_json(d), exact=exact) for d, _ in members]
    parts = [g.source_init(n, seed=SEED) for g, (_, n) in zip(geoms, members)]
    return geoms, parts


def _ev(**kw):
    return N.default_opts(mode=N.MODE_EVENT, p_absorb=PA, seed=SEED, **kw)


# chunk 32 with depth 256: many chunks per geometry, a warp switches geometry
# often; chunk 1000: chunks that continue within a geometry; chunk 100000:
# one chunk per geometry (every geometry drains a single warp)
@pytest.mark.parametrize("chunk,depth", [(32, 256), (1000, 32), (1000, 512), (100_000, 128)])
def test_batched_event_bit_exact_vs_per_geometry(chunk, depth):
    members = _members(12, 2_500)
    geoms, parts = _build(members, exact=True)
    b = N.Batch(geoms, parts, [n for _, n in members], records=True)
    b.upload(chunk)
    b.run(_ev(queue_depth=depth))
    torch.cuda.synchronize()
    for k, (g, p, (_, n)) in enumerate(zip(geoms, parts, members)):
        t, c, r = g.run_histories(p, n, records=True, p_absorb=PA, seed=SEED)
        torch.cuda.synchronize()
        assert np.array_equal(_u64(b.tallies[k]), _u64(t)), k
        assert np.array_equal(_u64(b.counters)[16 * k:16 * k + 11], _u64(c)[:11]), k
        assert np.array_equal(_u64(b.records[k])[:2 * n], _u64(r)), k
        assert _u64(b.counters)[16 * k + N.K["status"]] == 0


def test_batched_event_against_oracle():
    members = _members(6, 800, start=20)
    geoms, parts = _build(members, exact=True)
    b = N.Batch(geoms, parts, [n for _, n in members], records=True)
    b.upload(256)
    b.run(_ev(queue_depth=64))
    torch.cuda.synchronize()
    for k, ((d, n), g) in enumerate(zip(members, geoms)):
        mode = O.MODE_RECT if g.rect_ok else O.MODE_CSG
        ref = O.Geometry(I.to_json(d), mode).run(n, SEED, PA, threads=8)
        h, nseg, st = N.unpack_records(b.records[k][:2 * n])
        assert np.array_equal(h, ref["hash"]) and np.array_equal(_u64(b.tallies[k]), ref["tally"]), k
        assert np.array_equal(nseg, ref["nseg"]) and np.array_equal(st, ref["status"]), k


def test_batched_event_csg_tracker_everywhere():
    # tracker CSG for every member: one launch only (no rect chunks)
    members = _members(5, 1_500, start=40)
    geoms, parts = _build(members, exact=True)
    b = N.Batch(geoms, parts, [n for _, n in members], records=True, tracker=N.TRACKER_CSG)
    b.upload(512)
    b.run(_ev(queue_depth=128))
    torch.cuda.synchronize()
    for k, (g, p, (_, n)) in enumerate(zip(geoms, parts, members)):
        t, _, r = g.run_histories(p, n, records=True, p_absorb=PA, seed=SEED, tracker=N.TRACKER_CSG)
        assert np.array_equal(_u64(b.tallies[k]), _u64(t)), k
        assert np.array_equal(_u64(b.records[k])[:2 * n], _u64(r)), k


def test_batched_event_graph_replay_fp32():
    members = _members(8, 4_000)
    geoms, parts = _build(members, exact=False)
    b = N.Batch(geoms, parts, [n for _, n in members])
    b.upload(2048)
    opts = _ev(precision=N.FP32_LOCAL, queue_depth=256)
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


def test_batched_event_first_call_captured():
    # the first event-mode call of a batch (which creates its side stream)
    # made inside a graph capture: the replay equals an uncaptured run of an
    # identical batch; hex (CSG) and array members, so both launches and the
    # fork/join are captured
    members = _members(6, 3_000)
    counts = [n for _, n in members]
    opts = _ev(queue_depth=256)
    ref_geoms, ref_parts = _build(members, exact=True)
    ref = N.Batch(ref_geoms, ref_parts, counts)
    ref.upload(1024)
    ref.run(opts)
    torch.cuda.synchronize()
    geoms, parts = _build(members, exact=True)
    b = N.Batch(geoms, parts, counts)
    b.upload(1024)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        b.run(opts)
    graph.replay()
    torch.cuda.synchronize()
    for k in range(len(geoms)):
        assert np.array_equal(_u64(b.tallies[k]), _u64(ref.tallies[k])), k
    assert np.array_equal(_u64(b.counters), _u64(ref.counters))


def test_batched_event_autotune_then_exact():
    members = _members(10, 3_000)
    geoms, parts = _build(members, exact=True)
    counts = [n for _, n in members]
    b = N.Batch(geoms, parts, counts, records=True)
    opts, chunk, ms = b.autotune(_ev(), reps=1)
    assert opts.queue_depth in (384, 512) and chunk in (128, 256, 512, 2048) and ms > 0
    b.run(opts)
    torch.cuda.synchronize()
    for k, (g, p, n) in enumerate(zip(geoms, parts, counts)):
        t, _, _ = g.run_histories(p, n, p_absorb=PA, seed=SEED)
        assert np.array_equal(_u64(b.tallies[k]), _u64(t))


def test_batched_event_config4_full():
    # the whole 64-geometry workload: tallies equal the per-geometry runs
    members = _members(64, 0)
    geoms, parts = _build(members, exact=True)
    counts = [n for _, n in members]
    b = N.Batch(geoms, parts, counts)
    b.upload(16384)
    b.run(_ev(queue_depth=512))
    torch.cuda.synchronize()
    for k, (g, p, n) in enumerate(zip(geoms, parts, counts)):
        t, c, _ = g.run_histories(p, n, p_absorb=PA, seed=SEED)
        torch.cuda.synchronize()
        assert np.array_equal(_u64(b.tallies[k]), _u64(t)), k
        assert np.array_equal(_u64(b.counters)[16 * k:16 * k + 11], _u64(c)[:11]), k


def test_batched_event_round_limit():
    # a round limit far below what the histories need ends the launch with
    # TRK_E_TIMEOUT on a geometry's status counter; the context stays usable
    members = _members(3, 2_000)
    geoms, parts = _build(members, exact=False)
    b = N.Batch(geoms, parts, [n for _, n in members])
    b.upload(1000)
    b.run(_ev(queue_depth=64, max_rounds=3))
    torch.cuda.synchronize()
    st = _u64(b.counters).reshape(-1, 16)[:, N.K["status"]].view(np.int64)
    assert (st == -7).any()                              # TRK_E_TIMEOUT
    b.zero()
    b.run(_ev(queue_depth=64))
    torch.cuda.synchronize()
    assert _u64(b.counters).reshape(-1, 16)[:, N.K["status"]].sum() == 0


def test_batched_event_work_buffer_checks():
    members = _members(2, 500)
    geoms, parts = _build(members, exact=False)
    b = N.Batch(geoms, parts, [n for _, n in members])
    b.upload(512)
    with pytest.raises(N.TrkError):
        b.run(_ev(queue_depth=1024))
    with pytest.raises(N.TrkError):
        b.run(_ev(queue_depth=16))
