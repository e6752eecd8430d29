"""The library's sharded runs on one GPU: the benchmark's layout (contiguous
particle-id ranges, each rank running source_init + run_histories on its
range with first_id set) executed range after range, the tallies and
counters summed.  Integer tallies and id-keyed random numbers make the sum
equal to the unsplit run bit for bit, in both builds and both kernels."""
import numpy as np
import pytest
import torch

from paper_2406_13849_gb300 import inputs as I
from paper_2406_13849_gb300 import native as N
from paper_2406_13849_gb300 import sharding as S

pytestmark = pytest.mark.gpu


def _run(g, first, n, mode):
    parts = g.source_init(n, seed=1, first_id=first)
    tally, cnt, _ = g.run_histories(parts, n, tracker=N.TRACKER_CSG, mode=mode, queue_depth=512, first_id=first,
                                    seed=1, p_absorb=0.25)
    return tally, cnt


@pytest.mark.parametrize("exact", [True, False])
@pytest.mark.parametrize("mode", [N.MODE_EVENT, N.MODE_HISTORY])
@pytest.mark.parametrize("world", [2, 3])
def test_id_range_shards_sum_to_the_whole_run(exact, mode, world):
    desc = I.config2()
    g = N.Geometry(I.to_json(desc), exact=exact)
    n_total = 300_001
    whole_t, whole_c = _run(g, 0, n_total, mode)
    sum_t = torch.zeros_like(whole_t)
    sum_c = torch.zeros_like(whole_c)
    for r in range(world):
        first, n = S.shard_range(n_total, r, world)
        t, c = _run(g, first, n, mode)
        sum_t += t
        sum_c += c
    torch.cuda.synchronize()
    assert torch.equal(sum_t, whole_t)
    assert torch.equal(sum_c, whole_c)
    assert int(whole_c[N.K["segments"]]) > 20 * n_total
