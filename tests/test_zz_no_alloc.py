"""gj_count_noalloc: the fused multi-query count for callers that cannot
allocate device memory during the call (their device memory belongs to
another framework's pool, or an allocation's implicit device synchronization
would stall their other streams). Its scratch is a fixed array inside the
library, so it must give the same counts and checksums as gj_count_many on
every call, including a second call right after the first (the array keeps
the previous call's contents and must be cleared where it accumulates).

This file is named to be collected last."""
import numpy as np
import pytest

from paper_1802_03760_b300 import gj
from paper_1802_03760_b300.inputs import QUERIES, er_edges, rmat_edges

pytestmark = pytest.mark.gpu


def test_noalloc_matches_count_many_on_consecutive_calls():
    ctx = gj.Context(0)
    try:
        s, d = er_edges(2000, 20000, seed=1)
        g_small = gj.Graph(ctx, s, d, 2000)
        s, d = rmat_edges(14, seed=3)
        g_rmat = gj.Graph(ctx, s, d, 1 << 14)
        names = sorted(QUERIES)
        qs = [gj.Query(ctx, *QUERIES[nm]) for nm in names]
        for g in (g_small, g_rmat):
            want = gj.count_many(g, qs, engine=gj.ENGINE_FUSED)
            assert sum(want[0]) > 0
            for _ in range(2):
                assert gj.count_noalloc(g, qs) == want
        # a smaller query set after a larger one: stale plans or counters must not leak in
        sub = [qs[names.index("triangle")], qs[names.index("4-clique")]]
        want = gj.count_many(g_rmat, sub, engine=gj.ENGINE_FUSED)
        assert gj.count_noalloc(g_rmat, sub) == want
        assert gj.count_noalloc(g_rmat, sub) == want
    finally:
        ctx.close()


def test_noalloc_rejects_more_queries_than_its_scratch_holds():
    ctx = gj.Context(0)
    try:
        s, d = er_edges(200, 1000, seed=2)
        g = gj.Graph(ctx, s, d, 200)
        q = gj.Query(ctx, *QUERIES["triangle"])
        with pytest.raises(gj.GJError) as ei:
            gj.count_noalloc(g, [q] * 65)
        assert ei.value.code == -1
        assert "at most 64" in str(ei.value)
        c, h = gj.count_noalloc(g, [q] * 64)
        assert len(set(c)) == 1 and c[0] == gj.count(g, q)[0]
    finally:
        ctx.close()
