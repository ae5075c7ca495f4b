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

import oracle
from paper_1802_03760_b300 import gj
from paper_1802_03760_b300.inputs import QUERIES, SPECIALISED, er_edges, rmat_edges

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
            want_work = ctx.last_work().as_dict()
            assert sum(want[0]) > 0
            for _ in range(2):
                assert gj.count_noalloc(g, qs) == want
                assert ctx.last_work().as_dict() == want_work
        # both agree with the oracle on the small graph (not only with each other)
        og = oracle.Graph(2000, *er_edges(2000, 20000, seed=1))
        oracle_want = [og.count(oracle.Query(*QUERIES[nm])) for nm in names]
        assert list(zip(*gj.count_noalloc(g_small, qs))) == oracle_want
        # a smaller query set after a larger one: stale plans or counters must not leak in
        sub = [qs[names.index("triangle")], qs[names.index("4-clique")]]
        want = gj.count_many(g_rmat, sub, engine=gj.ENGINE_FUSED)
        assert gj.count_noalloc(g_rmat, sub) == want
        assert gj.count_noalloc(g_rmat, sub) == want
        # the context's launch settings apply here too (results never depend on them)
        gj.set_tuning(ctx, seed_chunk=128, blocks_per_sm=1)
        assert gj.count_noalloc(g_rmat, sub) == want
        gj.set_tuning(ctx)
    finally:
        ctx.close()


def test_noalloc_needs_a_built_triangle_index():
    """A query over the triangle index would have to build it (an allocation):
    refused until the index exists, then counted like the other entry points."""
    ctx = gj.Context(0)
    try:
        s, d = er_edges(500, 6000, seed=4)
        g = gj.Graph(ctx, s, d, 500)
        sp = SPECIALISED["4-clique-tr"]
        q = gj.Query(ctx, sp["k"], sp["atoms"], sp["order"], tri=sp["tri"], lt=sp["lt"])
        with pytest.raises(gj.GJError) as ei:
            gj.count_noalloc(g, [q])
        assert ei.value.code == -1 and "triangle index" in str(ei.value)
        g.build_triangles()
        want = gj.count_many(g, [q], engine=gj.ENGINE_FUSED)
        assert gj.count_noalloc(g, [q]) == want
        assert gj.count_noalloc(g, [q]) == want
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
