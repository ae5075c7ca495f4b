"""Failure detection without a GPU fault: the fused engine's end-of-launch
wait is bounded in time (it gives up once the work-donation queue shows no
progress for the bound), a count that passes 2^63 - 1 is reported as
GJ_E_OVERFLOW, and a failed device allocation anywhere in a call is
reported as GJ_E_NOMEM with the graph left as it was. All are driven by
the context's failure-injection setting: the wait is made to expect a warp
that never arrives, the counts start just below 2^63, or the allocations
after the first k fail (on the host, before anything is launched with
them). In each case the call returns the error status and the context
stays usable."""
import time

import numpy as np
import pytest

import oracle
from paper_1802_03760_b300 import gj
from paper_1802_03760_b300.inputs import QUERIES, er_edges

pytestmark = pytest.mark.gpu
GJ_E_NOMEM, GJ_E_TIMEOUT, GJ_E_OVERFLOW = -3, -6, -7


@pytest.fixture(scope="module")
def setup():
    ctx = gj.Context(0)
    s, d = er_edges(2000, 20000, seed=1)
    og = oracle.Graph(2000, s, d)
    g = gj.Graph(ctx, s, d, 2000)
    names = ["triangle", "diamond", "4-clique"]
    qs = [gj.Query(ctx, *QUERIES[nm]) for nm in names]
    want = [og.count(oracle.Query(*QUERIES[nm])) for nm in names]
    yield ctx, g, qs, want
    ctx.close()


def test_wait_without_progress_times_out(setup):
    ctx, g, qs, want = setup
    gj.set_tuning(ctx, wait_ms=50, fault=1)
    try:
        t0 = time.perf_counter()
        with pytest.raises(gj.GJError) as ei:
            gj.count_many(g, qs, engine=gj.ENGINE_FUSED)
        assert ei.value.code == GJ_E_TIMEOUT and "bounded wait" in str(ei.value)
        assert time.perf_counter() - t0 < 30.0
        assert gj.get_tuning(ctx)["wait_ms"] == 50
    finally:
        gj.set_tuning(ctx)
    # the context still works and gives the oracle's counts
    assert list(zip(*gj.count_many(g, qs, engine=gj.ENGINE_FUSED))) == want


def test_default_bound_does_not_fire_on_real_work(setup):
    ctx, g, qs, want = setup
    gj.set_tuning(ctx, donation=1)  # every batch through the queue: the most waiting
    try:
        assert list(zip(*gj.count_many(g, qs, engine=gj.ENGINE_FUSED))) == want
    finally:
        gj.set_tuning(ctx)


def test_count_past_int64_is_an_overflow(setup):
    ctx, g, qs, want = setup
    small = gj.Query(ctx, 2, [(0, 1)], None, lt=[(0, 1)])  # edges u -> v with u < v
    og = oracle.Graph(2000, *er_edges(2000, 20000, seed=1))
    want_small = og.count(oracle.Query(2, [(0, 1)], None, lt=[(0, 1)]), mode=1)
    assert want_small[0] > 1023
    tiny_s = np.array([0, 1, 2], np.uint32)
    tiny_d = np.array([1, 2, 0], np.uint32)
    tiny = gj.Graph(ctx, tiny_s, tiny_d, 3)
    gj.set_tuning(ctx, fault=2)
    try:
        with pytest.raises(gj.GJError) as ei:
            gj.count_many(g, [small], engine=gj.ENGINE_FUSED)
        assert ei.value.code == GJ_E_OVERFLOW
        # below the injected margin the counts are still exact
        assert gj.count_many(tiny, [small], engine=gj.ENGINE_FUSED)[0] == [2]
    finally:
        gj.set_tuning(ctx)
        tiny.free()
    assert gj.count(g, small, engine=gj.ENGINE_FUSED) == want_small


def _try(f):
    """f()'s result, or None if it failed with GJ_E_NOMEM."""
    try:
        return f()
    except gj.GJError as e:
        assert e.code == GJ_E_NOMEM, (e.code, str(e))
        return None


def test_allocation_failures_leave_no_trace():
    """For k = 0, 1, 2, ... the allocations after the first k fail: graph
    loads (with degree renaming and orientation), triangle-index builds,
    count calls on both engines of a fresh context and update batches either
    succeed with the oracle's results or return GJ_E_NOMEM; a failed batch
    leaves the graph's edges and version unchanged. The sweep ends once
    every call gets all the allocations it needs."""
    n = 600
    s, d = er_edges(n, 6000, seed=9)
    og = oracle.Graph(n, s, d)
    want_tri = og.transform(False, True, True)[0].num_triangles()
    want_4 = og.count(oracle.Query(*QUERIES["4-clique"]))
    names = ["triangle", "4-clique"]
    oq = [oracle.Query(*QUERIES[nm]) for nm in names]
    ctx = gj.Context(0)
    qs = [gj.Query(ctx, *QUERIES[nm]) for nm in names]
    g = gj.Graph(ctx, s, d, n)
    rng = np.random.default_rng(9)
    k, all_ok = 0, False
    while not all_ok:
        assert k < 300
        bs = rng.integers(0, n, 50).astype(np.uint32)
        bd = rng.integers(0, n, 50).astype(np.uint32)
        bg = rng.choice(np.array([-1, 1], np.int8), 50)
        before = g.stats()
        gj.set_tuning(ctx, fault=4, fault_count=k)
        g2 = _try(lambda: gj.Graph(ctx, s, d, n, flags=gj.LOAD_DEGREE_ORDER | gj.LOAD_ORIENT))
        gj.set_tuning(ctx, fault=4, fault_count=k)
        tri = _try(g2.build_triangles) if g2 is not None else None
        gj.set_tuning(ctx, fault=4, fault_count=k)
        res = _try(lambda: gj.apply_batch(g, bs, bd, bg, qs))
        gj.set_tuning(ctx)
        if g2 is not None:
            g2.free()
        if res is None:
            assert g.stats() == before, k
        else:
            (cs, cd, cg), og2 = oracle.apply_batch(og, bs, bd, bg)
            assert list(zip(*res)) == [oracle.delta(og, og2, cs, cd, cg, q) for q in oq], k
            og = og2
        assert tri is None or tri == want_tri, k
        # a fresh context, whose scratch buffers are still to be allocated
        c2 = gj.Context(0)
        g3 = gj.Graph(c2, s, d, n)
        q3 = gj.Query(c2, *QUERIES["4-clique"])
        cnt = []
        for e in (gj.ENGINE_PLAIN, gj.ENGINE_FUSED):
            gj.set_tuning(c2, fault=4, fault_count=k)
            cnt.append(_try(lambda: gj.count(g3, q3, engine=e)))
        gj.set_tuning(c2)
        assert all(c is None or c == want_4 for c in cnt), k
        assert gj.count(g3, q3, engine=gj.ENGINE_FUSED) == want_4
        c2.close()
        all_ok = None not in (g2, tri, res) and None not in cnt
        k += 1
    assert k > 3  # the sweep did reach failures deep inside the calls
    assert [gj.count(g, q) for q in qs] == [og.count(q) for q in oq]
    ctx.close()
