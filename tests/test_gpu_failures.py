"""Failure detection without a GPU fault: the fused engine's end-of-launch
wait is bounded in time (it gives up once the work-donation queue shows no
progress for the bound) and a count that passes 2^63 - 1 is reported as
GJ_E_OVERFLOW. Both are driven by the context's failure-injection setting:
the wait is made to expect a warp that never arrives, or the counts start
just below 2^63. In each case the call returns the error status and the
context stays usable."""
import time

import numpy as np
import pytest

import oracle
from paper_1802_03760_b300 import gj
from paper_1802_03760_b300.inputs import QUERIES, er_edges

pytestmark = pytest.mark.gpu
GJ_E_TIMEOUT, GJ_E_OVERFLOW = -6, -7


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
