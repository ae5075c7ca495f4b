"""Many queries in one persistent launch (the batched multi-query workload's
shape at a size the oracle finishes), launch-setting invariance, and the
autotuner: counts and checksums must not depend on the settings."""
import numpy as np
import pytest

import oracle
from paper_1802_03760_b300 import gj
from paper_1802_03760_b300.inputs import mixed_queries, rmat_edges

pytestmark = pytest.mark.gpu
M64 = (1 << 64) - 1


@pytest.fixture(scope="module")
def setup():
    scale = 9
    s, d = rmat_edges(scale, seed=9)
    n = 1 << scale
    ctx = gj.Context(0)
    g = gj.Graph(ctx, s, d, n)
    mq = mixed_queries(64, seed=3)
    qs = [gj.Query(ctx, k, atoms, order) for _, k, atoms, order in mq]
    og = oracle.Graph(n, s, d)
    want = [og.count(oracle.Query(k, atoms, order), mode=1) for _, k, atoms, order in mq]
    yield ctx, g, qs, want, n
    ctx.close()


def test_64_queries_one_launch(setup):
    ctx, g, qs, want, n = setup
    l0 = ctx.launches
    c, h = gj.count_many(g, qs, engine=gj.ENGINE_FUSED)
    assert ctx.launches - l0 == 3  # seed ranges, work-queue reset, one persistent launch for all 64 queries
    assert list(zip(c, h)) == want


@pytest.mark.parametrize("chunk,bps,donation", [(64, 0, 0), (128, 1, 1), (256, 2, 2), (32, 1, 1), (32, 0, 1),
                                                (8, 0, 1), (16, 0, 0), (40, 1, 1)])
def test_fused_settings_do_not_change_results(setup, chunk, bps, donation):
    """Seeds per grab, blocks per SM and work donation (1 = donate whenever a
    queue slot is free, which exercises the queue on every descent) must not
    change any count or checksum."""
    ctx, g, qs, want, n = setup
    gj.set_tuning(ctx, seed_chunk=chunk, blocks_per_sm=bps, donation=donation)
    try:
        assert list(zip(*gj.count_many(g, qs, engine=gj.ENGINE_FUSED))) == want
    finally:
        gj.set_tuning(ctx)


@pytest.mark.parametrize("budget", [1 << 20, 64 << 20])
def test_plain_budget_does_not_change_results(setup, budget):
    ctx, g, qs, want, n = setup
    gj.set_tuning(ctx, prefix_buffer_bytes=budget)
    try:
        sub = list(range(0, 64, 7))
        c, h = gj.count_many(g, [qs[i] for i in sub], engine=gj.ENGINE_PLAIN)
        assert list(zip(c, h)) == [want[i] for i in sub]
    finally:
        gj.set_tuning(ctx)


def test_sampled_ranges_add_up(setup):
    ctx, g, qs, want, n = setup
    tc = np.zeros(64, dtype=object)
    th = np.zeros(64, dtype=object)
    for lo in range(0, n, n // 8):
        c, h = gj.count_many(g, qs, v_range=(lo, lo + n // 8))
        tc += np.array(c, dtype=object)
        th = (th + np.array(h, dtype=object)) % (1 << 64)
    assert list(zip(tc.tolist(), th.tolist())) == want


def test_autotune_picks_valid_settings(setup):
    ctx, g, qs, want, n = setup
    t = gj.autotune(g, qs[:10], v_range=(0, n // 4), prefix_cap_bytes=256 << 20)
    assert t["seed_chunk"] in (8, 32, 128)
    assert t["prefix_buffer_bytes"] in (64 << 20, 256 << 20)
    assert t["fused_ms"] > 0 and t["plain_ms"] > 0
    assert gj.get_tuning(ctx)["seed_chunk"] == t["seed_chunk"]
    assert list(zip(*gj.count_many(g, qs))) == want
    gj.set_tuning(ctx)
    with pytest.raises(gj.GJError):
        gj.set_tuning(ctx, seed_chunk=44)
