"""Delta queries on the GPU (gj_apply_batch) against the CPU oracle: the
change of every query's count and checksum must equal recount-after minus
recount-before exactly, the committed graph must equal the oracle's R + Delta R,
and the batch semantics (last update decides, self-loops ignored, no-op
updates dropped) must match the oracle's normalisation."""
import numpy as np
import pytest

import oracle
from paper_1802_03760_b300 import gj
from paper_1802_03760_b300.inputs import QUERIES, UpdateStream, rmat_edges

pytestmark = pytest.mark.gpu
M64 = (1 << 64) - 1
NAMES = sorted(QUERIES)


@pytest.fixture(scope="module", params=[gj.FLAG_DELTA_PLAIN, gj.FLAG_DELTA_FUSED, 0],
                ids=["level-sync", "fused", "by-size"])
def ctx(request):
    """Delta queries on the level-synchronous engine, on the fused one, and
    chosen by batch size (the default): all are checked."""
    c = gj.Context(0, flags=request.param)
    yield c
    c.close()


def random_batch(rng, n, g_edges, size, frac_del=0.3):
    bs = rng.integers(0, n, size)
    bd = rng.integers(0, n, size)
    bg = rng.choice([-1, 1], size)
    es, ed = g_edges
    if len(es):
        pick = rng.integers(0, len(es), max(1, int(frac_del * size)))
        bs = np.concatenate([bs, es[pick], bs[: size // 5]])  # deletes of existing edges, repeats
        bd = np.concatenate([bd, ed[pick], bd[: size // 5]])
        bg = np.concatenate([bg, -np.ones(len(pick), np.int64), -bg[: size // 5]])
    loops = rng.integers(0, n, 3)
    bs = np.concatenate([bs, loops])
    bd = np.concatenate([bd, loops])
    bg = np.concatenate([bg, np.ones(3, np.int64)])
    return bs.astype(np.uint32), bd.astype(np.uint32), bg.astype(np.int8)


@pytest.mark.parametrize("seed", range(8))
def test_random_batches_equal_recount(ctx, seed):
    rng = np.random.default_rng(300 + seed)
    n = int(rng.integers(20, 150))
    s = rng.integers(0, n, 6 * n).astype(np.uint32)
    d = rng.integers(0, n, 6 * n).astype(np.uint32)
    og = oracle.Graph(n, s, d)
    g = gj.Graph(ctx, s, d, n)
    qs = [gj.Query(ctx, *QUERIES[nm]) for nm in NAMES]
    oqs = [oracle.Query(*QUERIES[nm]) for nm in NAMES]
    before = [og.count(q) for q in oqs]
    for step in range(4):
        bs, bd, bg = random_batch(rng, n, og.edges(), int(rng.integers(1, 3 * n)))
        (cs, cd, cg), og2 = oracle.apply_batch(og, bs, bd, bg)
        after = [og2.count(q) for q in oqs]
        dc, dh = gj.apply_batch(g, bs, bd, bg, qs)
        for i, nm in enumerate(NAMES):
            assert dc[i] == after[i][0] - before[i][0], (nm, step)
            assert dh[i] == (after[i][1] - before[i][1]) & M64, (nm, step)
        assert gj.last_batch_changes(g) == len(cs)
        off, nbr = g.export()
        es, ed = og2.edges()
        assert np.array_equal(nbr, ed) and np.array_equal(np.repeat(np.arange(n), np.diff(off)), es)
        assert g.stats() == (og2.m, step + 1)
        # static counts on the committed graph, both engines
        for q, oq, nm in zip(qs, oqs, NAMES):
            for eng in (gj.ENGINE_PLAIN, gj.ENGINE_FUSED):
                assert gj.count(g, q, engine=eng) == og2.count(oq), (nm, eng)
        og, before = og2, after


def test_delta_order_and_direction_variants(ctx):
    rng = np.random.default_rng(7)
    n = 60
    s = rng.integers(0, n, 500).astype(np.uint32)
    d = rng.integers(0, n, 500).astype(np.uint32)
    og = oracle.Graph(n, s, d)
    g = gj.Graph(ctx, s, d, n)
    variants = [(4, [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)], [3, 2, 1, 0]),
                (4, [(1, 0), (0, 2), (3, 1), (2, 3), (1, 2)], [2, 3, 1, 0]),
                (3, [(0, 1), (1, 0), (1, 2), (2, 0)], None),
                (2, [(0, 1), (1, 0)], None)]
    qs = [gj.Query(ctx, k, at, o) for k, at, o in variants]
    oqs = [oracle.Query(k, at, o) for k, at, o in variants]
    for _ in range(3):
        bs, bd, bg = random_batch(rng, n, og.edges(), 80)
        (cs, cd, cg), og2 = oracle.apply_batch(og, bs, bd, bg)
        dc, dh = gj.apply_batch(g, bs, bd, bg, qs)
        for i, oq in enumerate(oqs):
            c0, h0 = og.count(oq)
            c1, h1 = og2.count(oq)
            assert (dc[i], dh[i]) == (c1 - c0, (h1 - h0) & M64), variants[i]
            assert (dc[i], dh[i]) == oracle.delta(og, og2, cs, cd, cg, oq)
        og = og2


def test_rmat_update_stream_against_delta_oracle(ctx):
    """The dynamic workload's shape at a size the oracle's Delta-GJ handles:
    R-MAT base graph, 90% R-MAT inserts / 10% deletes of existing edges."""
    scale = 13
    s, d = rmat_edges(scale, seed=5)
    n = 1 << scale
    og = oracle.Graph(n, s, d)
    g = gj.Graph(ctx, s, d, n)
    stream = UpdateStream(s, d, scale, seed=5)
    names = ["triangle", "4-clique"]
    qs = [gj.Query(ctx, *QUERIES[nm]) for nm in names]
    oqs = [oracle.Query(*QUERIES[nm]) for nm in names]
    total = [0, 0]
    c_start = [og.count(q)[0] for q in oqs]
    for b in (100, 1000, 1000, 100):
        bs, bd, bg = stream.next_batch(b)
        (cs, cd, cg), og2 = oracle.apply_batch(og, bs, bd, bg)
        dc, dh = gj.apply_batch(g, bs, bd, bg, qs)
        for i, oq in enumerate(oqs):
            assert (dc[i], dh[i]) == oracle.delta(og, og2, cs, cd, cg, oq), (names[i], b)
            total[i] += dc[i]
        og = og2
    # the deltas telescope to the recount difference over the stream
    for i, oq in enumerate(oqs):
        assert total[i] == og.count(oq)[0] - c_start[i]
        assert gj.count(g, qs[i]) == og.count(oq)


def test_batch_errors_leave_graph_unchanged(ctx):
    s = np.array([0, 1, 2], np.uint32)
    d = np.array([1, 2, 0], np.uint32)
    g = gj.Graph(ctx, s, d, 5)
    q = gj.Query(ctx, *QUERIES["cyclic-triangle"])
    with pytest.raises(gj.GJError) as ei:
        gj.apply_batch(g, [0], [9], [1], [q])
    assert ei.value.code == -2
    with pytest.raises(gj.GJError) as ei:
        gj.apply_batch(g, [0], [3], [2], [q])
    assert ei.value.code == -1
    assert g.stats() == (3, 0)
    assert gj.count(g, q)[0] == 3
    # an empty batch changes nothing but advances the version
    assert gj.apply_batch(g, np.array([], np.uint32), np.array([], np.uint32), np.array([], np.int8), [q]) == ([0], [0])
    assert g.stats() == (3, 1)
    # deleting the cycle's edge: all three rotations disappear
    dc, dh = gj.apply_batch(g, [1], [2], [-1], [q])
    assert dc == [-3] and gj.count(g, q) == (0, 0)


def test_device_batch_inputs(ctx):
    import torch
    rng = np.random.default_rng(17)
    n = 100
    s = rng.integers(0, n, 800).astype(np.uint32)
    d = rng.integers(0, n, 800).astype(np.uint32)
    og = oracle.Graph(n, s, d)
    g = gj.Graph(ctx, s, d, n)
    q = gj.Query(ctx, *QUERIES["triangle"])
    bs, bd, bg = random_batch(rng, n, og.edges(), 200)
    (cs, cd, cg), og2 = oracle.apply_batch(og, bs, bd, bg)
    dc, dh = gj.apply_batch(g, torch.from_numpy(bs.view(np.int32)).cuda(), torch.from_numpy(bd.view(np.int32)).cuda(),
                            torch.from_numpy(bg).cuda(), [q])
    oq = oracle.Query(*QUERIES["triangle"])
    assert dc[0] == og2.count(oq)[0] - og.count(oq)[0]


def test_commits_reuse_arrays_and_move_hash_sets(ctx):
    """A long stream of batches on one graph: each commit writes the next
    version into the previous version's arrays (shifting untouched lists and
    hash sets, rebuilding the touched ones). Lists cross the hash-set
    threshold of 16 entries both ways, and the exported index and every count
    equal the oracle's after each batch."""
    rng = np.random.default_rng(77)
    n = 300
    # vertex 5 has 15 out-neighbours (no hash set); vertex 9 has 17 (a hash set)
    s = np.concatenate([np.full(15, 5), np.full(17, 9), rng.integers(0, n, 2500)]).astype(np.uint32)
    d = np.concatenate([np.arange(20, 35), np.arange(40, 57), rng.integers(0, n, 2500)]).astype(np.uint32)
    og = oracle.Graph(n, s, d)
    g = gj.Graph(ctx, s, d, n)
    names = ["triangle", "diamond", "4-clique"]
    qs = [gj.Query(ctx, *QUERIES[nm]) for nm in names]
    oqs = [oracle.Query(*QUERIES[nm]) for nm in names]
    fixed = [
        (np.array([5, 5, 9, 9, 9], np.uint32), np.array([100, 101, 40, 41, 42], np.uint32),
         np.array([1, 1, -1, -1, -1], np.int8)),  # 5 -> 17 entries, 9 -> 14
        (np.array([5, 5, 5, 9, 9], np.uint32), np.array([100, 20, 21, 40, 200], np.uint32),
         np.array([-1, -1, -1, 1, 1], np.int8)),  # 5 -> 14, 9 -> 16
    ]
    for step in range(12):
        bs, bd, bg = fixed[step] if step < 2 else random_batch(rng, n, og.edges(), int(rng.integers(1, 400)))
        (cs, cd, cg), og2 = oracle.apply_batch(og, bs, bd, bg)
        dc, dh = gj.apply_batch(g, bs, bd, bg, qs)
        for i, q in enumerate(oqs):
            c0, h0 = og.count(q)
            c1, h1 = og2.count(q)
            assert (dc[i], dh[i]) == (c1 - c0, (h1 - h0) & M64), (step, names[i])
            assert gj.count(g, qs[i]) == (c1, h1), (step, names[i])
        off, nbr = g.export()
        es, ed = og2.edges()
        assert np.array_equal(nbr, ed) and np.array_equal(np.repeat(np.arange(n), np.diff(off)), es), step
        og = og2
