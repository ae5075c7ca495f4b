"""The seeded input generators against the recipes they state. They stand
in for the paper's datasets (Section 5, Table 1) and feed both the oracle
and the CUDA path: R-MAT quadrant probabilities at every recursion level,
the seeded relabelling, the directed Erdos-Renyi draw, planted hubs, update
streams (inserts from an independent R-MAT stream, deletes of distinct base
edges, each batch a pure function of the seed and the batch sizes) and the
mixed-query list."""
import json
import os

import numpy as np
import pytest

from paper_1802_03760_b300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_stream_is_splitmix64():
    gold = json.load(open(os.path.join(GOLDEN, "splitmix64_seed0.json")))
    for i, want in enumerate(gold["outputs"]):
        assert I.subseed(0, i) == int(want, 16)


def test_rmat_quadrant_probabilities_per_level():
    scale, N = 10, 200_000
    s, d = I.rmat_edges(scale, count=N, permute=False, seed=5)
    assert s.max() < (1 << scale) and d.max() < (1 << scale)
    a, b, c = I.RMAT_ABC
    want = np.array([a, b, c, 1 - a - b - c])
    for bit in range(scale):  # the first recursion level decides the most significant bit
        q = ((s >> bit) & 1).astype(np.int64) * 2 + ((d >> bit) & 1).astype(np.int64)
        freq = np.bincount(q, minlength=4) / N
        # five binomial standard deviations at N = 200,000 is below 0.006
        assert np.all(np.abs(freq - want) < 0.006), (bit, freq)


def test_rmat_relabelling_slices_and_seeds():
    scale, n = 9, 1 << 9
    s, d = I.rmat_edges(scale, seed=3)
    assert len(s) == 16 * n
    raw_s, raw_d = I.rmat_edges(scale, seed=3, permute=False)
    perm = I.permutation(n, I.subseed(3, 7))
    assert sorted(perm.tolist()) == list(range(n))
    assert np.array_equal(s, perm[raw_s]) and np.array_equal(d, perm[raw_d])
    # a sample depends only on (seed, stream, its index)
    ps, pd = I.rmat_edges(scale, seed=3, first=1000, count=77)
    assert np.array_equal(ps, s[1000:1077]) and np.array_equal(pd, d[1000:1077])
    s2, d2 = I.rmat_edges(scale, seed=3)
    assert np.array_equal(s, s2) and np.array_equal(d, d2)
    s3, _ = I.rmat_edges(scale, seed=4)
    assert not np.array_equal(s, s3)
    i3, _ = I.rmat_edges(scale, seed=3, stream=3)
    assert not np.array_equal(s, i3)


def test_er_edges_distinct_no_loops():
    n, m = 200, 5000
    s, d = I.er_edges(n, m, seed=2)
    assert len(s) == m and s.max() < n and d.max() < n and not np.any(s == d)
    assert len({(int(u), int(v)) for u, v in zip(s, d)}) == m
    s2, d2 = I.er_edges(n, m, seed=2)
    assert np.array_equal(s, s2) and np.array_equal(d, d2)
    assert sorted(zip(*I.er_edges(3, 6, seed=1))) == [(u, v) for u in range(3) for v in range(3) if u != v]
    with pytest.raises(ValueError):
        I.er_edges(3, 7, seed=1)


def test_distinct_edges_is_the_sorted_edge_set():
    rng = np.random.default_rng(0)
    s = rng.integers(0, 30, 2000).astype(np.uint32)
    d = rng.integers(0, 30, 2000).astype(np.uint32)
    us, ud = I.distinct_edges(s, d)
    want = sorted({(int(u), int(v)) for u, v in zip(s, d) if u != v})
    assert list(zip(us.tolist(), ud.tolist())) == want


def test_hub_edges():
    n, h, deg = 5000, 6, 700
    ids, s, d = I.hub_edges(n, h, deg, seed=4)
    assert len(set(ids.tolist())) == h
    for k, hub in enumerate(ids.tolist()):
        out_s, out_d = s[2 * k * deg:(2 * k + 1) * deg], d[2 * k * deg:(2 * k + 1) * deg]
        in_s, in_d = s[(2 * k + 1) * deg:(2 * k + 2) * deg], d[(2 * k + 1) * deg:(2 * k + 2) * deg]
        assert np.all(out_s == hub) and len(set(out_d.tolist())) == deg and hub not in set(out_d.tolist())
        assert np.all(in_d == hub) and len(set(in_s.tolist())) == deg and hub not in set(in_s.tolist())
    with pytest.raises(ValueError):
        I.hub_edges(100, 1, 100, seed=1)


def test_update_stream():
    scale = 10
    s, d = I.rmat_edges(scale, seed=6)
    bs, bd = I.distinct_edges(s, d)
    base = set(zip(bs.tolist(), bd.tolist()))
    st = I.UpdateStream(s, d, scale, seed=6)
    deleted = set()
    cursor = 0
    batches = []
    for b in (1000, 37, 2500):
        src, dst, sign = st.next_batch(b)
        batches.append((src, dst, sign))
        ni = int(round(0.9 * b))
        assert len(src) == b and np.all(sign[:ni] == 1) and np.all(sign[ni:] == -1)
        ins_s, ins_d = I.rmat_edges(scale, seed=6, first=cursor, count=ni, stream=3)
        cursor += ni
        assert np.array_equal(src[:ni], ins_s) and np.array_equal(dst[:ni], ins_d)
        dels = list(zip(src[ni:].tolist(), dst[ni:].tolist()))
        assert set(dels) <= base and len(set(dels)) == len(dels) and not (set(dels) & deleted)
        deleted |= set(dels)
    st2 = I.UpdateStream(s, d, scale, seed=6)
    for b, (src, dst, sign) in zip((1000, 37, 2500), batches):
        s2, d2, g2 = st2.next_batch(b)
        assert np.array_equal(src, s2) and np.array_equal(dst, d2) and np.array_equal(sign, g2)
    small = I.UpdateStream(np.array([0, 1], np.uint32), np.array([1, 2], np.uint32), scale, seed=1)
    with pytest.raises(ValueError):
        small.next_batch(100)  # 10 deletes requested, 2 base edges


def test_mixed_queries():
    mq = I.mixed_queries(64, seed=3)
    assert len(mq) == 64 and len({nm for nm, *_ in mq}) == 64
    shapes = ["triangle", "4-cycle", "diamond", "4-clique", "5-clique"]
    for (nm, k, atoms, order), shape in zip(mq[:5], shapes):
        assert (nm, k, atoms, order) == (shape, I.QUERIES[shape][0], list(I.QUERIES[shape][1]), list(range(k)))
    for nm, k, atoms, order in mq:
        shape = nm.split("-v")[0]
        assert k == I.QUERIES[shape][0] and sorted(order) == list(range(k))
        assert [tuple(sorted(a)) for a in atoms] == [tuple(sorted(a)) for a in I.QUERIES[shape][1]]
        assert I.connected_order(atoms, order)
    assert mq == I.mixed_queries(64, seed=3)
    assert mq[5:] != I.mixed_queries(64, seed=4)[5:]
