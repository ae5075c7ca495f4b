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


# The recipe restated in plain Python, draw by draw: SplitMix64 output of
# state seed + (ctr + 1) * 0x9e3779b97f4a7c15; stream seeds subseed(seed, tag)
# = draw tag of stream seed; uniform integers below a bound by multiply-high.
M64 = (1 << 64) - 1
GOLDEN_GAMMA = 0x9E3779B97F4A7C15


def py_mix64(z):
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def py_rand(seed, ctr):
    return py_mix64((seed + (ctr + 1) * GOLDEN_GAMMA) & M64)


def py_below(r, bound):
    return (r * bound) >> 64


def test_rmat_samples_follow_the_recipe_exactly():
    """Sample e, level l: a 53-bit uniform from draw e * 64 + l of stream
    subseed(seed, 2) picks the quadrant (a, b, c, d); the first level sets
    the most significant bit; ids then pass through the permutation of
    stream subseed(seed, 7)."""
    scale, seed, count = 12, 1, 96
    a, b, c = I.RMAT_ABC
    st = py_rand(seed, 2)
    s, d = I.rmat_edges(scale, seed=seed, permute=False, count=count)
    for e in range(count):
        u = v = 0
        for lvl in range(scale):
            x = (py_rand(st, e * 64 + lvl) >> 11) * (1.0 / 9007199254740992.0)
            q = 0 if x < a else 1 if x < a + b else 2 if x < a + b + c else 3
            u, v = (u << 1) | (q >> 1), (v << 1) | (q & 1)
        assert (int(s[e]), int(d[e])) == (u, v), e
    ps, pd = I.rmat_edges(scale, seed=seed, count=count)
    perm = I.permutation(1 << scale, py_rand(seed, 7))
    assert np.array_equal(ps, perm[s]) and np.array_equal(pd, perm[d])


def test_permutation_is_fisher_yates_on_the_stream():
    n, seed = 1000, 12345
    want = list(range(n))
    for i in range(n, 1, -1):
        j = py_below(py_rand(seed, i), i)
        want[i - 1], want[j] = want[j], want[i - 1]
    assert I.permutation(n, seed).tolist() == want


def test_er_draws_follow_the_recipe_exactly():
    """Draw ctr of stream subseed(seed, 1) gives u from its low and v from its
    high 32 bits, each scaled to [0, n) by multiply-high; pairs with u == v
    and repeats are skipped."""
    n, m, seed = 37, 300, 9
    st = py_rand(seed, 1)
    want, seen, ctr = [], set(), 0
    while len(want) < m:
        r = py_rand(st, ctr)
        ctr += 1
        u, v = ((r & 0xFFFFFFFF) * n) >> 32, ((r >> 32) * n) >> 32
        if u != v and (u, v) not in seen:
            seen.add((u, v))
            want.append((u, v))
    s, d = I.er_edges(n, m, seed=seed)
    assert list(zip(s.tolist(), d.tolist())) == want


def test_uniform_draws_follow_the_recipe_exactly():
    bound, seed, first = 1_000_003, 77, 5
    got = I.uniform(bound, 40, seed, first=first)
    assert got.tolist() == [py_below(py_rand(seed, first + i), bound) for i in range(40)]
    assert I.subseed(seed, 3) == py_rand(seed, 3)


def test_hubs_follow_the_recipe_exactly():
    """Hub ids: distinct draws below n from stream subseed(seed, 11). Hub h's
    out- (t = 2h) and in-neighbours (t = 2h + 1): distinct draws below n,
    skipping the hub, from the stream seeded subseed(seed, 12) xor
    0x5bd1e995 * (t + 1)."""
    n, nh, deg, seed = 500, 3, 40, 8
    ids, ctr = [], 0
    while len(ids) < nh:
        x = py_below(py_rand(py_rand(seed, 11), ctr), n)
        ctr += 1
        if x not in ids:
            ids.append(x)
    base = py_rand(seed, 12)
    want_s, want_d = [], []
    for t in range(2 * nh):
        hub = ids[t // 2]
        st = base ^ ((0x5BD1E995 * (t + 1)) & M64)
        seen, got, ctr = {hub}, [], 0
        while len(got) < deg:
            x = py_below(py_rand(st, ctr), n)
            ctr += 1
            if x not in seen:
                seen.add(x)
                got.append(x)
        if t % 2:
            want_s += got
            want_d += [hub] * deg
        else:
            want_s += [hub] * deg
            want_d += got
    gi, gs, gd = I.hub_edges(n, nh, deg, seed=seed)
    assert gi.tolist() == ids and gs.tolist() == want_s and gd.tolist() == want_d
