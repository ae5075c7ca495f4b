"""Parity of the CUDA path (through the C ABI) with the CPU oracle: counts and
checksums must be bit-exact. Sizes span many warps' batches and ragged tails;
the R-MAT scale-20 workload is checked on sampled first-attribute ranges the
oracle can finish, plus properties that hold at any size."""
import itertools

import numpy as np
import pytest

import oracle
from paper_1802_03760_b300 import gj
from paper_1802_03760_b300.inputs import QUERIES, er_edges, rmat_edges

pytestmark = pytest.mark.gpu
M64 = (1 << 64) - 1
ENGINES = [gj.ENGINE_PLAIN, gj.ENGINE_FUSED]


@pytest.fixture(scope="module")
def ctx():
    c = gj.Context(0)
    yield c
    c.close()


def valid_order(k, atoms, order):
    pos = {a: i for i, a in enumerate(order)}
    if not any({pos[s], pos[d]} == {0, 1} for s, d in atoms):
        return False
    for j in range(2, k):
        if not any((pos[s] == j and pos[d] < j) or (pos[d] == j and pos[s] < j) for s, d in atoms):
            return False
    return True


def random_graph(rng, n, m, recip=0.2):
    s = rng.integers(0, n, m).astype(np.uint32)
    d = rng.integers(0, n, m).astype(np.uint32)
    r = rng.random(m) < recip
    s = np.concatenate([s, d[r]])
    d = np.concatenate([d, s[: m][r]])
    return s, d


def test_er2000_all_queries(ctx):
    s, d = er_edges(2000, 20000, seed=1)
    og = oracle.Graph(2000, s, d)
    g = gj.Graph(ctx, s, d, 2000)
    assert g.m == og.m == 20000
    for name, (k, atoms) in QUERIES.items():
        want = og.count(oracle.Query(k, atoms))
        for eng in ENGINES:
            assert gj.count(g, gj.Query(ctx, k, atoms), engine=eng) == want, (name, eng)


def test_index_matches_oracle(ctx):
    rng = np.random.default_rng(3)
    s, d = random_graph(rng, 3000, 40000)
    s = np.concatenate([s, np.arange(50, dtype=np.uint32)])  # self-loops
    d = np.concatenate([d, np.arange(50, dtype=np.uint32)])
    og = oracle.Graph(3000, s, d)
    g = gj.Graph(ctx, s, d, 3000)
    off, nbr = g.export()
    os_, od = og.edges()
    assert g.m == og.m
    assert np.array_equal(nbr, od)
    assert np.array_equal(np.repeat(np.arange(3000), np.diff(off)), os_)


@pytest.mark.parametrize("seed", range(12))
def test_random_graphs_random_orders(ctx, seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(20, 400))
    m = int(rng.integers(100, 6000))
    s, d = random_graph(rng, n, m, recip=float(rng.uniform(0, 0.5)))
    og = oracle.Graph(n, s, d)
    g = gj.Graph(ctx, s, d, n)
    for name, (k, atoms) in sorted(QUERIES.items()):
        # flip some atom directions, pick a random valid order
        atoms = [(b, a) if rng.random() < 0.3 else (a, b) for a, b in atoms]
        orders = [o for o in itertools.permutations(range(k)) if valid_order(k, atoms, o)]
        order = list(orders[int(rng.integers(0, len(orders)))])
        want, wh, st = og.count(oracle.Query(k, atoms, order), stats=True, mode=1)
        q = gj.Query(ctx, k, atoms, order)
        for eng in ENGINES:
            c, h, w = gj.count(g, q, engine=eng, stats=True)
            assert (c, h) == (want, wh), (name, order, eng)
            for j in range(2, k):
                assert w.extended[j] == st.extended[j], (name, eng, j)
                assert w.proposals[j] == st.proposals[j], (name, eng, j)
                assert w.nbind[j] == st.nbind_sum[j], (name, eng, j)
            for j in range(3, k + 1):
                assert w.produced[j] == st.prefixes[j], (name, eng, j)


def test_extra_atoms_over_seed_pair(ctx):
    """Atoms over the first two attributes besides the seed atom filter the seeds."""
    rng = np.random.default_rng(5)
    s, d = random_graph(rng, 60, 900, recip=0.5)
    og = oracle.Graph(60, s, d)
    g = gj.Graph(ctx, s, d, 60)
    for k, atoms in [(2, [(0, 1), (1, 0)]), (2, [(0, 1)]), (3, [(0, 1), (1, 0), (1, 2), (2, 0)]),
                     (3, [(1, 0), (0, 1), (0, 1), (2, 1), (0, 2)])]:
        want = og.count(oracle.Query(k, atoms))
        for eng in ENGINES:
            assert gj.count(g, gj.Query(ctx, k, atoms), engine=eng) == want, (atoms, eng)


@pytest.mark.parametrize("eng", ENGINES)
def test_edge_cases(ctx, eng):
    tri = gj.Query(ctx, *QUERIES["triangle"])
    clique = gj.Query(ctx, *QUERIES["4-clique"])
    e = np.array([], np.uint32)
    g = gj.Graph(ctx, e, e, 10)
    assert g.m == 0
    assert gj.count(g, tri, engine=eng) == (0, 0)
    loops = np.arange(10, dtype=np.uint32)
    g = gj.Graph(ctx, loops, loops, 10)
    assert g.m == 0 and gj.count(g, clique, engine=eng) == (0, 0)
    g = gj.Graph(ctx, np.array([3], np.uint32), np.array([7], np.uint32), 10)
    assert g.m == 1 and gj.count(g, tri, engine=eng) == (0, 0)
    # duplicates of a single triangle
    s = np.array([0, 1, 0, 0, 1, 0], np.uint32)
    d = np.array([1, 2, 2, 1, 2, 2], np.uint32)
    og = oracle.Graph(3, s, d)
    g = gj.Graph(ctx, s, d, 3)
    assert gj.count(g, tri, engine=eng) == og.count(oracle.Query(*QUERIES["triangle"])) and g.m == 3
    # complete DAG on 40 vertices: closed forms C(n,3), C(n,4)
    n = 40
    s, d = np.triu_indices(n, 1)
    g = gj.Graph(ctx, s.astype(np.uint32), d.astype(np.uint32), n)
    assert gj.count(g, tri, engine=eng)[0] == 9880
    assert gj.count(g, clique, engine=eng)[0] == 91390


def test_vertex_range_errors(ctx):
    with pytest.raises(gj.GJError) as ei:
        gj.Graph(ctx, np.array([1, 2], np.uint32), np.array([2, 9], np.uint32), 5)
    assert ei.value.code == -2


def test_create_rejects_device_past_the_last():
    import ctypes
    h = ctypes.c_void_p()
    assert gj.lib().gj_create(1 << 20, None, ctypes.byref(h)) == -1 and not h.value


def test_invalid_queries(ctx):
    for k, atoms, order in [(3, [(0, 0), (1, 2)], None), (3, [(0, 1)], None), (3, [(0, 1), (1, 2)], [0, 0, 1]),
                            (3, [(0, 1), (1, 2)], [0, 2, 1]), (4, [(0, 1), (2, 3)], None), (1, [(0, 0)], None)]:
        with pytest.raises(gj.GJError) as ei:
            gj.Query(ctx, k, atoms, order)
        assert ei.value.code == -1


def test_device_inputs(ctx):
    import torch
    rng = np.random.default_rng(9)
    s, d = random_graph(rng, 500, 8000)
    og = oracle.Graph(500, s, d)
    g = gj.Graph(ctx, torch.from_numpy(s.astype(np.int32)).cuda(), torch.from_numpy(d.astype(np.int32)).cuda(), 500)
    for name in ("triangle", "diamond"):
        k, atoms = QUERIES[name]
        assert gj.count(g, gj.Query(ctx, k, atoms)) == og.count(oracle.Query(k, atoms))


def test_listing(ctx):
    rng = np.random.default_rng(11)
    s, d = random_graph(rng, 80, 1200, recip=0.4)
    og = oracle.Graph(80, s, d)
    g = gj.Graph(ctx, s, d, 80)
    for name in ("triangle", "4-cycle", "4-clique"):
        k, atoms = QUERIES[name]
        want, wh = og.list(oracle.Query(k, atoms))
        got, total, h, trunc = gj.list_matches(g, gj.Query(ctx, k, atoms), cap=len(want) + 5)
        assert not trunc and total == len(want) and h == wh
        assert {tuple(t) for t in got.tolist()} == {tuple(t) for t in want.tolist()}
        if len(want) > 3:
            got, total, h, trunc = gj.list_matches(g, gj.Query(ctx, k, atoms), cap=3)
            assert trunc and total == len(want) and len(got) == 3 and h == wh
            assert {tuple(t) for t in got.tolist()} <= {tuple(t) for t in want.tolist()}


def test_count_many_one_launch(ctx):
    rng = np.random.default_rng(13)
    s, d = random_graph(rng, 1000, 30000)
    og = oracle.Graph(1000, s, d)
    g = gj.Graph(ctx, s, d, 1000)
    names = sorted(QUERIES) * 3
    qs = [gj.Query(ctx, *QUERIES[nm]) for nm in names]
    want = [og.count(oracle.Query(*QUERIES[nm])) for nm in names]
    for eng in ENGINES:
        c, h = gj.count_many(g, qs, engine=eng)
        assert list(zip(c, h)) == want, eng


@pytest.mark.parametrize("donation", [1, 2])
def test_work_donation_stress(ctx, donation):
    """Donating every batch of new prefixes to the queue (1) or never (2)
    gives the same counts as the oracle, including delta-free deep queries."""
    rng = np.random.default_rng(61)
    s, d = random_graph(rng, 3000, 60000, recip=0.3)
    og = oracle.Graph(3000, s, d)
    g = gj.Graph(ctx, s, d, 3000)
    names = ["diamond", "4-clique", "5-clique", "4-cycle"]
    qs = [gj.Query(ctx, *QUERIES[nm]) for nm in names]
    want = [og.count(oracle.Query(*QUERIES[nm]), mode=1) for nm in names]
    gj.set_tuning(ctx, donation=donation)
    try:
        assert list(zip(*gj.count_many(g, qs, engine=gj.ENGINE_FUSED))) == want
        for q, w in zip(qs, want):
            assert gj.count(g, q, engine=gj.ENGINE_FUSED) == w
    finally:
        gj.set_tuning(ctx)


@pytest.fixture(scope="module")
def hub_graph():
    """H hubs with edges h_i -> h_j (i < j) and h_i -> every vertex of a
    common set S, plus a sprinkle of random edges; the oracle's counts."""
    rng = np.random.default_rng(71)
    n, H, S = 12000, 40, 5000
    ids = rng.permutation(n).astype(np.uint32)
    hubs, common = ids[:H], ids[H:H + S]
    hs, hd = zip(*[(hubs[i], hubs[j]) for i in range(H) for j in range(i + 1, H)])
    s = np.concatenate([np.array(hs, np.uint32), np.repeat(hubs, S)])
    d = np.concatenate([np.array(hd, np.uint32), np.tile(common, H)])
    core = len(s)
    s = np.concatenate([s, rng.integers(0, n, 20000).astype(np.uint32)])
    d = np.concatenate([d, rng.integers(0, n, 20000).astype(np.uint32)])
    names = ["triangle", "4-clique", "diamond"]
    og = oracle.Graph(n, s, d)
    want = [og.count(oracle.Query(*QUERIES[nm]), mode=1) for nm in names]
    return n, H, S, s, d, core, names, want


@pytest.mark.parametrize("donation", [0, 1, 2])
def test_long_lists_split_ranges(ctx, hub_graph, donation):
    """Every seed prefix has thousands of candidates, so warps split their
    candidate ranges (range donation) inside prefixes that are not the last
    of their batch, and the last level runs its long-list steps. Without
    the random edges the triangle count has the closed form sum over
    i < j of |S| + H-1-j."""
    n, H, S, s, d, core, names, want = hub_graph
    qs = [gj.Query(ctx, *QUERIES[nm]) for nm in names]
    g0 = gj.Graph(ctx, s[:core], d[:core], n)
    assert gj.count(g0, qs[0])[0] == sum(S + H - 1 - j for i in range(H) for j in range(i + 1, H))
    g0.free()
    g = gj.Graph(ctx, s, d, n)
    gj.set_tuning(ctx, donation=donation)
    try:
        assert list(zip(*gj.count_many(g, qs, engine=gj.ENGINE_FUSED))) == want
        for q, w in zip(qs, want):
            assert gj.count(g, q, engine=gj.ENGINE_FUSED) == w
    finally:
        gj.set_tuning(ctx)
        g.free()


@pytest.fixture(scope="module")
def rmat20(ctx):
    s, d = rmat_edges(20, seed=1)
    return s, d, oracle.Graph(1 << 20, s, d), gj.Graph(ctx, s, d, 1 << 20)


@pytest.mark.parametrize("name", ["triangle", "diamond", "4-clique"])
def test_rmat20_sampled_ranges(ctx, rmat20, name):
    """R-MAT scale 20 (16M samples): full-size CUDA runs, checked against the
    oracle on first-attribute ranges it can finish in seconds."""
    s, d, og, g = rmat20
    assert g.m == og.m
    k, atoms = QUERIES[name]
    q = gj.Query(ctx, k, atoms)
    oq = oracle.Query(k, atoms)
    n = 1 << 20
    rng = np.random.default_rng(21)
    for lo in rng.integers(0, n - 512, 3):
        lo = int(lo)
        rg = (lo, lo + 256)
        want = og.count(oq, first_range=rg)
        for eng in ENGINES:
            assert gj.count(g, q, engine=eng, v_range=rg) == want, (name, rg, eng)


@pytest.mark.parametrize("name", ["triangle", "diamond", "4-clique"])
def test_rmat20_full_properties(ctx, rmat20, name):
    """At full size: both engines agree, and the counts of disjoint first-attribute
    ranges add up to the total (counts and checksums)."""
    s, d, og, g = rmat20
    k, atoms = QUERIES[name]
    q = gj.Query(ctx, k, atoms)
    full_f = gj.count(g, q, engine=gj.ENGINE_FUSED)
    full_p = gj.count(g, q, engine=gj.ENGINE_PLAIN)
    assert full_f == full_p
    n = 1 << 20
    tc, th = 0, 0
    for lo in range(0, n, n // 4):
        c, h = gj.count(g, q, engine=gj.ENGINE_FUSED, v_range=(lo, lo + n // 4))
        tc += c
        th = (th + h) & M64
    assert (tc, th) == full_f
