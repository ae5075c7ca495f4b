"""Parity of the CUDA path with the oracle for the specialisations of Section
5.4 and the aggregation of identical lookups (Section 3.4.2): tri atoms over
the triangle index, inequality filters, degree renaming and orientation at
load, and last-level groups of prefixes that share their extensions.
Counts, checksums and the work counters (in the units of the cost model,
which count every prefix, also those an aggregated group extends at once)
are bit-exact."""
import numpy as np
import pytest

import oracle
from paper_1802_03760_b300 import gj
from paper_1802_03760_b300.inputs import QUERIES, SPECIALISED, er_edges, rmat_edges

pytestmark = pytest.mark.gpu
ENGINES = [gj.ENGINE_PLAIN, gj.ENGINE_FUSED]


@pytest.fixture(scope="module")
def ctx():
    c = gj.Context(0)
    yield c
    c.close()


def gq(ctx, name):
    sp = SPECIALISED[name]
    return gj.Query(ctx, sp["k"], sp["atoms"], sp["order"], tri=sp["tri"], lt=sp["lt"])


def oq(name):
    sp = SPECIALISED[name]
    return oracle.Query(sp["k"], sp["atoms"], sp["order"], tri=sp["tri"], lt=sp["lt"])


def random_graph(rng, n, m, recip=0.3):
    s = rng.integers(0, n, m).astype(np.uint32)
    d = rng.integers(0, n, m).astype(np.uint32)
    r = rng.random(m) < recip
    return np.concatenate([s, d[r]]), np.concatenate([d, s[r]])


def check_work(name, k, w, st1, eng):
    for j in range(2, k):
        assert w.extended[j] == st1.extended[j], (name, eng, j)
        assert w.nbind[j] == st1.nbind_sum[j], (name, eng, j)
        assert w.proposals[j] == st1.proposals[j], (name, eng, j)
    for j in range(3, k + 1):
        assert w.produced[j] == st1.prefixes[j], (name, eng, j)


@pytest.mark.parametrize("seed", range(6))
def test_formulations_random_graphs(ctx, seed):
    rng = np.random.default_rng(800 + seed)
    n = int(rng.integers(30, 300))
    s, d = random_graph(rng, n, int(rng.integers(500, 6000)), recip=float(rng.uniform(0.1, 0.6)))
    og = oracle.Graph(n, s, d)
    g = gj.Graph(ctx, s, d, n)
    assert g.build_triangles() == og.num_triangles()
    for name in sorted(SPECIALISED):
        sp = SPECIALISED[name]
        c1, h1, st1 = og.count(oq(name), stats=True, mode=1)
        q = gq(ctx, name)
        for eng in ENGINES:
            c, h, w = gj.count(g, q, engine=eng, stats=True)
            assert (c, h) == (c1, h1), (name, eng)
            check_work(name, sp["k"], w, st1, eng)


@pytest.fixture(scope="module")
def hub_graph():
    """Hubs joined to one another and to a common set: seeds whose
    aggregated groups hold far more than one batch of prefixes."""
    rng = np.random.default_rng(71)
    n, H, S, B = 9000, 8, 6000, 80
    ids = rng.permutation(n).astype(np.uint32)
    hubs, common = ids[:H], ids[H:H + S]
    hs, hd = zip(*[(hubs[i], hubs[j]) for i in range(H) for j in range(H) if i != j])
    s = np.concatenate([np.array(hs, np.uint32), np.repeat(hubs, S), np.tile(common[:B], H)])
    d = np.concatenate([np.array(hd, np.uint32), np.tile(common, H), np.repeat(hubs, B)])
    s = np.concatenate([s, rng.integers(0, n, 20000).astype(np.uint32)])
    d = np.concatenate([d, rng.integers(0, n, 20000).astype(np.uint32)])
    og = oracle.Graph(n, s, d)
    names = ["diamond-f", "house-f", "house-tr", "4-clique-tr"]
    return n, s, d, names, [og.count(oq(nm), mode=2) for nm in names]


@pytest.mark.parametrize("donation", [0, 1, 2])
def test_aggregated_groups_on_hubs(ctx, hub_graph, donation):
    """diamond-f and house-f: every seed between two hubs has thousands of
    first-trailing extensions, so its group spans many batches, and the second
    trailing list is long enough for ranges to be split and donated."""
    n, s, d, names, want = hub_graph
    g = gj.Graph(ctx, s, d, n)
    qs = [gq(ctx, nm) for nm in names]
    gj.set_tuning(ctx, donation=donation)
    try:
        assert list(zip(*gj.count_many(g, qs, engine=gj.ENGINE_FUSED))) == want
        for q, w in zip(qs, want):
            assert gj.count(g, q, engine=gj.ENGINE_FUSED) == w
        # the same shapes with their default orders and edge atoms
        for nm, w in zip(["diamond", "house", "house", "4-clique"], want):
            assert gj.count(g, gj.Query(ctx, *QUERIES[nm]), engine=gj.ENGINE_FUSED) == w, nm
    finally:
        gj.set_tuning(ctx)
        g.free()


@pytest.mark.parametrize("seed", range(3))
def test_load_flags_degree_renaming(ctx, seed):
    rng = np.random.default_rng(900 + seed)
    n = 400
    s, d = random_graph(rng, n, 5000, recip=0.2)
    og = oracle.Graph(n, s, d)
    for flags, kw in [(gj.LOAD_SYMMETRIZE, dict(symmetrize=True)),
                      (gj.LOAD_SYMMETRIZE | gj.LOAD_DEGREE_ORDER, dict(symmetrize=True, degree_order=True)),
                      (gj.LOAD_SYMMETRIZE | gj.LOAD_DEGREE_ORDER | gj.LOAD_ORIENT,
                       dict(symmetrize=True, degree_order=True, orient=True)),
                      (gj.LOAD_ORIENT, dict(orient=True)), (gj.LOAD_DEGREE_ORDER, dict(degree_order=True))]:
        og2, want_map = og.transform(**kw)
        g = gj.Graph(ctx, s, d, n, flags=flags)
        assert np.array_equal(g.relabel_map(), want_map), flags
        off, nbr = g.export()
        es, ed = og2.edges()
        assert g.m == og2.m and np.array_equal(nbr, ed), flags
        assert np.array_equal(np.repeat(np.arange(n), np.diff(off)), es), flags
        for name in ["4-clique-sym", "house-sym", "5-clique-sym", "4-clique-tr"]:
            want = og2.count(oq(name), mode=1)
            for eng in ENGINES:
                assert gj.count(g, gq(ctx, name), engine=eng) == want, (flags, name, eng)
        for name in ["triangle", "4-clique"]:
            want = og2.count(oracle.Query(*QUERIES[name]), mode=1)
            assert gj.count(g, gj.Query(ctx, *QUERIES[name])) == want, (flags, name)
        g.free()


def test_symmetry_breaking_counts_undirected_cliques_once(ctx):
    """On the oriented degree-renamed graph, the clique query and its tri form
    each count every undirected clique once: 1/k! of the symmetric graph's."""
    s, d = er_edges(300, 6000, seed=5)
    g_sym = gj.Graph(ctx, s, d, 300, flags=gj.LOAD_SYMMETRIZE)
    g_or = gj.Graph(ctx, s, d, 300, flags=gj.LOAD_SYMMETRIZE | gj.LOAD_DEGREE_ORDER | gj.LOAD_ORIENT)
    for k, nm in [(3, "triangle"), (4, "4-clique"), (5, "5-clique")]:
        full = gj.count(g_sym, gj.Query(ctx, *QUERIES[nm]))[0]
        once = gj.count(g_or, gj.Query(ctx, *QUERIES[nm]))[0]
        assert full == once * [1, 1, 2, 6, 24, 120][k]
        if k >= 4:
            assert gj.count(g_or, gq(ctx, nm + "-tr"))[0] == once


def test_tri_queries_refused_in_batches(ctx):
    s, d = er_edges(100, 800, seed=2)
    g = gj.Graph(ctx, s, d, 100)
    with pytest.raises(gj.GJError) as ei:
        gj.apply_batch(g, [1], [2], [1], [gq(ctx, "4-clique-tr")])
    assert ei.value.code == -1
    # the batch was not applied; counting a tri query after a batch rebuilds the index
    m0 = g.m
    gj.apply_batch(g, [1, 3], [2, 4], [1, 1], [gj.Query(ctx, *QUERIES["triangle"])])
    og = oracle.Graph(100, np.concatenate([s, [1, 3]]), np.concatenate([d, [2, 4]]))
    assert g.m == og.m >= m0
    assert gj.count(g, gq(ctx, "4-clique-tr")) == og.count(oq("4-clique-tr"), mode=1)


def test_inequalities_in_delta_queries(ctx):
    """Delta queries keep the inequality filters: the change of a symmetry-broken
    count equals the recount difference."""
    rng = np.random.default_rng(17)
    n = 200
    s, d = random_graph(rng, n, 3000)
    og = oracle.Graph(n, s, d)
    g = gj.Graph(ctx, s, d, n)
    name = "4-clique-sym"
    q = gq(ctx, name)
    bs = rng.integers(0, n, 300).astype(np.uint32)
    bd = rng.integers(0, n, 300).astype(np.uint32)
    bg = rng.choice([-1, 1], 300).astype(np.int8)
    (cs, cd, cg), og2 = oracle.apply_batch(og, bs, bd, bg)
    c0, h0 = og.count(oq(name), mode=1)
    c1, h1 = og2.count(oq(name), mode=1)
    dc, dh = gj.apply_batch(g, bs, bd, bg, [q])
    assert (dc[0], dh[0]) == (c1 - c0, (h1 - h0) % (1 << 64))
    assert gj.count(g, q) == (c1, h1)


def test_device_inputs_written_by_a_pending_kernel(ctx):
    """A device tensor produced by a kernel that may still be running on
    torch's stream is read only after it is complete."""
    import torch
    torch.manual_seed(3)
    n = 3000
    s = torch.randint(0, n, (200000,), device="cuda", dtype=torch.int32)
    d = (s * 7 + torch.randint(1, n, (200000,), device="cuda", dtype=torch.int32)) % n
    g = gj.Graph(ctx, s, d, n)
    og = oracle.Graph(n, s.cpu().numpy().view(np.uint32), d.cpu().numpy().view(np.uint32))
    assert g.m == og.m
    assert gj.count(g, gj.Query(ctx, *QUERIES["triangle"])) == og.count(oracle.Query(*QUERIES["triangle"]))


def test_rmat11_all_formulations(ctx):
    """R-MAT scale 11 (2^15 samples, skewed degrees) in full: the formulations
    against the oracle (house: 2.6e8 matches, the most the oracle hashes in
    seconds)."""
    s, d = rmat_edges(11, seed=4)
    n = 1 << 11
    og = oracle.Graph(n, s, d)
    g = gj.Graph(ctx, s, d, n)
    names = ["diamond-f", "4-clique-tr", "house-f"]
    want = [og.count(oq(nm), mode=2) for nm in names]
    assert list(zip(*gj.count_many(g, [gq(ctx, nm) for nm in names], engine=gj.ENGINE_FUSED))) == want
    assert gj.count(g, gq(ctx, "4-clique-tr"), engine=gj.ENGINE_PLAIN) == want[1]
