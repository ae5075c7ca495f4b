"""Full-size parity on the static R-MAT scale-20 workload (16,084,904 edges):
the CUDA path's counts, checksums and work units equal the oracle's
full-graph values in tests/golden/rmat20_static.json bit for bit. The
golden was computed by the oracle alone (range-partitioned over first-
attribute chunks, see tests/golden/make_rmat_static.py). Also at full size:
the plain formulations (edge atoms, default orders) give the same counts
and checksums, on both engines, as Theorem 2.1 requires."""
import json
import os

import pytest

from paper_1802_03760_b300 import gj
from paper_1802_03760_b300.inputs import QUERIES, SPECIALISED, rmat_edges

pytestmark = pytest.mark.gpu
GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "rmat20_static.json")))


def gq(ctx, name):
    sp = SPECIALISED.get(name)
    if sp is None:
        return gj.Query(ctx, *QUERIES[name])
    return gj.Query(ctx, sp["k"], sp["atoms"], sp["order"], tri=sp["tri"], lt=sp["lt"])


@pytest.fixture(scope="module")
def graph():
    ctx = gj.Context(0)
    s, d = rmat_edges(GOLD["scale"], seed=GOLD["seed"])
    g = gj.Graph(ctx, s, d, 1 << GOLD["scale"])
    yield ctx, g
    ctx.close()


def want(name):
    q = GOLD["queries"][name]
    return q["count"], int(q["checksum"], 16)


def test_graph_size(graph):
    ctx, g = graph
    assert g.m == GOLD["edges"]
    assert g.build_triangles() == GOLD["queries"]["triangle"]["count"]


def test_formulations_one_launch_equal_golden(graph):
    ctx, g = graph
    names = list(GOLD["queries"])
    got = gj.count_many(g, [gq(ctx, nm) for nm in names], engine=gj.ENGINE_FUSED)
    assert list(zip(*got)) == [want(nm) for nm in names]


@pytest.mark.parametrize("name", ["triangle", "diamond-f", "4-clique-tr"])
def test_work_units_equal_golden(graph, name):
    """Every level's work units, in the cost model's units; a factorised level
    (mode 2) is extended once per prefix of the earlier attributes in the
    oracle, so there only the prefixes reached are compared."""
    ctx, g = graph
    q = GOLD["queries"][name]
    st, k = q["stats"], q["spec"]["k"]
    c, h, w = gj.count(g, gq(ctx, name), engine=gj.ENGINE_FUSED, stats=True)
    assert (c, h) == want(name)
    assert w.seeds == GOLD["edges"]
    last_unfactorised = k - 1 if q["oracle_mode"] == 2 else k
    for j in range(2, last_unfactorised):
        assert w.extended[j] == st["extended"][j], (name, j)
        assert w.nbind[j] == st["nbind_sum"][j], (name, j)
        assert w.proposals[j] == st["proposals"][j], (name, j)
    for j in range(3, k + 1):
        assert w.produced[j] == st["prefixes"][j], (name, j)


@pytest.mark.parametrize("shape,name", [("diamond", "diamond-f"), ("4-clique", "4-clique-tr")])
def test_plain_formulations_equal_golden(graph, shape, name):
    """Theorem 2.1 at full size: the edge-atom formulations in their default
    orders reach the same matches (count and checksum)."""
    ctx, g = graph
    assert gj.count(g, gj.Query(ctx, *QUERIES[shape]), engine=gj.ENGINE_FUSED) == want(name)


@pytest.mark.parametrize("name", ["triangle", "4-clique-tr"])
def test_level_synchronous_engine_equals_golden(graph, name):
    ctx, g = graph
    c, h, w = gj.count(g, gq(ctx, name), engine=gj.ENGINE_PLAIN, stats=True)
    assert (c, h) == want(name)
    st = GOLD["queries"][name]["stats"]
    k = GOLD["queries"][name]["spec"]["k"]
    for j in range(2, k):
        assert (w.extended[j], w.proposals[j]) == (st["extended"][j], st["proposals"][j]), (name, j)
