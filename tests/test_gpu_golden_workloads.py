"""Parity at the full sizes of the batched multi-query and the dynamic
workloads, against values only the CPU oracle computed (committed goldens,
each written by its script beside it in tests/golden/):

- rmat24_multi64.json: the 64 mixed queries (five shapes, seeded direction
  and order variants) on R-MAT scale 24, matches whose first attribute lies
  in [0, 64) -- the sample the multi-query benchmark times. All 64 run in
  one fused launch and, separately, on the level-synchronous engine; counts,
  checksums and the cost model's work units must equal the oracle's.
- rmat22_delta1k.json: the first 20 batches of 1,000 updates of the R-MAT
  scale-22 update stream; each batch's change of the triangle and 4-clique
  counts and checksums (Delta-GJ, Section 3.3.1) and the edge count after
  it must equal the oracle's, on both delta engines."""
import json
import os

import pytest

from paper_1802_03760_b300 import gj
from paper_1802_03760_b300.inputs import QUERIES, UpdateStream, rmat_edges

pytestmark = pytest.mark.gpu
HERE = os.path.join(os.path.dirname(__file__), "golden")
MULTI = json.load(open(os.path.join(HERE, "rmat24_multi64.json")))
DELTA = json.load(open(os.path.join(HERE, "rmat22_delta1k.json")))


@pytest.fixture(scope="module")
def multi():
    ctx = gj.Context(0)
    s, d = rmat_edges(MULTI["scale"], seed=MULTI["seed"])
    g = gj.Graph(ctx, s, d, 1 << MULTI["scale"])
    del s, d
    qs = [gj.Query(ctx, q["k"], [tuple(a) for a in q["atoms"]], q["order"]) for q in MULTI["queries"]]
    yield ctx, g, qs
    ctx.close()


def _want():
    return [(q["count"], int(q["checksum"], 16)) for q in MULTI["queries"]]


@pytest.mark.parametrize("engine", [gj.ENGINE_FUSED, gj.ENGINE_PLAIN])
def test_multi_query_sample_equals_golden(multi, engine):
    ctx, g, qs = multi
    got = gj.count_many(g, qs, engine=engine, v_range=(0, MULTI["first"]))
    assert list(zip(*got)) == _want()


@pytest.mark.parametrize("i", [0, 1, 2, 3, 4, 13, 41])
def test_multi_query_work_units_equal_golden(multi, i):
    ctx, g, qs = multi
    q = MULTI["queries"][i]
    st, k = q["stats"], q["k"]
    c, h, w = gj.count(g, qs[i], engine=gj.ENGINE_FUSED, v_range=(0, MULTI["first"]), stats=True)
    assert (c, h) == (q["count"], int(q["checksum"], 16))
    for j in range(2, k):
        assert (w.extended[j], w.nbind[j], w.proposals[j]) == \
            (st["extended"][j], st["nbind_sum"][j], st["proposals"][j]), (q["name"], j)
    for j in range(3, k + 1):
        assert w.produced[j] == st["prefixes"][j], (q["name"], j)


@pytest.mark.parametrize("flags", [gj.FLAG_DELTA_PLAIN, gj.FLAG_DELTA_FUSED], ids=["plain", "fused"])
def test_update_stream_deltas_equal_golden(flags):
    ctx = gj.Context(0, flags=flags)  # the delta engine
    n = 1 << DELTA["scale"]
    s, d = rmat_edges(DELTA["scale"], seed=DELTA["seed"])
    stream = UpdateStream(s, d, DELTA["scale"], seed=DELTA["seed"])
    g = gj.Graph(ctx, s, d, n)
    del s, d
    qs = [gj.Query(ctx, *QUERIES[nm]) for nm in DELTA["queries"]]
    for b in DELTA["batches"]:
        bs, bd, bg = stream.next_batch(DELTA["size"])
        c, h = gj.apply_batch(g, bs, bd, bg, qs)
        want = [(b["delta"][nm]["count"], int(b["delta"][nm]["checksum"], 16)) for nm in DELTA["queries"]]
        assert list(zip(c, h)) == want, b["batch"]
        assert gj.last_batch_changes(g) == b["changes"], b["batch"]
        assert g.m == b["edges_after"], b["batch"]
    ctx.close()
