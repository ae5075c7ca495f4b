"""The largest queries the C ABI accepts: k = 8 attributes and 16 edge
atoms, against the oracle on both static engines and on both delta engines.
On the transitive tournament T_n (edges i -> j for i < j) a query whose atoms
all point from a lower to a higher attribute and include the path a0 -> a1
-> ... -> a7 matches exactly the increasing 8-tuples: C(n, 8)."""
import math

import numpy as np
import pytest

import oracle
from paper_1802_03760_b300 import gj
from paper_1802_03760_b300.inputs import QUERIES

pytestmark = pytest.mark.gpu

K8_PATH = [(i, i + 1) for i in range(7)]
K8_16 = K8_PATH + [(i, i + 2) for i in range(6)] + [(0, 3), (2, 5), (4, 7)]
MIDDLE_OUT = [3, 4, 2, 5, 1, 6, 0, 7]  # a connected order that does not start at a0


def tournament(n):
    s, d = np.triu_indices(n, 1)
    return s.astype(np.uint32), d.astype(np.uint32)


def test_k8_sixteen_atoms_on_the_transitive_tournament():
    n = 12
    s, d = tournament(n)
    og = oracle.Graph(n, s, d)
    ctx = gj.Context(0)
    g = gj.Graph(ctx, s, d, n)
    tri = og.count(oracle.Query(*QUERIES["triangle"]))
    for atoms in (K8_PATH, K8_16):
        assert len(atoms) <= 16
        for order in (None, MIDDLE_OUT):
            want = og.count(oracle.Query(8, atoms, order))
            assert want[0] == math.comb(n, 8)
            q = gj.Query(ctx, 8, atoms, order)
            for eng in (gj.ENGINE_PLAIN, gj.ENGINE_FUSED):
                assert gj.count(g, q, engine=eng) == want, (len(atoms), order, eng)
            # with a 3-attribute query in the same fused launch
            got = list(zip(*gj.count_many(g, [q, gj.Query(ctx, *QUERIES["triangle"])], engine=gj.ENGINE_FUSED)))
            assert got == [want, tri]
    ctx.close()


def test_k8_path_on_a_random_graph():
    rng = np.random.default_rng(81)
    n = 60
    A = rng.random((n, n)) < 0.08
    np.fill_diagonal(A, False)
    s, d = (x.astype(np.uint32) for x in np.nonzero(A))
    og = oracle.Graph(n, s, d)
    ctx = gj.Context(0)
    g = gj.Graph(ctx, s, d, n)
    for order in (None, MIDDLE_OUT):
        want = og.count(oracle.Query(8, K8_PATH, order))
        assert want[0] > 0
        q = gj.Query(ctx, 8, K8_PATH, order)
        for eng in (gj.ENGINE_PLAIN, gj.ENGINE_FUSED):
            assert gj.count(g, q, engine=eng) == want, (order, eng)
    ctx.close()


@pytest.mark.parametrize("flags", [gj.FLAG_DELTA_PLAIN, gj.FLAG_DELTA_FUSED], ids=["level-sync", "fused"])
def test_k8_sixteen_atoms_delta_queries(flags):
    """Sixteen delta queries dQ_1..dQ_16 per batch (Section 3.3.1): inserts
    and deletes on T_14 change the count by recount-after minus
    recount-before."""
    M64 = (1 << 64) - 1
    n = 14
    s, d = tournament(n)
    og = oracle.Graph(n, s, d)
    ctx = gj.Context(0, flags=flags)
    g = gj.Graph(ctx, s, d, n)
    q = gj.Query(ctx, 8, K8_16)
    oq = oracle.Query(8, K8_16)
    rng = np.random.default_rng(82)
    before = og.count(oq)
    for _ in range(3):
        b = 24
        bs = rng.integers(0, n, b)
        bd = rng.integers(0, n, b)
        bg = rng.choice([-1, 1], b, p=[0.6, 0.4])
        (cs, cd, cg), og2 = oracle.apply_batch(og, bs, bd, bg)
        after = og2.count(oq)
        dc, dh = gj.apply_batch(g, bs.astype(np.uint32), bd.astype(np.uint32), bg.astype(np.int8), [q])
        assert (dc[0], dh[0]) == (after[0] - before[0], (after[1] - before[1]) & M64)
        assert gj.count(g, q) == after
        og, before = og2, after
    ctx.close()
