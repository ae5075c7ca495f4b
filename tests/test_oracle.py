"""Pins for the CPU oracle: each test fixes the oracle against something other
than itself (brute force over V^k, closed forms, matrix identities, the worked
example of Appendix A, SplitMix64 reference outputs, Delta-GJ against
recounting). None of these need a GPU."""
import itertools
import json
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from paper_1802_03760_b300.inputs import QUERIES, er_edges

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
M64 = (1 << 64) - 1


def py_mix64(z):
    z &= M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def py_hash(t):
    """H(t) = q(k) * prod_a f_a(t_a) mod 2^64 (odd factors; see include/gj.h)."""
    h = py_mix64(len(t)) | 1
    for a, x in enumerate(t):
        h = (h * (py_mix64(int(x) ^ (((a + 1) * 0x9E3779B97F4A7C15) & M64)) | 1)) & M64
    return h


def brute_force(n, edges, k, atoms):
    """Join semantics written out: every assignment in V^k checked against every atom."""
    A = np.zeros((n, n), dtype=bool)
    for u, v in edges:
        if u != v:
            A[u, v] = True
    X = np.indices((n,) * k).reshape(k, -1)
    mask = np.ones(X.shape[1], dtype=bool)
    for s, d in atoms:
        mask &= A[X[s], X[d]]
    tuples = X[:, mask].T
    chk = 0
    for t in tuples:
        chk = (chk + py_hash(t)) & M64
    return len(tuples), chk, {tuple(int(x) for x in t) for t in tuples}


def random_edges(rng, n, p, recip=0.3):
    e = []
    for u in range(n):
        for v in range(n):
            if u != v and rng.random() < p:
                e.append((u, v))
                if rng.random() < recip:
                    e.append((v, u))
    e += [(u, u) for u in range(n) if rng.random() < 0.2]  # self-loops are dropped by the loader
    e += e[: len(e) // 4]  # duplicates too
    return e


def og(n, edges):
    s = np.array([a for a, _ in edges], np.uint32)
    d = np.array([b for _, b in edges], np.uint32)
    return oracle.Graph(n, s, d)


def test_splitmix64_reference_outputs():
    gold = json.load(open(os.path.join(GOLDEN, "splitmix64_seed0.json")))
    gamma = int(gold["gamma"], 16)
    for i, want in enumerate(gold["outputs"]):
        state = (gamma * (i + 1)) & M64
        assert oracle.mix64(state) == int(want, 16)
        assert py_mix64(state) == int(want, 16)
    assert oracle.tuple_hash([3, 1, 4]) == py_hash([3, 1, 4])


@pytest.mark.parametrize("name", sorted(QUERIES))
@pytest.mark.parametrize("seed", range(6))
def test_brute_force_named_queries(name, seed):
    rng = np.random.default_rng(1000 + seed)
    n = int(rng.integers(4, 7))
    edges = random_edges(rng, n, float(rng.uniform(0.25, 0.7)))
    k, atoms = QUERIES[name]
    want_c, want_h, want_set = brute_force(n, edges, k, atoms)
    g = og(n, edges)
    q = oracle.Query(k, atoms)
    assert g.count(q) == (want_c, want_h)
    assert g.count(q, mode=1) == (want_c, want_h)
    got, h = g.list(q)
    assert {tuple(int(x) for x in t) for t in got} == want_set
    assert h == want_h


@pytest.mark.parametrize("seed", range(40))
def test_brute_force_random_queries(seed):
    """Random atom sets, directions and attribute orders (including orders whose
    prefixes are not connected, which need the projection extension sets)."""
    rng = np.random.default_rng(seed)
    k = int(rng.integers(2, 5))
    while True:
        na = int(rng.integers(k - 1, 7))
        atoms = []
        for _ in range(na):
            s, d = rng.choice(k, 2, replace=False)
            atoms.append((int(s), int(d)))
        if len({a for p in atoms for a in p}) == k:
            break
    order = [int(x) for x in rng.permutation(k)]
    n = int(rng.integers(3, 7))
    edges = random_edges(rng, n, float(rng.uniform(0.2, 0.8)))
    want_c, want_h, want_set = brute_force(n, edges, k, atoms)
    g = og(n, edges)
    assert g.count(oracle.Query(k, atoms, order)) == (want_c, want_h)
    # a listing is in query attribute order whatever the evaluation order
    got, h = g.list(oracle.Query(k, atoms, order))
    assert {tuple(int(x) for x in t) for t in got} == want_set and len(got) == want_c and h == want_h
    # the implementation's evaluation (edge seeds, bound atoms only) on every connected order
    for o in itertools.permutations(range(k)):
        if connected_order(atoms, o):
            assert g.count(oracle.Query(k, atoms, o), mode=1) == (want_c, want_h), o


def connected_order(atoms, order):
    pos = {a: i for i, a in enumerate(order)}
    if not any({pos[s], pos[d]} == {0, 1} for s, d in atoms):
        return False
    return all(any((pos[s] == j and pos[d] < j) or (pos[d] == j and pos[s] < j) for s, d in atoms)
               for j in range(2, len(order)))


@pytest.mark.parametrize("n", [5, 6, 8, 9])
def test_complete_graph_closed_forms(n):
    dag = [(i, j) for i in range(n) for j in range(i + 1, n)]
    sym = [(i, j) for i in range(n) for j in range(n) if i != j]
    C = math.comb
    P = math.perm
    g = og(n, dag)
    want_dag = {"triangle": C(n, 3), "4-clique": C(n, 4), "5-clique": C(n, 5), "diamond": C(n, 4),
                "4-cycle": C(n, 4), "cyclic-triangle": 0}
    for name, want in want_dag.items():
        assert g.count(oracle.Query(*QUERIES[name]))[0] == want, name
    g = og(n, sym)
    want_sym = {"triangle": P(n, 3), "4-clique": P(n, 4), "5-clique": P(n, 5),
                "diamond": n * (n - 1) * (n - 2) ** 2, "4-cycle": (n - 1) ** 4 + (n - 1),
                "cyclic-triangle": P(n, 3)}
    for name, want in want_sym.items():
        assert g.count(oracle.Query(*QUERIES[name]))[0] == want, name


def matrix_counts(A):
    """Join counts of the shapes as sums of products of adjacency entries
    (exact int64 sparse products, so n = 2000 takes milliseconds)."""
    S = sp.csr_matrix(np.asarray(A, np.int64))
    A2 = S @ S
    AtA = S.T @ S
    AAt = S @ S.T
    return {
        "triangle": int(S.multiply(A2).sum()),                  # sum A12 A23 A13
        "cyclic-triangle": int((A2 @ S).diagonal().sum()),      # closed directed walks of length 3
        "diamond": int(S.multiply(AtA).multiply(AAt).sum()),    # sum_{2,3} A23 (A^T A)_23 (A A^T)_23
        "4-cycle": int(A2.multiply(AtA).sum()),                 # sum_{1,3} (A^2)_13 (A^T A)_13
    }


@pytest.mark.parametrize("seed", range(4))
def test_directed_matrix_identities(seed):
    rng = np.random.default_rng(seed)
    n = 150
    A = (rng.random((n, n)) < 0.08).astype(np.int64)
    np.fill_diagonal(A, 0)
    s, d = np.nonzero(A)
    g = oracle.Graph(n, s, d)
    for name, want in matrix_counts(A).items():
        assert g.count(oracle.Query(*QUERIES[name]))[0] == want, name


def test_er_2000_triangle_matrix_identity():
    """The small triangle workload (directed ER, n=2000, 20000 edges)."""
    s, d = er_edges(2000, 20000, seed=1)
    A = np.zeros((2000, 2000), np.int64)
    A[s, d] = 1
    g = oracle.Graph(2000, s, d)
    assert g.m == 20000
    want = matrix_counts(A)
    for name in ("triangle", "cyclic-triangle", "diamond", "4-cycle"):
        assert g.count(oracle.Query(*QUERIES[name]))[0] == want[name], name


@pytest.mark.parametrize("seed", range(3))
def test_symmetric_traces(seed):
    rng = np.random.default_rng(50 + seed)
    n = 120
    U = np.triu((rng.random((n, n)) < 0.1).astype(np.int64), 1)
    A = U + U.T
    s, d = np.nonzero(A)
    g = oracle.Graph(n, s, d)
    A2 = A @ A
    tri = int(np.trace(A2 @ A))
    assert g.count(oracle.Query(*QUERIES["triangle"]))[0] == tri
    assert tri % 6 == 0  # six ordered copies of each undirected triangle
    assert g.count(oracle.Query(*QUERIES["4-cycle"]))[0] == int(np.trace(A2 @ A2))


def test_appendix_a_worked_example():
    ex = json.load(open(os.path.join(GOLDEN, "appendix_a_cyclic_triangle.json")))
    n = ex["n"]
    g = og(n, [tuple(e) for e in ex["edges"]])
    s, d = g.edges()
    assert sorted(set(s.tolist())) == ex["paper_sources"]
    assert sorted(set(d.tolist())) == ex["paper_destinations"]
    q = oracle.Query(ex["k"], [tuple(a) for a in ex["atoms"]])
    c, h, st = g.count(q, stats=True)
    assert st.prefixes[1] == len(ex["paper_P1"])
    assert st.prefixes[2] == len(ex["paper_P2"])
    assert c == st.prefixes[3] == len(ex["paper_P3"])
    got, _ = g.list(q)
    assert {tuple(t) for t in got.tolist()} == {tuple(t) for t in ex["paper_P3"]}
    # the P2 prefixes are the 2-attribute restriction: R1(a1,a2) with a1 in P1 and a2 a source of R2
    p2 = {(u, v) for u, v in zip(s.tolist(), d.tolist()) if u in {1, 6, 7} and v in ex["paper_sources"]}
    assert p2 == {tuple(t) for t in ex["paper_P2"]}


@pytest.mark.parametrize("name", ["triangle", "4-cycle", "diamond", "4-clique"])
def test_order_invariance(name):
    """Theorem 2.1 holds for any attribute order; the result does not depend on it."""
    rng = np.random.default_rng(7)
    n = 40
    A = rng.random((n, n)) < 0.25
    np.fill_diagonal(A, False)
    s, d = np.nonzero(A)
    g = oracle.Graph(n, s, d)
    k, atoms = QUERIES[name]
    ref = g.count(oracle.Query(k, atoms))
    for order in itertools.permutations(range(k)):
        assert g.count(oracle.Query(k, atoms, order)) == ref, order


@pytest.mark.parametrize("mode", [0, 1])
def test_first_attribute_ranges_add_up(mode):
    s, d = er_edges(300, 4000, seed=3)
    g = oracle.Graph(300, s, d)
    q = oracle.Query(*QUERIES["diamond"])
    c, h = g.count(q)
    tc, th = 0, 0
    for lo in range(0, 300, 37):
        a, b = g.count(q, first_range=(lo, min(lo + 37, 300)), mode=mode)
        tc += a
        th = (th + b) & M64
    assert (tc, th) == (c, h)


def test_implementation_mode_seeds_are_edges():
    """Section 4.2: the length-2 prefixes are the edges of the seed atom (filtered by
    other atoms over the same pair), not the projection-restricted P2 of Fig. 1."""
    ex_edges = [(0, 1), (1, 2), (2, 0), (3, 0)]  # 0->1 where 1 has out-degree, 3->0 ...
    g = og(4, ex_edges)
    q = oracle.Query(*QUERIES["cyclic-triangle"])
    _, _, st0 = g.count(q, stats=True, mode=0)
    _, _, st1 = g.count(q, stats=True, mode=1)
    assert st1.prefixes[2] == 4          # every edge seeds
    assert st0.prefixes[2] == 3          # (3,0) drops: 3 is not a destination, so not in P1


def test_triangle_work_counters():
    """The instrumented units follow from degrees: for the transitive triangle in
    order a1,a2,a3, every edge is a P2 prefix and proposes min(out(a1), out(a2))."""
    s, d = er_edges(500, 6000, seed=4)
    g = oracle.Graph(500, s, d)
    c, h, st = g.count(oracle.Query(*QUERIES["triangle"]), stats=True, mode=1)
    dout = np.bincount(s, minlength=500)
    assert st.extended[2] == 6000
    assert st.nbind_sum[2] == 2 * 6000
    assert st.proposals[2] == int(np.minimum(dout[s], dout[d]).sum())
    assert st.probes[2] == st.proposals[2]
    assert st.prefixes[3] == c


def test_normalize_semantics():
    g = og(6, [(0, 1), (1, 2), (2, 3)])
    src = [0, 4, 4, 1, 2, 5, 0, 3, 3]
    dst = [1, 5, 5, 2, 3, 5, 2, 4, 4]
    sgn = [+1, +1, -1, -1, -1, +1, +1, -1, +1]
    # (0,1) insert of present: no-op; (4,5) insert then delete: absent at end, was absent: no-op;
    # (1,2) delete of present: -1; (2,3) delete: -1; (5,5) self-loop dropped; (0,2) insert: +1;
    # (3,4) delete then insert: present at end, was absent: +1
    s, d, c = g.normalize(src, dst, sgn)
    assert list(zip(s.tolist(), d.tolist(), c.tolist())) == [(0, 2, 1), (1, 2, -1), (2, 3, -1), (3, 4, 1)]
    g2 = g.apply(s, d, c)
    s2, d2 = g2.edges()
    assert list(zip(s2.tolist(), d2.tolist())) == [(0, 1), (0, 2), (3, 4)]
    with pytest.raises(oracle.OracleError):
        g.normalize([0], [9], [1])
    with pytest.raises(oracle.OracleError):
        g.normalize([0], [1], [2])


@pytest.mark.parametrize("name", sorted(QUERIES))
@pytest.mark.parametrize("seed", range(5))
def test_delta_queries_equal_recount(name, seed):
    """Section 3.3.1: Q' - Q equals the signed sum of dQ_1..dQ_n."""
    rng = np.random.default_rng(500 + seed)
    n = 25
    A = rng.random((n, n)) < 0.3
    np.fill_diagonal(A, False)
    s, d = np.nonzero(A)
    g = oracle.Graph(n, s, d)
    k, atoms = QUERIES[name]
    q = oracle.Query(k, atoms)
    for _ in range(3):
        b = int(rng.integers(1, 60))
        bs = rng.integers(0, n, b)
        bd = rng.integers(0, n, b)
        bg = rng.choice([-1, 1], b)
        ex_s, ex_d = g.edges()  # include deletes of existing edges
        pick = rng.integers(0, len(ex_s), 10)
        bs = np.concatenate([bs, ex_s[pick]])
        bd = np.concatenate([bd, ex_d[pick]])
        bg = np.concatenate([bg, -np.ones(10, np.int64)])
        (cs, cd, cg), g2 = oracle.apply_batch(g, bs, bd, bg)
        c0, h0 = g.count(q)
        c1, h1 = g2.count(q)
        assert oracle.delta(g, g2, cs, cd, cg, q) == (c1 - c0, (h1 - h0) & M64)
        g = g2


# shapes with two atoms over the same attribute pair: a seed filter atom of
# dQ_i reads the new version when it comes before atom i, the old after
RECIPROCAL = {"2-cycle-tail": (3, [(0, 1), (1, 0), (1, 2)]),
              "reciprocal-triangle": (3, [(0, 1), (1, 2), (1, 0), (2, 0)])}


@pytest.mark.parametrize("name", sorted(QUERIES) + sorted(RECIPROCAL))
@pytest.mark.parametrize("seed", range(4))
def test_each_delta_query_brute_force(name, seed):
    """Section 3.3.1, each part on its own: dQ_i joins the new versions of
    the atoms before i, the signed changes of atom i and the old versions of
    the atoms after i. Written out over V^k with A_old, A_new and Delta =
    A_new - A_old (the batch applied update by update, the last update of an
    edge deciding). The other telescoping order (old before i, new after)
    has the same sum, so only the parts tell the two apart."""
    rng = np.random.default_rng(700 + seed)
    k, atoms = QUERIES[name] if name in QUERIES else RECIPROCAL[name]
    n = 6 if k <= 4 else 5
    A_old = rng.random((n, n)) < 0.45
    np.fill_diagonal(A_old, False)
    s, d = np.nonzero(A_old)
    g = oracle.Graph(n, s, d)
    b = 30
    bs, bd, bg = rng.integers(0, n, b), rng.integers(0, n, b), rng.choice([-1, 1], b)
    A_new = A_old.copy()
    for u, v, sg in zip(bs, bd, bg):
        if u != v:
            A_new[u, v] = sg > 0
    Dl = A_new.astype(np.int64) - A_old.astype(np.int64)
    (cs, cd, cg), g2 = oracle.apply_batch(g, bs, bd, bg)
    assert sorted(zip(cs.tolist(), cd.tolist(), cg.tolist())) == \
        sorted((int(u), int(v), int(Dl[u, v])) for u, v in zip(*np.nonzero(Dl)))
    X = np.indices((n,) * k).reshape(k, -1)
    want = []
    for i in range(len(atoms)):
        w = np.ones(X.shape[1], np.int64)
        for t, (sa, da) in enumerate(atoms):
            M = A_new if t < i else (A_old if t > i else Dl)
            w *= M[X[sa], X[da]]
        chk = 0
        for c in np.nonzero(w)[0]:
            chk = (chk + int(w[c]) * py_hash(X[:, c])) & M64
        want.append((int(w.sum()), chk))
    q = oracle.Query(k, atoms)
    assert oracle.delta_each(g, g2, cs, cd, cg, q) == want
    assert oracle.delta(g, g2, cs, cd, cg, q) == (sum(c for c, _ in want), sum(h for _, h in want) & M64)


def test_delta_order_does_not_matter():
    rng = np.random.default_rng(9)
    n = 30
    A = rng.random((n, n)) < 0.25
    np.fill_diagonal(A, False)
    s, d = np.nonzero(A)
    g = oracle.Graph(n, s, d)
    (cs, cd, cg), g2 = oracle.apply_batch(g, rng.integers(0, n, 40), rng.integers(0, n, 40), rng.choice([-1, 1], 40))
    k, atoms = QUERIES["4-clique"]
    ref = oracle.delta(g, g2, cs, cd, cg, oracle.Query(k, atoms))
    for order in [(3, 2, 1, 0), (1, 3, 0, 2)]:
        assert oracle.delta(g, g2, cs, cd, cg, oracle.Query(k, atoms, order)) == ref


def test_rejects_invalid():
    g = og(4, [(0, 1)])
    for k, atoms, order in [(3, [(0, 0), (1, 2)], None), (3, [(0, 1)], None), (3, [(0, 1), (1, 2)], [0, 0, 1]),
                            (9, [(0, 1)], None), (3, [(0, 3), (1, 2)], None)]:
        with pytest.raises(oracle.OracleError):
            g.count(oracle.Query(k, atoms, order))
    with pytest.raises(oracle.OracleError):
        oracle.Graph(4, np.array([0], np.uint32), np.array([4], np.uint32))


def test_edge_seeded_mode_needs_each_attribute_bound_by_earlier_ones():
    """The path a0 -> a1 -> a2 -> a3 in the order a0, a1, a3, a2: the seed
    pair (a0, a1) is an atom, but when a3 comes no atom joins it to a bound
    attribute. The definition (mode 0) extends by the projection and still
    counts every path; the edge-seeded evaluation (Section 4.1) has no
    relation to propose a3 from and refuses the order."""
    rng = np.random.default_rng(11)
    n = 6
    edges = random_edges(rng, n, 0.5)
    k, atoms, order = 4, [(0, 1), (1, 2), (2, 3)], [0, 1, 3, 2]
    want_c, want_h, _ = brute_force(n, edges, k, atoms)
    g = og(n, edges)
    assert g.count(oracle.Query(k, atoms, order), mode=0) == (want_c, want_h)
    with pytest.raises(oracle.OracleError):
        g.count(oracle.Query(k, atoms, order), mode=1)
    assert g.count(oracle.Query(k, atoms, [0, 1, 2, 3]), mode=1) == (want_c, want_h)


def test_empty_graph():
    g = oracle.Graph(5, np.array([], np.uint32), np.array([], np.uint32))
    assert g.m == 0
    for name, (k, atoms) in QUERIES.items():
        assert g.count(oracle.Query(k, atoms)) == (0, 0)


@pytest.mark.parametrize("seed", range(5))
def test_apply_is_set_update(seed):
    """R' = R + Delta R: inserted edges present, deleted edges absent, the rest unchanged."""
    rng = np.random.default_rng(900 + seed)
    n = 20
    A = rng.random((n, n)) < 0.3
    np.fill_diagonal(A, False)
    s, d = np.nonzero(A)
    g = oracle.Graph(n, s, d)
    for _ in range(4):
        ex_s, ex_d = g.edges()
        pick = rng.integers(0, len(ex_s), 15)
        bs = np.concatenate([rng.integers(0, n, 30), ex_s[pick]])
        bd = np.concatenate([rng.integers(0, n, 30), ex_d[pick]])
        bg = np.concatenate([rng.choice([-1, 1], 30), -np.ones(15, np.int64)])
        (cs, cd, cg), g2 = oracle.apply_batch(g, bs, bd, bg)
        E0 = set(zip(ex_s.tolist(), ex_d.tolist()))
        final = dict()
        for u, v, c in zip(bs.tolist(), bd.tolist(), bg.tolist()):
            if u != v:
                final[(u, v)] = c
        want = (E0 | {e for e, c in final.items() if c > 0}) - {e for e, c in final.items() if c < 0}
        assert set(zip(*[x.tolist() for x in g2.edges()])) == want
        g = g2
