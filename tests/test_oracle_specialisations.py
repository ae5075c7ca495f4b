"""Pins for the oracle's specialisations of Section 5.4: inequality
constraints (symmetry breaking), renaming by degree, the ternary triangle
relation tri(a_i, a_j, a_l) indexed by (a_i, a_j), and factorised output
for trailing attributes that constrain one another in no way.

Each is fixed against something other than the oracle: brute force over
V^k (with tri and the inequalities written out), undirected cliques
counted by combinations, closed forms on complete graphs, the matrix
identity for the size of tri, the automorphism counts of the shapes, and
the work units of factorised extension recomputed from degrees."""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_1802_03760_b300.inputs import QUERIES, SPECIALISED

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


def adjacency(n, edges):
    A = np.zeros((n, n), dtype=bool)
    for u, v in edges:
        if u != v:
            A[u, v] = True
    return A


def brute(A, k, atoms=(), tri=(), lt=()):
    """Join semantics written out over V^k: edge atoms, tri atoms as their three
    edges, inequalities as comparisons of vertex ids."""
    n = A.shape[0]
    X = np.indices((n,) * k).reshape(k, -1)
    mask = np.ones(X.shape[1], dtype=bool)
    for s, d in atoms:
        mask &= A[X[s], X[d]]
    for a, b, c in tri:
        mask &= A[X[a], X[b]] & A[X[a], X[c]] & A[X[b], X[c]]
    for a, b in lt:
        mask &= X[a] < X[b]
    tuples = X[:, mask].T
    chk = 0
    for t in tuples:
        chk = (chk + py_hash(t)) & M64
    return len(tuples), chk


def graph(A):
    s, d = np.nonzero(A)
    return oracle.Graph(A.shape[0], s.astype(np.uint32), d.astype(np.uint32))


def q_of(name):
    sp = SPECIALISED[name]
    return oracle.Query(sp["k"], sp["atoms"], sp["order"], tri=sp["tri"], lt=sp["lt"])


def valid_mode1(k, atoms, tri, order):
    """Orders the edge-seeded evaluation accepts: the first two attributes are
    joined by an edge atom or are the indexed pair of a tri atom, every tri atom
    binds its third attribute after its first two, and every later attribute has
    a binding atom."""
    pos = {a: i for i, a in enumerate(order)}
    if not (any({pos[s], pos[d]} == {0, 1} for s, d in atoms) or any({pos[a], pos[b]} == {0, 1} for a, b, _ in tri)):
        return False
    if any(pos[c] < pos[a] or pos[c] < pos[b] for a, b, c in tri):
        return False
    for j in range(2, k):
        if not (any((pos[s] == j and pos[d] < j) or (pos[d] == j and pos[s] < j) for s, d in atoms)
                or any(pos[c] == j for _, _, c in tri)):
            return False
    return True


@pytest.mark.parametrize("seed", range(4))
def test_tri_relation_size_is_the_transitive_triangle_count(seed):
    """|tri| = sum of A o A^2: a -> b -> c with a -> c."""
    rng = np.random.default_rng(70 + seed)
    n = 90
    A = rng.random((n, n)) < 0.12
    np.fill_diagonal(A, False)
    Ai = A.astype(np.int64)
    assert graph(A).num_triangles() == int((Ai * (Ai @ Ai)).sum())


@pytest.mark.parametrize("seed", range(40))
def test_brute_force_tri_and_inequality_queries(seed):
    """Random queries mixing edge atoms, tri atoms and inequalities, on every
    order the edge-seeded evaluation accepts, with and without factorisation."""
    rng = np.random.default_rng(3000 + seed)
    while True:
        k = int(rng.integers(3, 6))
        atoms = [tuple(int(x) for x in rng.choice(k, 2, replace=False)) for _ in range(int(rng.integers(0, 4)))]
        tri = [tuple(int(x) for x in rng.choice(k, 3, replace=False)) for _ in range(int(rng.integers(0, 3)))]
        lt = [tuple(int(x) for x in rng.choice(k, 2, replace=False)) for _ in range(int(rng.integers(0, 3)))]
        used = {a for p in atoms for a in p} | {a for t in tri for a in t}
        orders = [o for o in itertools.permutations(range(k)) if valid_mode1(k, atoms, tri, o)]
        if len(used) == k and (atoms or tri) and orders:
            break
    n = int(rng.integers(4, 7)) if k < 5 else int(rng.integers(4, 6))
    A = rng.random((n, n)) < float(rng.uniform(0.3, 0.8))
    np.fill_diagonal(A, False)
    want = brute(A, k, atoms, tri, lt)
    g = graph(A)
    for o in orders[:6]:
        q = oracle.Query(k, atoms, o, tri=tri, lt=lt)
        assert g.count(q, mode=1) == want, (atoms, tri, lt, o)
        assert g.count(q, mode=2) == want, (atoms, tri, lt, o)
        if not tri:
            assert g.count(q, mode=0) == want, (atoms, lt, o)


@pytest.mark.parametrize("n", [4, 6, 9])
def test_inequality_between_unjoined_attributes_closed_form(n):
    """Two attributes that no atom joins may take the same vertex, so only a
    strict inequality between them keeps such tuples out. On the complete
    directed graph K_n, a -> b <- c with a < c has n * C(n-1, 2) matches
    (b, then two distinct others in ascending order), whichever of a and c
    is bound first."""
    g = graph(~np.eye(n, dtype=bool))
    atoms = [(0, 1), (2, 1)]
    want = n * math.comb(n - 1, 2)
    for lt in ([(0, 2)], [(2, 0)]):
        for o in itertools.permutations(range(3)):
            q = oracle.Query(3, atoms, o, lt=lt)
            assert g.count(q, mode=0)[0] == want, (lt, o)
            if valid_mode1(3, atoms, [], o):
                assert g.count(q, mode=1)[0] == want, (lt, o)


@pytest.mark.parametrize("name", sorted(SPECIALISED))
@pytest.mark.parametrize("seed", range(3))
def test_specialised_formulations_equal_their_shape(name, seed):
    """Each formulation has the matches of the shape it is named after: on any
    directed graph for tri and factorised forms, brute force with the
    inequalities for the symmetry-broken forms."""
    rng = np.random.default_rng(4000 + seed)
    n = 7
    A = rng.random((n, n)) < 0.55
    np.fill_diagonal(A, False)
    sp = SPECIALISED[name]
    shape = name.split("-")[0] if not name.startswith(("4-", "5-")) else "-".join(name.split("-")[:2])
    k, atoms = QUERIES[shape]
    want = brute(A, k, atoms, (), sp["lt"])
    q = q_of(name)
    assert graph(A).count(q, mode=1) == want
    assert graph(A).count(q, mode=2) == want


@pytest.mark.parametrize("n", [5, 6, 9])
def test_complete_graph_closed_forms(n):
    C, P = math.comb, math.perm
    dag = np.triu(np.ones((n, n), bool), 1)
    sym = ~np.eye(n, dtype=bool)
    for A, k4, k5 in [(dag, C(n, 4), C(n, 5)), (sym, P(n, 4), P(n, 5))]:
        g = graph(A)
        assert g.count(q_of("4-clique-tr"), mode=1)[0] == k4
        assert g.count(q_of("5-clique-tr"), mode=1)[0] == k5
    # symmetry breaking: one match per undirected clique of the complete graph
    g = graph(sym)
    assert g.count(q_of("4-clique-sym"), mode=1)[0] == C(n, 4)
    assert g.count(q_of("5-clique-sym"), mode=1)[0] == C(n, 5)
    # house on the complete symmetric graph: n choices per position, all distinct? no: join
    # semantics only forbids equal endpoints of an edge; a1 may equal a4 or a5
    house = QUERIES["house"]
    full = g.count(oracle.Query(*house), mode=1)[0]
    assert full == P(n, 4) * (n - 2)  # the 4-clique a2..a5 is injective, a1 avoids a2 and a3
    assert g.count(q_of("house-f"), mode=2)[0] == full


def undirected_cliques(A, k):
    U = A | A.T
    return sum(1 for c in itertools.combinations(range(A.shape[0]), k) if all(U[a, b] for a, b in itertools.combinations(c, 2)))


@pytest.mark.parametrize("seed", range(4))
def test_symmetry_breaking_counts_each_undirected_subgraph_once(seed):
    """On the symmetrised graph renamed by degree: a clique query with a1 < ... < ak
    (or the plain clique query on the graph oriented from lower to higher id) has
    one match per undirected clique, and k! times as many without; the house
    query has |Aut(house)| = 4 times as many matches without its inequalities."""
    rng = np.random.default_rng(5000 + seed)
    n = 9
    A = rng.random((n, n)) < 0.4
    np.fill_diagonal(A, False)
    g0 = graph(A)
    gs, _ = g0.transform(symmetrize=True, degree_order=True)
    go, _ = g0.transform(symmetrize=True, degree_order=True, orient=True)
    for k, name in [(4, "4-clique"), (5, "5-clique")]:
        und = undirected_cliques(A, k)
        assert gs.count(q_of(name + "-sym"), mode=1)[0] == und
        assert go.count(oracle.Query(*QUERIES[name]), mode=1)[0] == und
        assert go.count(q_of(name + "-tr"), mode=1)[0] == und
        assert gs.count(oracle.Query(*QUERIES[name]), mode=1)[0] == und * math.factorial(k)
    sym_house = gs.count(q_of("house-sym"), mode=2)[0]
    assert 4 * sym_house == gs.count(oracle.Query(*QUERIES["house"]), mode=1)[0]


@pytest.mark.parametrize("seed", range(5))
def test_degree_renaming(seed):
    """New ids ascend with the degree in the symmetrised graph (ties by old id);
    orientation keeps the edges from a lower to a higher new id."""
    rng = np.random.default_rng(6000 + seed)
    n = 40
    A = rng.random((n, n)) < 0.1
    np.fill_diagonal(A, False)
    g0 = graph(A)
    U = A | A.T
    deg = U.sum(1)
    rank = sorted(range(n), key=lambda v: (deg[v], v))
    want_map = np.empty(n, np.int64)
    want_map[rank] = np.arange(n)
    gs, m = g0.transform(symmetrize=True, degree_order=True)
    assert np.array_equal(m, want_map)
    us, vs = np.nonzero(U)
    assert set(zip(*[x.tolist() for x in gs.edges()])) == {(int(want_map[u]), int(want_map[v])) for u, v in zip(us, vs)}
    go, m2 = g0.transform(symmetrize=True, degree_order=True, orient=True)
    assert np.array_equal(m2, want_map)
    assert set(zip(*[x.tolist() for x in go.edges()])) == {
        (int(want_map[u]), int(want_map[v])) for u, v in zip(us, vs) if want_map[u] < want_map[v]}
    gi, mi = g0.transform()
    assert np.array_equal(mi, np.arange(n)) and gi.m == g0.m
    # without symmetrisation the renaming ascends with the out-degree of the directed graph
    dout = A.sum(1)
    rank_d = sorted(range(n), key=lambda v: (dout[v], v))
    want_d = np.empty(n, np.int64)
    want_d[rank_d] = np.arange(n)
    gd, md = g0.transform(degree_order=True)
    assert np.array_equal(md, want_d)
    s0, d0 = np.nonzero(A)
    assert set(zip(*[x.tolist() for x in gd.edges()])) == {(int(want_d[u]), int(want_d[v])) for u, v in zip(s0, d0)}


@pytest.mark.parametrize("name", ["diamond-f", "house-f", "house-tr"])
@pytest.mark.parametrize("seed", range(3))
def test_factorised_work_units(name, seed):
    """Factorised extension counts each trailing attribute's extension once per
    prefix of the non-trailing attributes: extended[j] is the number of such
    prefixes (found by brute force), proposals[j] the sum of their smallest
    extension-set sizes (recomputed from degrees and triangle lists); the
    prefix counts are those of unfactorised evaluation."""
    rng = np.random.default_rng(7000 + seed)
    n = 12
    A = rng.random((n, n)) < 0.45
    np.fill_diagonal(A, False)
    sp = SPECIALISED[name]
    k, order, atoms, tri = sp["k"], sp["order"], sp["atoms"], sp["tri"]
    g = graph(A)
    q = q_of(name)
    c1, h1, st1 = g.count(q, stats=True, mode=1)
    c2, h2, st2 = g.count(q, stats=True, mode=2)
    assert (c1, h1) == (c2, h2)
    assert list(st2.prefixes) == list(st1.prefixes)
    f = k - 2
    head = order[:f]
    pos = {a: i for i, a in enumerate(order)}
    # parents: assignments of the first f attributes meeting every constraint among them
    parents = []
    for vals in itertools.product(range(n), repeat=f):
        x = dict(zip(head, vals))
        ok = all(A[x[s], x[d]] for s, d in atoms if s in x and d in x)
        ok = ok and all(A[x[a], x[b]] and A[x[a], x[c]] and A[x[b], x[c]] for a, b, c in tri
                        if a in x and b in x and c in x)
        if ok:
            parents.append(x)
    assert st2.prefixes[f] == len(parents)
    for j in (f, f + 1):
        a_new = order[j]
        sizes = []
        for x in parents:
            s = [int(A[x[u]].sum()) if d == a_new else int(A[:, x[d]].sum())
                 for u, d in atoms if (d == a_new and u in x) or (u == a_new and d in x)]
            s += [int((A[x[a]] & A[x[b]]).sum()) if A[x[a], x[b]] else 0 for a, b, c in tri if c == a_new]
            sizes.append(s)
        assert st2.extended[j] == len(parents)
        assert st2.nbind_sum[j] == sum(len(s) for s in sizes)
        assert st2.proposals[j] == sum(min(s) for s in sizes)


@pytest.mark.parametrize("seed", range(3))
def test_factorised_star_work_units(seed):
    """The star E(a0, a1), E(a0, a2), E(a0, a3) in the order a0..a3: a1 is
    joined only to the seed attribute a0, a2 and a3 to no later attribute, so
    exactly a2 and a3 factorise (the seed pair never does). Each seed edge
    u -> v is then extended once at both factorised levels, with the single
    set out(u): extended = |E| and proposals = sum over edges of outdeg(u),
    while the count is the sum over vertices of outdeg^3."""
    rng = np.random.default_rng(7100 + seed)
    n = 14
    A = rng.random((n, n)) < 0.35
    np.fill_diagonal(A, False)
    g = graph(A)
    q = oracle.Query(4, [(0, 1), (0, 2), (0, 3)], [0, 1, 2, 3])
    out = A.sum(axis=1).astype(np.int64)
    c2, _, st2 = g.count(q, stats=True, mode=2)
    assert c2 == int((out ** 3).sum())
    m = int(A.sum())
    for j in (2, 3):
        assert st2.extended[j] == m
        assert st2.nbind_sum[j] == m
        assert st2.proposals[j] == int((out * out).sum())


def test_rejects_invalid_specialisations():
    g = graph(np.triu(np.ones((5, 5), bool), 1))
    bad = [
        dict(k=3, atoms=[], tri=[(0, 1, 1)], lt=[], order=None),          # repeated attribute
        dict(k=3, atoms=[], tri=[(0, 1, 2)], lt=[(1, 1)], order=None),    # x < x
        dict(k=3, atoms=[], tri=[(0, 1, 2)], lt=[], order=[2, 0, 1]),     # third attribute first
        # edge seed (0, 2) and attribute 1 bound by E(0, 1), but tri(0, 1, 2)'s
        # third attribute comes before its second
        dict(k=3, atoms=[(0, 2), (0, 1)], tri=[(0, 1, 2)], lt=[], order=[0, 2, 1]),
        dict(k=3, atoms=[], tri=[(0, 1, 3)], lt=[], order=None),          # out of range
    ]
    for sp in bad:
        with pytest.raises(oracle.OracleError):
            g.count(oracle.Query(sp["k"], sp["atoms"], sp["order"], tri=sp["tri"], lt=sp["lt"]), mode=1)
    with pytest.raises(oracle.OracleError):  # the definition (mode 0) has no tri relation
        g.count(q_of("4-clique-tr"), mode=0)
