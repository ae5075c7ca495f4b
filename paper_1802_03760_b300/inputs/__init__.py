"""Seeded synthetic inputs shared by the CPU oracle and the CUDA path.

The paper evaluates on LiveJournal, Twitter, UK-2007 and Common Crawl
(Section 5, Table 1); none of them is available here, so seeded power-law
R-MAT graphs and a directed Erdos-Renyi graph stand in for them. This module
only makes inputs (edge samples, permutations, update batches). It contains
no part of the join method, and it imports neither the oracle nor the CUDA
library. The C kernels live in ``gen.c`` beside this file and are compiled
with gcc on first use.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB_PATH = os.path.join(_HERE, "libgjinputs.so")
_lib = None
_lock = threading.Lock()

RMAT_ABC = (0.57, 0.19, 0.19)  # d = 0.05


def build(force: bool = False) -> str:
    """Compile gen.c into libgjinputs.so (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u32p = ctypes.POINTER(ctypes.c_uint32)
            u64p = ctypes.POINTER(ctypes.c_uint64)
            lib.gjin_rand.restype = ctypes.c_uint64
            lib.gjin_rand.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            lib.gjin_er.restype = ctypes.c_int64
            lib.gjin_er.argtypes = [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64, u32p, u32p]
            lib.gjin_permutation.restype = None
            lib.gjin_permutation.argtypes = [ctypes.c_uint32, ctypes.c_uint64, u32p]
            lib.gjin_rmat.restype = None
            lib.gjin_rmat.argtypes = [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                      ctypes.c_double, ctypes.c_double, ctypes.c_double, u32p, u32p, u32p]
            lib.gjin_hubs.restype = ctypes.c_int
            lib.gjin_hubs.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64,
                                      u32p, u32p, u32p]
            lib.gjin_uniform.restype = None
            lib.gjin_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, u64p]
            _lib = lib
    return _lib


def _p32(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


def _p64(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def subseed(seed: int, tag: int) -> int:
    """An independent stream seed derived from (seed, tag)."""
    return int(_load().gjin_rand(seed & (2**64 - 1), tag))


def er_edges(n: int, m: int, seed: int = 1):
    """Directed Erdos-Renyi graph: m distinct (u, v) pairs, u != v, uniform over [0, n)^2."""
    src = np.empty(m, dtype=np.uint32)
    dst = np.empty(m, dtype=np.uint32)
    got = _load().gjin_er(n, m, subseed(seed, 1), _p32(src), _p32(dst))
    if got != m:
        raise ValueError("cannot draw %d distinct edges on %d vertices" % (m, n))
    return src, dst


_perm_cache: dict = {}


def permutation(n: int, seed: int) -> np.ndarray:
    key = (n, seed)
    if key not in _perm_cache:
        perm = np.empty(n, dtype=np.uint32)
        _load().gjin_permutation(n, seed, _p32(perm))
        if len(_perm_cache) > 4:
            _perm_cache.clear()
        _perm_cache[key] = perm
    return _perm_cache[key]


def rmat_edges(scale: int, edge_factor: int = 16, seed: int = 1, first: int = 0, count: int | None = None,
               abc=RMAT_ABC, permute: bool = True, stream: int = 2):
    """Raw R-MAT samples first..first+count-1 on 2**scale vertices.

    The default count is edge_factor * 2**scale (16M samples at scale 20).
    Vertex ids pass through a seeded permutation. Duplicates and self-loops
    are kept; the graph loaders drop them. ``stream`` picks an independent
    sample stream (2 = the base graph, 3 = inserts of update batches).
    """
    n = 1 << scale
    if count is None:
        count = edge_factor * n
    perm = permutation(n, subseed(seed, 7)) if permute else None
    src = np.empty(count, dtype=np.uint32)
    dst = np.empty(count, dtype=np.uint32)
    _load().gjin_rmat(scale, first, count, subseed(seed, stream), abc[0], abc[1], abc[2],
                      _p32(perm) if perm is not None else None, _p32(src), _p32(dst))
    return src, dst


def hub_edges(n: int, nhubs: int, deg: int, seed: int = 1):
    """Planted hubs: nhubs distinct vertex ids, each with deg distinct out- and deg distinct in-neighbours."""
    ids = np.empty(nhubs, dtype=np.uint32)
    chosen = set()
    ctr = 0
    while len(chosen) < nhubs:
        x = int(uniform(n, 1, subseed(seed, 11), first=ctr)[0])
        ctr += 1
        if x not in chosen:
            ids[len(chosen)] = x
            chosen.add(x)
    src = np.empty(2 * nhubs * deg, dtype=np.uint32)
    dst = np.empty(2 * nhubs * deg, dtype=np.uint32)
    if _load().gjin_hubs(n, nhubs, deg, subseed(seed, 12), _p32(ids), _p32(src), _p32(dst)) != 0:
        raise ValueError("hub degree too large")
    return ids, src, dst


def uniform(bound: int, count: int, seed: int, first: int = 0) -> np.ndarray:
    out = np.empty(count, dtype=np.uint64)
    _load().gjin_uniform(bound, first, count, seed, _p64(out))
    return out


def distinct_edges(src, dst):
    """Sorted distinct (u, v) pairs with u != v, as two uint32 arrays.

    Input shaping for update streams (deletions are drawn from existing
    edges); the loaders of both sides build their own indices independently.
    """
    keep = src != dst
    key = (src[keep].astype(np.uint64) << np.uint64(32)) | dst[keep].astype(np.uint64)
    key.sort()
    if len(key):
        key = key[np.concatenate(([True], key[1:] != key[:-1]))]
    return (key >> np.uint64(32)).astype(np.uint32), (key & np.uint64(0xffffffff)).astype(np.uint32)


class UpdateStream:
    """Insert/delete edge batches over a base graph (the dynamic-maintenance workload).

    Each batch holds round(0.9 b) inserts, fresh R-MAT samples from an
    independent stream of the same distribution, followed by b - round(0.9 b)
    deletes. Deletes walk a seeded permutation of the base graph's distinct
    edges, so every delete names an edge that exists at that point (no base
    edge is deleted twice, and inserts never remove edges). Batch t of the
    stream is a pure function of (seed, sizes of batches 0..t).
    """

    def __init__(self, base_src, base_dst, scale: int, seed: int = 1, insert_frac: float = 0.9):
        self.scale = scale
        self.seed = seed
        self.insert_frac = insert_frac
        bs, bd = distinct_edges(base_src, base_dst)
        self.base_src, self.base_dst = bs, bd
        m = len(bs)
        # seeded shuffle of base edge indices via sort of random keys
        keys = uniform(2**63, m, subseed(seed, 21))
        self.del_order = np.argsort(keys, kind="stable")
        self.del_cursor = 0
        self.ins_cursor = 0

    def next_batch(self, b: int):
        n_ins = int(round(self.insert_frac * b))
        n_del = b - n_ins
        if self.del_cursor + n_del > len(self.del_order):
            raise ValueError("update stream ran out of base edges to delete")
        isrc, idst = rmat_edges(self.scale, seed=self.seed, first=self.ins_cursor, count=n_ins, stream=3)
        self.ins_cursor += n_ins
        idx = self.del_order[self.del_cursor:self.del_cursor + n_del]
        self.del_cursor += n_del
        src = np.concatenate([isrc, self.base_src[idx]])
        dst = np.concatenate([idst, self.base_dst[idx]])
        sign = np.concatenate([np.ones(n_ins, np.int8), -np.ones(n_del, np.int8)])
        return src, dst, sign


# Query shapes of the evaluation (Section 5.1), as edge atoms E(a_s, a_d)
# over attributes 0..k-1 (a1..ak in the paper's numbering). "diamond" is the
# five-atom diamond E(a1,a2), E(a1,a3), E(a2,a4), E(a3,a4), E(a2,a3): two
# transitive triangles sharing the atom E(a2,a3). "4-cycle" is the paper's
# four-atom shape e(a1,a2), e(a2,a3), e(a4,a1), e(a4,a3). "triangle" is the
# transitive triangle of Section 5.1; "cyclic-triangle" is the one of
# Section 1 and Appendix A. "house" is the query of Section 5.4: a2..a5 form
# a clique and a1 is joined to a2 and a3 only (every edge oriented from the
# lower to the higher attribute).
QUERIES = {
    "triangle": (3, [(0, 1), (1, 2), (0, 2)]),
    "cyclic-triangle": (3, [(0, 1), (1, 2), (2, 0)]),
    "4-cycle": (4, [(0, 1), (1, 2), (3, 0), (3, 2)]),
    "diamond": (4, [(0, 1), (0, 2), (1, 3), (2, 3), (1, 2)]),
    "4-clique": (4, [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]),
    "5-clique": (5, [(i, j) for i in range(5) for j in range(i + 1, 5)]),
    "house": (5, [(0, 1), (0, 2), (1, 2), (1, 3), (1, 4), (2, 3), (2, 4), (3, 4)]),
}

# Formulations of the shapes above with the specialisations of Section 5.4,
# as keyword arguments of a query definition: "tri" lists ternary atoms
# tri(a_i, a_j, a_l) over the graph's triangles (a_i -> a_j, a_i -> a_l,
# a_j -> a_l, indexed by (a_i, a_j)); "lt" lists inequalities x_a < x_b
# (symmetry breaking on a symmetrised graph); "order" is an attribute
# order whose trailing attributes constrain one another in no way, so that
# their extensions can be factorised. Each has the same matches as the
# shape it is named after (on the graphs stated).
SPECIALISED = {
    # triangle indexing: each 4-clique is three triangles on a1
    "4-clique-tr": dict(k=4, atoms=[], tri=[(0, 1, 2), (0, 1, 3), (0, 2, 3)], lt=[], order=None),
    "5-clique-tr": dict(k=5, atoms=[], tri=[(0, 1, 2), (0, 1, 3), (0, 2, 3), (0, 1, 4), (0, 2, 4), (0, 3, 4)],
                        lt=[], order=None),
    # factorised: a1 and a4 (diamond), a1 and a5 (house) extend independently
    "diamond-f": dict(k=4, atoms=QUERIES["diamond"][1], tri=[], lt=[], order=[1, 2, 0, 3]),
    "house-f": dict(k=5, atoms=QUERIES["house"][1], tri=[], lt=[], order=[1, 2, 3, 0, 4]),
    # house with its clique a2..a5 from triangles and a1 joined by edge atoms, factorised
    "house-tr": dict(k=5, atoms=[(0, 1), (0, 2)], tri=[(1, 2, 3), (1, 2, 4), (1, 3, 4), (2, 3, 4)], lt=[],
                     order=[1, 2, 3, 0, 4]),
    # symmetry breaking on a symmetrised graph: one match per undirected subgraph
    "4-clique-sym": dict(k=4, atoms=QUERIES["4-clique"][1], tri=[], lt=[(0, 1), (1, 2), (2, 3)], order=None),
    "5-clique-sym": dict(k=5, atoms=QUERIES["5-clique"][1], tri=[], lt=[(0, 1), (1, 2), (2, 3), (3, 4)],
                         order=None),
    "house-sym": dict(k=5, atoms=QUERIES["house"][1], tri=[], lt=[(1, 2), (3, 4)], order=[1, 2, 3, 0, 4]),
}


def connected_order(atoms, order) -> bool:
    """True if the first two attributes of order share an atom and every later
    attribute shares an atom with an earlier one (the orders the loaders'
    edge-seeded evaluation accepts)."""
    pos = {a: i for i, a in enumerate(order)}
    if not any({pos[s], pos[d]} == {0, 1} for s, d in atoms):
        return False
    return all(any((pos[s] == j and pos[d] < j) or (pos[d] == j and pos[s] < j) for s, d in atoms)
               for j in range(2, len(order)))


def mixed_queries(count: int = 64, seed: int = 1):
    """The batched multi-query workload: the five evaluation shapes (triangle,
    4-cycle, diamond, 4-clique, 5-clique) in their canonical form, then
    seeded variants in which every atom's direction flips with probability
    1/2 and the attribute order is a random connected order. Returns
    (name, k, atoms, order) tuples."""
    shapes = ["triangle", "4-cycle", "diamond", "4-clique", "5-clique"]
    out = [(nm, QUERIES[nm][0], list(QUERIES[nm][1]), list(range(QUERIES[nm][0]))) for nm in shapes]
    ctr = 0
    rs = subseed(seed, 31)
    while len(out) < count:
        r = uniform(2**62, 64, rs, first=64 * ctr)
        ctr += 1
        nm = shapes[int(r[0] % 5)]
        k, atoms = QUERIES[nm]
        atoms = [(b, a) if (int(r[1 + t]) & 1) else (a, b) for t, (a, b) in enumerate(atoms)]
        # a random permutation of the attributes from the remaining draws
        order = sorted(range(k), key=lambda a: int(r[20 + a]))
        if not connected_order(atoms, order):
            continue
        out.append(("%s-v%d" % (nm, len(out)), k, atoms, order))
    return out
