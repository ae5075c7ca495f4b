"""CPU oracle for the Generic Join prefix-extension method (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may use this package. The library path never imports it.

``gj_oracle.c`` is a plain single-threaded C implementation of Generic Join
(Fig. 1, Section 2.2) starting from P0 = {()}, and of Delta-GJ's delta
queries (Section 3.3.1), with the specialisations of Section 5.4
(inequality constraints, degree-ordered renaming, the ternary triangle
relation, factorised output). It shares no code with the CUDA path. This
module only marshals arguments through ctypes and compiles the C file with
gcc.

Pins (what fixes the oracle other than itself) live in tests/test_oracle.py
and tests/test_oracle_specialisations.py: brute-force enumeration of V^k on
tiny graphs, closed forms on complete graphs, traces of adjacency powers on
symmetric graphs, the worked example of Appendix A, SplitMix64 reference
outputs, invariance under attribute order, delta = recount-after minus
recount-before and each delta query against its definition.
tests/test_oracle_mutants.py checks that the pins reject copies of
gj_oracle.c with planted mistakes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gj_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libgjoracle.so")
_lib = None
_lock = threading.Lock()

MAX_K = 8


class OracleError(RuntimeError):
    pass


_ERRS = {-1: "invalid argument", -2: "vertex id out of range", -3: "out of memory", -5: "output truncated"}


class Stats(ctypes.Structure):
    _fields_ = [("prefixes", ctypes.c_int64 * (MAX_K + 1)),
                ("extended", ctypes.c_int64 * (MAX_K + 1)),
                ("nbind_sum", ctypes.c_int64 * (MAX_K + 1)),
                ("proposals", ctypes.c_int64 * (MAX_K + 1)),
                ("probes", ctypes.c_int64 * (MAX_K + 1))]

    def as_dict(self):
        return {f: list(getattr(self, f)) for f, _ in self._fields_}


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-Wall", "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            # GJ_ORACLE_LIB names a separately compiled copy of gj_oracle.c;
            # tests/test_oracle_mutants.py points it at copies with planted
            # mistakes to check that the pins reject each one
            lib = ctypes.CDLL(os.environ.get("GJ_ORACLE_LIB") or build())
            u32p = ctypes.POINTER(ctypes.c_uint32)
            i8p = ctypes.POINTER(ctypes.c_int8)
            i64p = ctypes.POINTER(ctypes.c_int64)
            u64p = ctypes.POINTER(ctypes.c_uint64)
            ip = ctypes.POINTER(ctypes.c_int)
            vp = ctypes.c_void_p
            lib.og_graph_new.restype = vp
            lib.og_graph_new.argtypes = [ctypes.c_uint32, u32p, u32p, ctypes.c_uint64, ip]
            lib.og_graph_free.restype = None
            lib.og_graph_free.argtypes = [vp]
            lib.og_graph_num_edges.restype = ctypes.c_uint64
            lib.og_graph_num_edges.argtypes = [vp]
            lib.og_graph_edges.restype = None
            lib.og_graph_edges.argtypes = [vp, u32p, u32p]
            lib.og_mix64.restype = ctypes.c_uint64
            lib.og_mix64.argtypes = [ctypes.c_uint64]
            lib.og_tuple_hash.restype = ctypes.c_uint64
            lib.og_tuple_hash.argtypes = [ctypes.c_uint32, u32p]
            lib.og_count.restype = ctypes.c_int
            lib.og_count.argtypes = [vp, ctypes.c_uint32, u32p, ctypes.c_uint32, u32p, ctypes.c_uint32,
                                     ctypes.c_uint32, ctypes.c_int, i64p, u64p, ctypes.POINTER(Stats), u32p,
                                     ctypes.c_uint64, u64p]
            lib.og_count_ex.restype = ctypes.c_int
            lib.og_count_ex.argtypes = [vp, ctypes.c_uint32, u32p, ctypes.c_uint32, u32p, ctypes.c_uint32, u32p,
                                        ctypes.c_uint32, u32p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int, i64p,
                                        u64p, ctypes.POINTER(Stats), u32p, ctypes.c_uint64, u64p]
            lib.og_graph_num_triangles.restype = ctypes.c_uint64
            lib.og_graph_num_triangles.argtypes = [vp]
            lib.og_graph_transform.restype = vp
            lib.og_graph_transform.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, u32p, ip]
            lib.og_normalize.restype = ctypes.c_int64
            lib.og_normalize.argtypes = [vp, u32p, u32p, i8p, ctypes.c_uint64, u32p, u32p, i8p]
            lib.og_graph_apply.restype = vp
            lib.og_graph_apply.argtypes = [vp, u32p, u32p, i8p, ctypes.c_uint64, ip]
            lib.og_delta.restype = ctypes.c_int
            lib.og_delta.argtypes = [vp, vp, u32p, u32p, i8p, ctypes.c_uint64, ctypes.c_uint32, u32p,
                                     ctypes.c_uint32, u32p, i64p, u64p]
            lib.og_delta_each.restype = ctypes.c_int
            lib.og_delta_each.argtypes = lib.og_delta.argtypes + [i64p, u64p]
            _lib = lib
    return _lib


def _u32(a):
    a = np.ascontiguousarray(a, dtype=np.uint32)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


def _i8(a):
    a = np.ascontiguousarray(a, dtype=np.int8)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int8))


def _check(rc):
    if rc < 0:
        raise OracleError(_ERRS.get(rc, "error %d" % rc))
    return rc


def mix64(z: int) -> int:
    return int(_load().og_mix64(z))


def tuple_hash(xs) -> int:
    x, px = _u32(xs)
    return int(_load().og_tuple_hash(len(x), px))


class Query:
    """Q(a_0..a_{k-1}) := E(a_s, a_d), ..., tri(a_i, a_j, a_l), ... with x_a < x_b constraints.

    atoms: (s, d) pairs of attribute ids (edge atoms); tri: (i, j, l) triples
    (the ternary triangle relation of Section 5.4: i -> j, i -> l, j -> l,
    indexed by (i, j)); lt: (a, b) pairs meaning x_a < x_b (Section 5.4's
    inequality constraints, on vertex ids)."""

    def __init__(self, k: int, atoms, order=None, tri=(), lt=()):
        self.k = k
        self.atoms = [tuple(a) for a in atoms]
        self.tri = [tuple(t) for t in tri]
        self.lt = [tuple(c) for c in lt]
        self.order = list(order) if order is not None else None
        self._atoms = np.array([x for a in self.atoms for x in a] or [0], dtype=np.uint32)
        self._tri = np.array([x for t in self.tri for x in t] or [0], dtype=np.uint32)
        self._lt = np.array([x for c in self.lt for x in c] or [0], dtype=np.uint32)
        self._order = np.array(self.order, dtype=np.uint32) if self.order is not None else None

    def with_order(self, order):
        return Query(self.k, self.atoms, order, self.tri, self.lt)

    def _args(self):
        pa = self._atoms.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)) if self.atoms else None
        po = self._order.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)) if self._order is not None else None
        return pa, len(self.atoms), po

    def _ext_args(self):
        p = ctypes.POINTER(ctypes.c_uint32)
        pt = self._tri.ctypes.data_as(p) if self.tri else None
        pl = self._lt.ctypes.data_as(p) if self.lt else None
        return pt, len(self.tri), pl, len(self.lt)


class Graph:
    """The edge relation with forward and reverse indices (oracle copy)."""

    def __init__(self, n: int, src, dst, _handle=None):
        self.n = n
        lib = _load()
        if _handle is not None:
            self._h = _handle
        else:
            s, ps = _u32(src)
            d, pd = _u32(dst)
            if len(s) != len(d):
                raise ValueError("src and dst differ in length")
            err = ctypes.c_int(0)
            h = lib.og_graph_new(n, ps, pd, len(s), ctypes.byref(err))
            if not h:
                _check(err.value or -3)
            self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.og_graph_free(h)
            self._h = None

    @property
    def m(self) -> int:
        return int(_load().og_graph_num_edges(self._h))

    def edges(self):
        m = self.m
        s = np.empty(m, np.uint32)
        d = np.empty(m, np.uint32)
        _load().og_graph_edges(self._h, s.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                               d.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))
        return s, d

    def count(self, q: Query, first_range=None, stats: bool = False, mode: int = 0):
        """(count, checksum[, Stats]) of q; first_range = (lo, hi) limits the first attribute.

        mode 0: Generic Join from P0 as in Fig. 1 (the definition); mode 1:
        the paper's implementation (edge seeds, bound atoms only, Section 4.1
        and Section 4.2), whose work units the CUDA path reports; mode 2:
        mode 1 with factorised output for trailing attributes that constrain
        one another in no way (Section 5.4)."""
        lo, hi = first_range if first_range is not None else (0, 0xFFFFFFFF)
        c = ctypes.c_int64(0)
        h = ctypes.c_uint64(0)
        st = Stats() if stats else None
        pa, na, po = q._args()
        pt, nt, pl, nl = q._ext_args()
        _check(_load().og_count_ex(self._h, q.k, pa, na, pt, nt, pl, nl, po, lo, hi, mode, ctypes.byref(c),
                                   ctypes.byref(h), ctypes.byref(st) if st is not None else None, None, 0, None))
        if stats:
            return c.value, h.value, st
        return c.value, h.value

    def num_triangles(self) -> int:
        """Tuples of the ternary relation tri (a -> b, a -> c, b -> c)."""
        return int(_load().og_graph_num_triangles(self._h))

    def transform(self, symmetrize: bool = False, degree_order: bool = False, orient: bool = False):
        """(graph, new_of_old) after symmetry breaking's input transformation (Section 5.4):
        optional symmetrisation, renaming by ascending degree (ties by id), and keeping
        only the edges from a lower to a higher new id."""
        m = np.empty(max(self.n, 1), np.uint32)
        err = ctypes.c_int(0)
        h = _load().og_graph_transform(self._h, int(symmetrize), int(degree_order), int(orient),
                                       m.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), ctypes.byref(err))
        if not h:
            _check(err.value or -3)
        return Graph(self.n, None, None, _handle=h), m[:self.n].copy()

    def list(self, q: Query, cap: int | None = None):
        """All matches as a (count, k) uint32 array in query attribute order, plus the checksum."""
        if cap is None:
            cap = self.count(q)[0]
        out = np.zeros((max(cap, 1), q.k), np.uint32)
        c = ctypes.c_int64(0)
        h = ctypes.c_uint64(0)
        w = ctypes.c_uint64(0)
        pa, na, po = q._args()
        pt, nt, pl, nl = q._ext_args()
        _check(_load().og_count_ex(self._h, q.k, pa, na, pt, nt, pl, nl, po, 0, 0xFFFFFFFF, 1 if q.tri else 0,
                                   ctypes.byref(c), ctypes.byref(h), None,
                                   out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), cap, ctypes.byref(w)))
        return out[:w.value], h.value

    def normalize(self, src, dst, sign):
        """The net changes of an update batch under R' = R + Delta R, sorted by (src, dst)."""
        s, ps = _u32(src)
        d, pd = _u32(dst)
        g, pg = _i8(sign)
        b = len(s)
        os_ = np.empty(max(b, 1), np.uint32)
        od = np.empty(max(b, 1), np.uint32)
        og = np.empty(max(b, 1), np.int8)
        n = _check(_load().og_normalize(self._h, ps, pd, pg, b, os_.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                                        od.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                                        og.ctypes.data_as(ctypes.POINTER(ctypes.c_int8))))
        return os_[:n].copy(), od[:n].copy(), og[:n].copy()

    def apply(self, dsrc, dst, dsign) -> "Graph":
        """The graph after normalised changes."""
        s, ps = _u32(dsrc)
        d, pd = _u32(dst)
        g, pg = _i8(dsign)
        err = ctypes.c_int(0)
        h = _load().og_graph_apply(self._h, ps, pd, pg, len(s), ctypes.byref(err))
        if not h:
            _check(err.value or -3)
        return Graph(self.n, None, None, _handle=h)


def delta(g_old: Graph, g_new: Graph, dsrc, ddst, dsign, q: Query):
    """Delta-GJ: sum over dQ_i of signed matches (Section 3.3.1), from normalised changes."""
    s, ps = _u32(dsrc)
    d, pd = _u32(ddst)
    g, pg = _i8(dsign)
    c = ctypes.c_int64(0)
    h = ctypes.c_uint64(0)
    pa, na, po = q._args()
    _check(_load().og_delta(g_old._h, g_new._h, ps, pd, pg, len(s), q.k, pa, na, po, ctypes.byref(c),
                            ctypes.byref(h)))
    return c.value, h.value


def delta_each(g_old: Graph, g_new: Graph, dsrc, ddst, dsign, q: Query):
    """(count, checksum) of each delta query dQ_i, i in atom definition order
    (Section 3.3.1); their sums are delta()'s result."""
    s, ps = _u32(dsrc)
    d, pd = _u32(ddst)
    g, pg = _i8(dsign)
    c = ctypes.c_int64(0)
    h = ctypes.c_uint64(0)
    pa, na, po = q._args()
    ec = np.zeros(max(na, 1), np.int64)
    eh = np.zeros(max(na, 1), np.uint64)
    _check(_load().og_delta_each(g_old._h, g_new._h, ps, pd, pg, len(s), q.k, pa, na, po, ctypes.byref(c),
                                 ctypes.byref(h), ec.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                 eh.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))))
    return [(int(ec[i]), int(eh[i])) for i in range(na)]


def apply_batch(g: Graph, src, dst, sign):
    """(normalised changes, new graph) for one update batch."""
    ch = g.normalize(src, dst, sign)
    return ch, g.apply(*ch)


def algorithmic_bytes(st: Stats, k: int, count_only: bool = True) -> int:
    """Bytes the cost model moves for prefix lengths j >= 2 (the part after the edge seed).

    Per prefix of length j extended with n_j binding relations and min count c:
    4j (read the prefix) + 16 n_j (two 64-bit offsets per relation) + 4c
    (read the smallest list) + 4 c (n_j - 1) (one 4-byte membership probe per
    proposal per other relation), plus 4(j+1) per surviving prefix written
    for the next level (none at the last level when only counting).
    """
    total = 0
    for j in range(2, k):
        total += 4 * j * st.extended[j] + 16 * st.nbind_sum[j] + 4 * st.proposals[j] + 4 * st.probes[j]
        if j + 1 < k or not count_only:
            total += 4 * (j + 1) * st.prefixes[j + 1]
    return total
