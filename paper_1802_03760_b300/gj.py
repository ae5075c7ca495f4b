"""Thin Python binding of libgj (include/gj.h), argument marshalling only.

Every step of the evaluation runs in the CUDA library; this module converts
numpy arrays, torch tensors and Python lists to pointers and raises on error
codes. If ``libgj.so`` has not been built it raises instead of falling back
to anything else. With the environment variable GJ_CHECKS=1 it loads the
checked build ``libgj_checks.so`` instead (device bounds checks that return
GJ_E_CHECK).
"""
from __future__ import annotations

import ctypes
import os
import re
import weakref

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgj_checks.so" if os.environ.get("GJ_CHECKS") == "1" else "libgj.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "gj.h")

ENGINE_PLAIN = 0
ENGINE_FUSED = 1
FLAG_DELTA_FUSED = 1
FLAG_DELTA_PLAIN = 2
LOAD_SYMMETRIZE = 1
LOAD_DEGREE_ORDER = 2
LOAD_ORIENT = 4

ERRORS = {
    -1: "GJ_E_INVALID", -2: "GJ_E_RANGE", -3: "GJ_E_NOMEM", -4: "GJ_E_ADMIT", -5: "GJ_E_TRUNCATED",
    -6: "GJ_E_TIMEOUT", -7: "GJ_E_OVERFLOW", -8: "GJ_E_CUDA", -9: "GJ_E_PENDING", -10: "GJ_E_NOTFOUND",
    -11: "GJ_E_CHECK", -12: "GJ_E_CANCELLED",
}


class GJError(RuntimeError):
    def __init__(self, code: int, msg: str = ""):
        self.code = code
        super().__init__("%s (%d)%s" % (ERRORS.get(code, "error"), code, (": " + msg) if msg else ""))


class Options(ctypes.Structure):
    _fields_ = [("prefix_buffer_bytes", ctypes.c_uint64), ("window", ctypes.c_uint64),
                ("engine", ctypes.c_uint32), ("flags", ctypes.c_uint32), ("stream", ctypes.c_void_p)]


class WorkStats(ctypes.Structure):
    _fields_ = [("seeds", ctypes.c_int64), ("extended", ctypes.c_int64 * 9), ("nbind", ctypes.c_int64 * 9),
                ("proposals", ctypes.c_int64 * 9), ("produced", ctypes.c_int64 * 9)]

    def as_dict(self):
        return {"seeds": self.seeds, "extended": list(self.extended), "nbind": list(self.nbind),
                "proposals": list(self.proposals), "produced": list(self.produced)}


class Tuning(ctypes.Structure):
    _fields_ = [("seed_chunk", ctypes.c_uint32), ("blocks_per_sm", ctypes.c_uint32),
                ("prefix_buffer_bytes", ctypes.c_uint64), ("fused_ms", ctypes.c_double), ("plain_ms", ctypes.c_double),
                ("donation", ctypes.c_uint32), ("wait_ms", ctypes.c_uint32), ("fault", ctypes.c_uint32),
                ("fault_count", ctypes.c_uint32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class Result(ctypes.Structure):
    _fields_ = [("req_id", ctypes.c_uint64), ("status", ctypes.c_int32), ("kind", ctypes.c_uint32),
                ("nq", ctypes.c_uint32), ("reserved", ctypes.c_uint32), ("counts", ctypes.c_int64 * 64),
                ("checksums", ctypes.c_uint64 * 64), ("version", ctypes.c_uint64), ("submit_ms", ctypes.c_double),
                ("start_ms", ctypes.c_double), ("end_ms", ctypes.c_double)]

    def as_dict(self):
        n = self.nq
        return {"req_id": self.req_id, "status": self.status, "kind": "count" if self.kind == 0 else "batch",
                "counts": [int(x) for x in self.counts[:n]], "checksums": [int(x) for x in self.checksums[:n]],
                "version": self.version, "submit_ms": self.submit_ms, "start_ms": self.start_ms,
                "end_ms": self.end_ms, "latency_ms": self.end_ms - self.submit_ms}


_lib = None

_VP = ctypes.c_void_p
_U32P = ctypes.POINTER(ctypes.c_uint32)
_I64P = ctypes.POINTER(ctypes.c_int64)
_U64P = ctypes.POINTER(ctypes.c_uint64)

_SIGS = {
    "gj_create": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(Options), ctypes.POINTER(_VP)]),
    "gj_destroy": (None, [_VP]),
    "gj_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "gj_last_error": (ctypes.c_char_p, [_VP]),
    "gj_graph_load": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_uint64, ctypes.c_uint32, ctypes.POINTER(_VP)]),
    "gj_graph_load_ex": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                        ctypes.POINTER(_VP)]),
    "gj_graph_relabel_map": (ctypes.c_int, [_VP, _U32P]),
    "gj_graph_build_triangles": (ctypes.c_int, [_VP, _U64P]),
    "gj_graph_stats": (ctypes.c_int, [_VP, _U64P, _U64P]),
    "gj_graph_export": (ctypes.c_int, [_VP, _I64P, _U32P]),
    "gj_graph_free": (None, [_VP]),
    "gj_query_define": (ctypes.c_int, [_VP, ctypes.c_uint32, _U32P, ctypes.c_uint32, _U32P, ctypes.POINTER(_VP)]),
    "gj_query_define_ex": (ctypes.c_int, [_VP, ctypes.c_uint32, _U32P, ctypes.c_uint32, _U32P, ctypes.c_uint32, _U32P,
                                          ctypes.c_uint32, _U32P, ctypes.POINTER(_VP)]),
    "gj_query_free": (None, [_VP]),
    "gj_count": (ctypes.c_int, [_VP, _VP, _I64P, _U64P]),
    "gj_count_ex": (ctypes.c_int, [_VP, _VP, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, _I64P, _U64P,
                                   ctypes.POINTER(WorkStats)]),
    "gj_count_many": (ctypes.c_int, [_VP, ctypes.POINTER(_VP), ctypes.c_uint32, ctypes.c_uint32, _I64P, _U64P]),
    "gj_count_noalloc": (ctypes.c_int, [_VP, ctypes.POINTER(_VP), ctypes.c_uint32, _I64P, _U64P]),
    "gj_count_many_ex": (ctypes.c_int, [_VP, ctypes.POINTER(_VP), ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                        ctypes.c_uint32, _I64P, _U64P]),
    "gj_get_tuning": (ctypes.c_int, [_VP, ctypes.POINTER(Tuning)]),
    "gj_set_tuning": (ctypes.c_int, [_VP, ctypes.POINTER(Tuning)]),
    "gj_autotune": (ctypes.c_int, [_VP, ctypes.POINTER(_VP), ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint32,
                                   ctypes.c_uint32, ctypes.POINTER(Tuning)]),
    "gj_last_work": (ctypes.c_int, [_VP, ctypes.POINTER(WorkStats)]),
    "gj_list": (ctypes.c_int, [_VP, _VP, _U32P, ctypes.c_uint64, _U64P, _I64P, _U64P]),
    "gj_apply_batch": (ctypes.c_int, [_VP, _VP, _VP, _VP, ctypes.c_uint64, ctypes.POINTER(_VP), ctypes.c_uint32,
                                      _I64P, _U64P]),
    "gj_graph_last_batch": (ctypes.c_int, [_VP, _U64P]),
    "gj_serve_start": (ctypes.c_int, [_VP, _VP, ctypes.c_uint64]),
    "gj_serve_stop": (ctypes.c_int, [_VP]),
    "gj_submit_count": (ctypes.c_int, [_VP, ctypes.POINTER(_VP), ctypes.c_uint32, _U64P]),
    "gj_submit_batch": (ctypes.c_int, [_VP, _VP, _VP, _VP, ctypes.c_uint64, ctypes.POINTER(_VP), ctypes.c_uint32,
                                       _U64P]),
    "gj_poll": (ctypes.c_int, [_VP, ctypes.c_uint64, ctypes.c_int, ctypes.POINTER(Result)]),
    "gj_profile_enable": (ctypes.c_int, [_VP, ctypes.c_int]),
    "gj_profile_read": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_double), _U64P]),
    "gj_ctx_stream": (_VP, [_VP]),
    "gj_launch_count": (ctypes.c_uint64, [_VP]),
    "gj_checked_build": (ctypes.c_int, []),
    "gj_cancel": (ctypes.c_int, [_VP, ctypes.c_uint64]),
    "gj_sync": (ctypes.c_int, [_VP]),
}


def header_functions(path: str = HEADER):
    """Names of the functions include/gj.h declares."""
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gj_[a-z_0-9]+)\s*\(", text)))


def lib():
    """The loaded libgj (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(os.path.basename(LIB_PATH) + " is not built; run `python -m paper_1802_03760_b300.build` "
                              "(there is no fallback implementation)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ptr(a, elem: int = 4):
    """(pointer, keepalive) for a 1-D numpy array or sequence (converted to
    uint32, or int8 when elem == 1; values the target type cannot hold are
    refused, not wrapped), a 1-D contiguous integer torch tensor with
    elem-byte elements (host or device, read as is), or None."""
    if a is None:
        return None, None
    if hasattr(a, "data_ptr") and hasattr(a, "is_cuda"):
        if a.dim() != 1 or not a.is_contiguous() or a.element_size() != elem:
            raise ValueError("tensor arguments must be 1-D, contiguous, with %d-byte elements" % elem)
        if a.dtype.is_floating_point or a.dtype.is_complex or str(a.dtype) == "torch.bool":
            raise ValueError("tensor arguments must hold integers, not %s" % a.dtype)
        if a.is_cuda:
            # the library reads device inputs on its own stream: the work that
            # wrote this tensor (on the current stream) must have finished
            import torch
            torch.cuda.current_stream(a.device).synchronize()
        return ctypes.c_void_p(a.data_ptr()), a
    want = np.dtype(np.uint32 if elem == 4 else np.int8)
    src = np.asarray(a)
    if src.ndim != 1:
        raise ValueError("array arguments must be 1-D")
    if src.dtype != want and src.size:
        if src.dtype.kind not in "iu":
            raise ValueError("array arguments must hold integers, not %s" % src.dtype)
        lo, hi = np.iinfo(want).min, np.iinfo(want).max
        if int(src.min()) < lo or int(src.max()) > hi:
            raise ValueError("array values must lie in [%d, %d]" % (lo, hi))
    arr = np.ascontiguousarray(src, dtype=want)
    return ctypes.c_void_p(arr.ctypes.data), arr


def _same_length(*arrays) -> int:
    """The common length of the non-None arguments (0 if none); raises if they differ,
    since the library reads that many entries of each."""
    ns = {len(a) for a in arrays if a is not None}
    if len(ns) > 1:
        raise ValueError("edge arrays differ in length: %s" % sorted(ns))
    return ns.pop() if ns else 0


def _check(rc: int, ctx=None):
    if rc < 0:
        msg = ""
        if ctx is not None and ctx._h:
            m = lib().gj_last_error(ctx._h)
            msg = m.decode() if m else ""
        raise GJError(rc, msg)
    return rc


class Context:
    def __init__(self, device: int = 0, prefix_buffer_bytes: int = 0, window: int = 0, engine: int = ENGINE_FUSED,
                 stream=None, flags: int = 0):
        self._h = None
        self._server = None  # weakref to the context's running Server, if any
        o = Options(prefix_buffer_bytes, window, engine, flags, ctypes.c_void_p(stream) if stream else None)
        h = _VP()
        _check(lib().gj_create(device, ctypes.byref(o), ctypes.byref(h)))
        self._h = h
        self.device = device
        self._children = weakref.WeakSet()  # graphs and queries, freed before the context

    def _stop_server(self):
        """Stops the context's request loop (which may still read its graph
        and the queries of pending requests) before any of them is freed."""
        ref = getattr(self, "_server", None)
        s = ref() if ref is not None else None
        if s is not None:
            s.stop()
        self._server = None

    def close(self):
        if self._h:
            self._stop_server()
            for c in list(self._children):
                c.free()
            lib().gj_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def stream(self) -> int:
        return lib().gj_ctx_stream(self._h) or 0

    def sync(self):
        _check(lib().gj_sync(self._h), self)

    def profile(self, enabled: bool = True):
        _check(lib().gj_profile_enable(self._h, 1 if enabled else 0), self)

    def profile_read(self):
        ms = ctypes.c_double(0)
        n = ctypes.c_uint64(0)
        _check(lib().gj_profile_read(self._h, ctypes.byref(ms), ctypes.byref(n)), self)
        return ms.value, n.value

    @property
    def launches(self) -> int:
        return int(lib().gj_launch_count(self._h))

    def last_work(self) -> WorkStats:
        w = WorkStats()
        _check(lib().gj_last_work(self._h, ctypes.byref(w)), self)
        return w


def _check_device(ctx, *arrays):
    """Device tensors must be on the context's device (the library refuses others)."""
    for a in arrays:
        if a is not None and getattr(a, "is_cuda", False) and a.device.index != ctx.device:
            raise ValueError("tensor on cuda:%d, context on cuda:%d" % (a.device.index, ctx.device))


class Graph:
    def __init__(self, ctx: Context, src, dst, num_vertices: int, flags: int = 0):
        self.ctx = ctx
        self._h = None
        _check_device(ctx, src, dst)
        ps, ks = _ptr(src)
        pd, kd = _ptr(dst)
        m = _same_length(ks, kd)
        h = _VP()
        _check(lib().gj_graph_load_ex(ctx._h, ps, pd, m, num_vertices, flags, ctypes.byref(h)), ctx)
        self._h = h
        self.n = num_vertices
        ctx._children.add(self)

    def relabel_map(self):
        """new_of_old: the id each input vertex has in the graph's indices."""
        m = np.empty(max(self.n, 1), np.uint32)
        _check(lib().gj_graph_relabel_map(self._h, m.ctypes.data_as(_U32P)), self.ctx)
        return m[:self.n]

    def build_triangles(self) -> int:
        c = ctypes.c_uint64(0)
        _check(lib().gj_graph_build_triangles(self._h, ctypes.byref(c)), self.ctx)
        return c.value

    def free(self):
        if self._h:
            self.ctx._stop_server()  # gj_graph_free would stop it too, unseen by the Server object
            lib().gj_graph_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def stats(self):
        m = ctypes.c_uint64(0)
        v = ctypes.c_uint64(0)
        _check(lib().gj_graph_stats(self._h, ctypes.byref(m), ctypes.byref(v)), self.ctx)
        return m.value, v.value

    @property
    def m(self) -> int:
        return self.stats()[0]

    def export(self):
        off = np.empty(self.n + 1, np.int64)
        nbr = np.empty(max(self.m, 1), np.uint32)
        _check(lib().gj_graph_export(self._h, off.ctypes.data_as(_I64P), nbr.ctypes.data_as(_U32P)), self.ctx)
        return off, nbr[:self.m]


class Query:
    def __init__(self, ctx: Context, k: int, atoms, order=None, tri=(), lt=()):
        self.ctx = ctx
        self._h = None
        self.k = k
        self.atoms = [tuple(a) for a in atoms]
        self.tri = [tuple(t) for t in tri]
        self.lt = [tuple(c) for c in lt]
        flat = np.array([x for a in self.atoms for x in a] or [0], dtype=np.uint32)
        ft = np.array([x for t in self.tri for x in t] or [0], dtype=np.uint32)
        fl = np.array([x for c in self.lt for x in c] or [0], dtype=np.uint32)
        o = np.array(order, dtype=np.uint32) if order is not None else None
        h = _VP()
        _check(lib().gj_query_define_ex(ctx._h, k, flat.ctypes.data_as(_U32P) if self.atoms else None, len(self.atoms),
                                        ft.ctypes.data_as(_U32P) if self.tri else None, len(self.tri),
                                        fl.ctypes.data_as(_U32P) if self.lt else None, len(self.lt),
                                        o.ctypes.data_as(_U32P) if o is not None else None, ctypes.byref(h)), ctx)
        self._h = h
        ctx._children.add(self)

    def free(self):
        if self._h:
            ref = getattr(self.ctx, "_server", None)
            s = ref() if ref is not None else None
            if s is not None and any(q is self for qs in s._keep.values() for q in qs):
                s.stop()  # a pending request still reads this query: finish the requests first
            lib().gj_query_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def count(g: Graph, q: Query, engine: int | None = None, v_range=None, stats: bool = False):
    c = ctypes.c_int64(0)
    h = ctypes.c_uint64(0)
    if engine is None and v_range is None and not stats:
        _check(lib().gj_count(g._h, q._h, ctypes.byref(c), ctypes.byref(h)), g.ctx)
        return c.value, h.value
    lo, hi = v_range if v_range is not None else (0, 0xFFFFFFFF)
    w = WorkStats()
    _check(lib().gj_count_ex(g._h, q._h, ENGINE_FUSED if engine is None else engine, lo, hi, ctypes.byref(c),
                             ctypes.byref(h), ctypes.byref(w)), g.ctx)
    if stats:
        return c.value, h.value, w
    return c.value, h.value


def count_many(g: Graph, qs, engine: int = ENGINE_FUSED, v_range=None):
    n = len(qs)
    arr = (_VP * n)(*[q._h for q in qs])
    c = np.zeros(n, np.int64)
    h = np.zeros(n, np.uint64)
    if v_range is None:
        _check(lib().gj_count_many(g._h, arr, n, engine, c.ctypes.data_as(_I64P), h.ctypes.data_as(_U64P)), g.ctx)
    else:
        _check(lib().gj_count_many_ex(g._h, arr, n, engine, v_range[0], v_range[1], c.ctypes.data_as(_I64P),
                                      h.ctypes.data_as(_U64P)), g.ctx)
    return [int(x) for x in c], [int(x) for x in h]


def get_tuning(ctx: Context) -> dict:
    t = Tuning()
    _check(lib().gj_get_tuning(ctx._h, ctypes.byref(t)), ctx)
    return t.as_dict()


def checked_build() -> bool:
    """Whether the loaded library is the checked build (GJ_CHECKS=1)."""
    return bool(lib().gj_checked_build())


def set_tuning(ctx: Context, seed_chunk: int = 32, blocks_per_sm: int = 0, prefix_buffer_bytes: int = 0,
               donation: int = 0, wait_ms: int = 0, fault: int = 0, fault_count: int = 0):
    t = Tuning(seed_chunk, blocks_per_sm, prefix_buffer_bytes, 0.0, 0.0, donation, wait_ms, fault, fault_count)
    _check(lib().gj_set_tuning(ctx._h, ctypes.byref(t)), ctx)


def autotune(g: Graph, qs, v_range, prefix_cap_bytes: int = 2 << 30) -> dict:
    arr = (_VP * len(qs))(*[q._h for q in qs])
    t = Tuning()
    _check(lib().gj_autotune(g._h, arr, len(qs), prefix_cap_bytes, v_range[0], v_range[1], ctypes.byref(t)), g.ctx)
    return t.as_dict()


def count_noalloc(g: Graph, qs):
    """gj_count_noalloc: the fused multi-query count without any device allocation in the call."""
    n = len(qs)
    arr = (_VP * n)(*[q._h for q in qs])
    c = np.zeros(max(n, 1), np.int64)
    h = np.zeros(max(n, 1), np.uint64)
    _check(lib().gj_count_noalloc(g._h, arr, n, c.ctypes.data_as(_I64P), h.ctypes.data_as(_U64P)), g.ctx)
    return [int(x) for x in c[:n]], [int(x) for x in h[:n]]


def _ptr8(a):
    return _ptr(a, 1)


def apply_batch(g: Graph, src, dst, sign, qs=()):
    """Applies one update batch; returns ([delta counts], [delta checksums]) of qs."""
    _check_device(g.ctx, src, dst, sign)
    ps, ks = _ptr(src)
    pd, kd = _ptr(dst)
    pg, kg = _ptr8(sign)
    b = _same_length(ks, kd, kg)
    n = len(qs)
    arr = (_VP * max(n, 1))(*[q._h for q in qs])
    c = np.zeros(max(n, 1), np.int64)
    h = np.zeros(max(n, 1), np.uint64)
    _check(lib().gj_apply_batch(g._h, ps, pd, pg, b, arr if n else None, n, c.ctypes.data_as(_I64P) if n else None,
                                h.ctypes.data_as(_U64P) if n else None), g.ctx)
    return [int(x) for x in c[:n]], [int(x) for x in h[:n]]


def last_batch_changes(g: Graph) -> int:
    c = ctypes.c_uint64(0)
    _check(lib().gj_graph_last_batch(g._h, ctypes.byref(c)), g.ctx)
    return c.value


class Server:
    """The request loop of a context on one graph (gj_serve_start .. gj_serve_stop)."""

    def __init__(self, g: Graph, memory_budget_bytes: int = 0):
        self.g = g
        self.ctx = g.ctx
        self._keep = {}
        self.running = False
        _check(lib().gj_serve_start(self.ctx._h, g._h, memory_budget_bytes), self.ctx)
        self.running = True
        self.ctx._server = weakref.ref(self)

    def submit_count(self, qs) -> int:
        arr = (_VP * len(qs))(*[q._h for q in qs])
        rid = ctypes.c_uint64(0)
        _check(lib().gj_submit_count(self.ctx._h, arr, len(qs), ctypes.byref(rid)), self.ctx)
        self._keep[rid.value] = list(qs)
        return rid.value

    def submit_batch(self, src, dst, sign, qs=()) -> int:
        ps, ks = _ptr(src)
        pd, kd = _ptr(dst)
        pg, kg = _ptr8(sign)
        b = _same_length(ks, kd, kg)
        n = len(qs)
        arr = (_VP * max(n, 1))(*[q._h for q in qs])
        rid = ctypes.c_uint64(0)
        _check(lib().gj_submit_batch(self.ctx._h, ps, pd, pg, b, arr if n else None, n, ctypes.byref(rid)),
               self.ctx)
        self._keep[rid.value] = list(qs)
        return rid.value

    def cancel(self, rid: int) -> bool:
        """gj_cancel: True if the request was withdrawn before it started,
        False if it had already started (it runs to its end)."""
        rc = lib().gj_cancel(self.ctx._h, rid)
        if rc == -9:  # GJ_E_PENDING
            return False
        _check(rc, self.ctx)
        return True

    def poll(self, rid: int, wait_ms: int = -1):
        """The request's result as a dict, or None while it is pending."""
        r = Result()
        rc = lib().gj_poll(self.ctx._h, rid, wait_ms, ctypes.byref(r))
        if rc == -9:
            return None
        _check(rc, self.ctx)
        self._keep.pop(rid, None)
        return r.as_dict()

    def stop(self):
        """gj_serve_stop: finishes every submitted request, then ends the loop."""
        if self.running:
            self.running = False
            _check(lib().gj_serve_stop(self.ctx._h), self.ctx)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.stop()

    def __del__(self):
        try:
            self.stop()
        except Exception:
            pass


def list_matches(g: Graph, q: Query, cap: int):
    out = np.zeros((max(cap, 1), q.k), np.uint32)
    w = ctypes.c_uint64(0)
    t = ctypes.c_int64(0)
    h = ctypes.c_uint64(0)
    rc = lib().gj_list(g._h, q._h, out.ctypes.data_as(_U32P), cap, ctypes.byref(w), ctypes.byref(t),
                       ctypes.byref(h))
    if rc not in (0, -5):
        _check(rc, g.ctx)
    return out[:w.value], t.value, h.value, rc == -5
