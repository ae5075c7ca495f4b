"""Handle lifetimes in the binding, with the library replaced by a
recorder (no device): a running request loop reads its graph and the
queries of pending requests, so the binding stops it before freeing any of
them, whether the context is closed, the graph or such a query is freed,
or the Server object is dropped."""
import ctypes
import gc
import weakref

import pytest

from paper_1802_03760_b300 import gj


class FakeLib:
    def __init__(self):
        self.calls = []

    def __getattr__(self, name):
        def call(*args):
            self.calls.append(name)
            return 0
        return call


@pytest.fixture
def fake(monkeypatch):
    f = FakeLib()
    f.objects = []
    monkeypatch.setattr(gj, "_lib", f)
    yield f
    # the real library comes back after this: no object may still hold a fake handle
    for o in f.objects:
        if isinstance(o, weakref.ref):  # a Server, held weakly so that a test can drop it
            s = o()
            if s is not None:
                s.running = False
        else:
            o._h = None
    f.objects.clear()
    gc.collect()


def make(fake):
    ctx = gj.Context.__new__(gj.Context)
    ctx._h, ctx.device, ctx._server, ctx._children = ctypes.c_void_p(1), 0, None, weakref.WeakSet()
    g = gj.Graph.__new__(gj.Graph)
    g.ctx, g._h = ctx, ctypes.c_void_p(2)
    q = gj.Query.__new__(gj.Query)
    q.ctx, q._h = ctx, ctypes.c_void_p(3)
    ctx._children.add(g)
    ctx._children.add(q)
    srv = gj.Server(g)
    srv._keep[7] = [q]  # a pending request that reads q
    fake.objects += [ctx, g, q, weakref.ref(srv)]
    fake.calls.clear()
    return ctx, g, q, srv


def test_close_stops_the_loop_before_freeing(fake):
    ctx, g, q, srv = make(fake)
    ctx.close()
    c = fake.calls
    assert c[0] == "gj_serve_stop" and c[-1] == "gj_destroy"
    assert sorted(c[1:-1]) == ["gj_graph_free", "gj_query_free"]
    assert not srv.running
    srv.stop()  # already stopped: no second call
    assert c.count("gj_serve_stop") == 1


def test_freeing_the_graph_stops_the_loop_first(fake):
    ctx, g, q, srv = make(fake)
    g.free()
    assert fake.calls == ["gj_serve_stop", "gj_graph_free"] and not srv.running


def test_freeing_a_query_of_a_pending_request_stops_the_loop_first(fake):
    ctx, g, q, srv = make(fake)
    other = gj.Query.__new__(gj.Query)
    other.ctx, other._h = ctx, ctypes.c_void_p(4)
    fake.objects.append(other)
    other.free()  # no request reads it: the loop keeps running
    assert fake.calls == ["gj_query_free"] and srv.running
    q.free()
    assert fake.calls == ["gj_query_free", "gj_serve_stop", "gj_query_free"] and not srv.running


def test_dropping_the_server_stops_the_loop(fake):
    ctx, g, q, srv = make(fake)
    del srv
    gc.collect()
    assert fake.calls == ["gj_serve_stop"]
    ctx.close()
    assert fake.calls.count("gj_serve_stop") == 1


def test_server_as_context_manager(fake):
    ctx, g, q, srv = make(fake)
    with srv as s:
        assert s is srv and s.running
    assert fake.calls == ["gj_serve_stop"] and not srv.running
