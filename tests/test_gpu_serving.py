"""The serving loop (gj_serve_start / gj_submit_* / gj_poll): requests that
overlap on the device (count waves merged into one fused launch, update
batches running while earlier waves still read the previous index) must
give exactly the results of running the same requests one by one, in
submission order, through the synchronous API; and a request must give the
same result alone as in the mix. Each wave balances its warps through a
donation queue of its own; forcing every batch through it changes no
result, and a wave whose bounded wait gives up fails its requests with
GJ_E_TIMEOUT without stopping the loop. A request withdrawn before it
starts (gj_cancel) is never run: the others give the results of the
sequential replay without it."""
import numpy as np
import pytest

import oracle
from paper_1802_03760_b300 import gj
from paper_1802_03760_b300.inputs import QUERIES, UpdateStream, rmat_edges

pytestmark = pytest.mark.gpu


def make_requests(seed, scale, nreq):
    s, d = rmat_edges(scale, seed=seed)
    stream = UpdateStream(s, d, scale, seed=seed)
    rng = np.random.default_rng(seed)
    names = sorted(QUERIES)
    reqs = []
    for _ in range(nreq):
        if rng.random() < 0.35:
            b = int(rng.choice([10, 100, 1000]))
            bs, bd, bg = stream.next_batch(b)
            reqs.append(("batch", (bs, bd, bg), ["triangle", "4-clique"]))
        else:
            k = int(rng.integers(1, 4))
            reqs.append(("count", None, [names[int(i)] for i in rng.choice(len(names), k, replace=False)]))
    return s, d, reqs


def replay(s, d, n, reqs):
    """The same requests one by one through the synchronous API on a fresh context."""
    ctx = gj.Context(0)
    g = gj.Graph(ctx, s, d, n)
    qmap = {nm: gj.Query(ctx, *QUERIES[nm]) for nm in QUERIES}
    out = []
    for kind, batch, names in reqs:
        qs = [qmap[nm] for nm in names]
        if kind == "count":
            c, h = gj.count_many(g, qs, engine=gj.ENGINE_FUSED)
        else:
            c, h = gj.apply_batch(g, *batch, qs)
        out.append((c, h, g.stats()[1]))
    ctx.close()
    return out


def serve(s, d, n, reqs, budget=0, **tuning):
    ctx = gj.Context(0)
    if tuning:
        gj.set_tuning(ctx, **tuning)
    g = gj.Graph(ctx, s, d, n)
    qmap = {nm: gj.Query(ctx, *QUERIES[nm]) for nm in QUERIES}
    srv = gj.Server(g, budget)
    ids = []
    for kind, batch, names in reqs:
        qs = [qmap[nm] for nm in names]
        ids.append(srv.submit_count(qs) if kind == "count" else srv.submit_batch(*batch, qs))
    res = [srv.poll(i) for i in ids]
    srv.stop()
    ctx.close()
    return res


def test_mixed_stream_equals_sequential_replay():
    scale = 12
    s, d, reqs = make_requests(41, scale, 40)
    want = replay(s, d, 1 << scale, reqs)
    got = serve(s, d, 1 << scale, reqs)
    for i, (r, (c, h, ver)) in enumerate(zip(got, want)):
        assert r["status"] == 0, (i, r)
        assert r["kind"] == reqs[i][0]
        assert (r["counts"], r["checksums"]) == (c, h), (i, reqs[i][0], reqs[i][2])
        assert r["version"] == ver, i
        assert r["end_ms"] >= r["start_ms"] >= r["submit_ms"]


def test_waves_with_forced_donation_equal_sequential_replay():
    scale = 12
    s, d, reqs = make_requests(53, scale, 24)
    want = replay(s, d, 1 << scale, reqs)
    got = serve(s, d, 1 << scale, reqs, donation=1)  # every batch of >= 32 prefixes handed on
    for i, (r, (c, h, ver)) in enumerate(zip(got, want)):
        assert r["status"] == 0, (i, r)
        assert (r["counts"], r["checksums"], r["version"]) == (c, h, ver), i


def test_wave_wait_gives_up_as_a_request_error():
    s, d = rmat_edges(10, seed=5)
    n = 1 << 10
    ctx = gj.Context(0)
    q = gj.Query(ctx, *QUERIES["triangle"])
    g = gj.Graph(ctx, s, d, n)
    want = gj.count(g, q)
    gj.set_tuning(ctx, wait_ms=50, fault=1)  # the queue waits on a warp that never finishes
    srv = gj.Server(g)
    r = srv.poll(srv.submit_count([q]))
    assert r["status"] == -6  # GJ_E_TIMEOUT
    srv.stop()
    gj.set_tuning(ctx)
    srv = gj.Server(g)
    r = srv.poll(srv.submit_count([q]))
    assert r["status"] == 0 and (r["counts"][0], r["checksums"][0]) == want
    srv.stop()
    ctx.close()


def test_cancelled_requests_are_never_run():
    scale = 13
    n = 1 << scale
    s, d = rmat_edges(scale, seed=61)
    stream = UpdateStream(s, d, scale, seed=61)
    reqs = []
    for i in range(40):
        if i % 2:
            reqs.append(("count", None, ["triangle", "4-clique"]))
        else:
            reqs.append(("batch", stream.next_batch(2000), ["triangle"]))
    ctx = gj.Context(0)
    g = gj.Graph(ctx, s, d, n)
    qmap = {nm: gj.Query(ctx, *QUERIES[nm]) for nm in QUERIES}
    srv = gj.Server(g)
    ids = [srv.submit_count([qmap[nm] for nm in names]) if kind == "count"
           else srv.submit_batch(*batch, [qmap[nm] for nm in names]) for kind, batch, names in reqs]
    # the newest first, while the loop works through the oldest
    cancelled = [False] * 10 + [srv.cancel(i) for i in reversed(ids[10:])][::-1]
    res = [srv.poll(i) for i in ids]
    with pytest.raises(gj.GJError) as ei:
        srv.cancel(ids[0])
    assert ei.value.code == -10  # retired by the poll
    srv.stop()
    ctx.close()
    assert any(cancelled)
    for r, c in zip(res, cancelled):
        assert (r["status"] == -12) == c  # GJ_E_CANCELLED
    want = replay(s, d, n, [q for q, c in zip(reqs, cancelled) if not c])
    got = [r for r, c in zip(res, cancelled) if not c]
    for i, (r, (c, h, ver)) in enumerate(zip(got, want)):
        assert r["status"] == 0, (i, r)
        assert (r["counts"], r["checksums"], r["version"]) == (c, h, ver), i


def test_request_alone_equals_in_mix():
    scale = 11
    s, d, reqs = make_requests(43, scale, 16)
    n = 1 << scale
    mixed = serve(s, d, n, reqs)
    # every count request, served alone on the graph state its predecessors leave
    for i, (kind, batch, names) in enumerate(reqs):
        if kind != "count" or i % 3:
            continue
        prefix = [r for r in reqs[:i] if r[0] == "batch"]
        alone = serve(s, d, n, prefix + [reqs[i]])[-1]
        assert (alone["counts"], alone["checksums"], alone["version"]) == \
            (mixed[i]["counts"], mixed[i]["checksums"], mixed[i]["version"]), i


def test_counts_match_oracle_after_served_batches():
    scale = 10
    s, d, reqs = make_requests(47, scale, 12)
    n = 1 << scale
    reqs.append(("count", None, sorted(QUERIES)))
    res = serve(s, d, n, reqs)
    og = oracle.Graph(n, s, d)
    for kind, batch, _ in reqs:
        if kind == "batch":
            og = oracle.apply_batch(og, *batch)[1]
    want = [og.count(oracle.Query(*QUERIES[nm])) for nm in sorted(QUERIES)]
    assert list(zip(res[-1]["counts"], res[-1]["checksums"])) == want


def test_admission_and_misuse():
    s, d = rmat_edges(10, seed=3)
    ctx = gj.Context(0)
    g = gj.Graph(ctx, s, d, 1 << 10)
    q = gj.Query(ctx, *QUERIES["triangle"])
    want = gj.count(g, q)
    srv = gj.Server(g, memory_budget_bytes=64 << 10)  # too small for any update batch
    rb = srv.submit_batch(np.array([1], np.uint32), np.array([2], np.uint32), np.array([1], np.int8), [q])
    rc = srv.submit_count([q])
    r = srv.poll(rb)
    assert r["status"] == -4  # GJ_E_ADMIT: the graph is unchanged
    r = srv.poll(rc)
    assert r["status"] == 0 and (r["counts"][0], r["checksums"][0]) == want and r["version"] == 0
    with pytest.raises(gj.GJError):
        gj.count(g, q)  # synchronous calls are refused while serving
    with pytest.raises(gj.GJError) as ei:
        srv.poll(rc)
    assert ei.value.code == -10  # retired
    srv.stop()
    assert gj.count(g, q) == want
    ctx.close()
