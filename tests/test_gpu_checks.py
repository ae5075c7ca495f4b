"""The checked build (libgj_checks.so, compiled with GJ_CHECKS): every
vertex id, list extent, edge slot, prefix-buffer slot and donated bundle
the kernels use is checked on the device, a failed check skips its access
and the call returns GJ_E_CHECK. On valid inputs no check may fail and the
results must equal the oracle's on every engine, query formulation and
update batch; a check made to fail on purpose (the context's failure
injection 3 narrows the graph views by one vertex, so the last vertex's
lists fall outside them -- no access leaves the real arrays) must be
reported, must leave the graph unchanged, and must leave the context
usable. The library is chosen when the binding is imported, so each case
runs in a child process with GJ_CHECKS=1."""
import os
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PRELUDE = textwrap.dedent('''
    import numpy as np
    import oracle
    from paper_1802_03760_b300 import gj
    from paper_1802_03760_b300.inputs import QUERIES, SPECIALISED, er_edges
    assert gj.checked_build() and gj.LIB_PATH.endswith("libgj_checks.so")
    n = 1500
    s, d = er_edges(n, 15000, seed=3)
    # the last vertex joined both ways to a few others, so its lists are read
    extra = np.array([1, 7, 20, 300], np.uint32)
    s = np.concatenate([s, np.full(4, n - 1, np.uint32), extra])
    d = np.concatenate([d, extra, np.full(4, n - 1, np.uint32)])
    og = oracle.Graph(n, s, d)
    ctx = gj.Context(0)
    g = gj.Graph(ctx, s, d, n)
''')

VALID = PRELUDE + textwrap.dedent('''
    names = sorted(QUERIES)
    for nm in names:
        want = og.count(oracle.Query(*QUERIES[nm]))
        q = gj.Query(ctx, *QUERIES[nm])
        for eng in (gj.ENGINE_PLAIN, gj.ENGINE_FUSED):
            assert gj.count(g, q, engine=eng) == want, (nm, eng)
    for nm, sp in sorted(SPECIALISED.items()):
        want = og.count(oracle.Query(sp["k"], sp["atoms"], sp["order"], tri=sp["tri"], lt=sp["lt"]), mode=1)
        q = gj.Query(ctx, sp["k"], sp["atoms"], sp["order"], tri=sp["tri"], lt=sp["lt"])
        for eng in (gj.ENGINE_PLAIN, gj.ENGINE_FUSED):
            assert gj.count(g, q, engine=eng) == want, (nm, eng)
    # every batch of prefixes through the donation queue
    gj.set_tuning(ctx, donation=1)
    qs = [gj.Query(ctx, *QUERIES[nm]) for nm in names]
    want = [og.count(oracle.Query(*QUERIES[nm])) for nm in names]
    assert list(zip(*gj.count_many(g, qs, engine=gj.ENGINE_FUSED))) == want
    gj.set_tuning(ctx)
    # update batches on both delta engines
    rng = np.random.default_rng(5)
    for flags in (gj.FLAG_DELTA_PLAIN, gj.FLAG_DELTA_FUSED):
        c2 = gj.Context(0, flags=flags)
        g2 = gj.Graph(c2, s, d, n)
        o2 = og
        q2 = [gj.Query(c2, *QUERIES[nm]) for nm in names]
        for b in range(3):
            bs = rng.integers(0, n, 400).astype(np.uint32)
            bd = rng.integers(0, n, 400).astype(np.uint32)
            bg = rng.choice(np.array([-1, 1], np.int8), 400)
            (cs, cd, cg), o3 = oracle.apply_batch(o2, bs, bd, bg)
            want = [oracle.delta(o2, o3, cs, cd, cg, oracle.Query(*QUERIES[nm])) for nm in names]
            assert list(zip(*gj.apply_batch(g2, bs, bd, bg, q2))) == want, (flags, b)
            o2 = o3
        c2.close()
    print("OK")
''')

INJECTED = PRELUDE + textwrap.dedent('''
    q = gj.Query(ctx, *QUERIES["triangle"])
    want = og.count(oracle.Query(*QUERIES["triangle"]))
    m0, v0 = g.stats()
    gj.set_tuning(ctx, fault=3)
    for eng in (gj.ENGINE_PLAIN, gj.ENGINE_FUSED):
        try:
            gj.count(g, q, engine=eng)
            raise SystemExit("no check failed on engine %d" % eng)
        except gj.GJError as e:
            assert e.code == -11 and "vertex id" in str(e), (eng, e.code, str(e))
    try:
        gj.apply_batch(g, np.array([0], np.uint32), np.array([n - 1], np.uint32), np.array([1], np.int8), [q])
        raise SystemExit("no check failed on the update batch")
    except gj.GJError as e:
        assert e.code == -11, e.code
    assert g.stats() == (m0, v0)  # not committed
    gj.set_tuning(ctx)
    for eng in (gj.ENGINE_PLAIN, gj.ENGINE_FUSED):
        assert gj.count(g, q, engine=eng) == want
    print("OK")
''')


def run_child(code):
    env = dict(os.environ, GJ_CHECKS="1")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0 and r.stdout.strip().endswith("OK"), r.stdout[-2000:] + r.stderr[-4000:]


def test_checked_build_on_valid_inputs_equals_oracle():
    run_child(VALID)


def test_checked_build_reports_a_failed_check():
    run_child(INJECTED)
