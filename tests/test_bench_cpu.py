"""Host logic of bench.py, on the CPU: the reference arm's JSON line (the
CPU oracle timed on a bounded sample of the benchmark's workload), the
silence of non-zero ranks under torchrun, and the cost model behind the
roofline's algorithmic bytes, worked by hand on complete DAGs."""
import contextlib
import io
import json
import types

import numpy as np

import bench
import oracle
from paper_1802_03760_b300.inputs import QUERIES


def _args(**kw):
    a = types.SimpleNamespace(gpus=1, steps=2, warmup=1, impl="reference", scale=10,
                              queries=list(bench.BENCH_QUERIES))
    a.__dict__.update(kw)
    return a


def _run_reference(monkeypatch, **env):
    orig = bench.cpu_sample
    # a short sample per step; the arm's own sizing gives each step seconds
    monkeypatch.setattr(bench, "cpu_sample", lambda s, d, n, target, q: orig(s, d, n, 0.05, q))
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    for k, v in env.items():
        monkeypatch.setenv(k, v)
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        rc = bench.run_reference(_args())
    return rc, [ln for ln in buf.getvalue().splitlines() if ln.strip()]


def test_reference_arm_prints_one_line(monkeypatch):
    rc, lines = _run_reference(monkeypatch)
    assert rc == 0 and len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference"
    assert line["metric"] == bench.METRIC and line["unit"] == "matches/s"
    assert line["higher_is_better"] is True and line["steps"] == 2 and line["warmup"] == 1
    assert line["value"] >= 0 and line["config"]["workload"] == bench.workload_name(10, bench.BENCH_QUERIES)
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == line["value"]
    assert "ranges of 64 vertex ids at seeded random offsets" in cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": "matches/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_are_silent(monkeypatch):
    rc, lines = _run_reference(monkeypatch, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    assert rc == 0 and lines == []


def _work(n, name):
    s, d = np.triu_indices(n, 1)
    og = oracle.Graph(n, s.astype(np.uint32), d.astype(np.uint32))
    c, _, st = og.count(oracle.Query(*QUERIES[name]), stats=True, mode=1)
    w = types.SimpleNamespace(seeds=n * (n - 1) // 2, extended=list(st.extended), nbind=list(st.nbind_sum),
                              proposals=list(st.proposals), produced=list(st.prefixes))
    return c, w


def test_algorithmic_bytes_triangle_on_complete_dag():
    # DAG on 4 vertices (i -> j for i < j): 6 seed edges (a, b), each extended
    # by 2 binding lists with min count 3 - b: 2 + 1 + 0 + 1 + 0 + 0 = 4 proposals.
    c, w = _work(4, "triangle")
    assert c == 4 and (w.extended[2], w.nbind[2], w.proposals[2]) == (6, 12, 4)
    assert bench.algorithmic_bytes(w, 3) == 8 * 6 + 4 * 2 * 6 + 16 * 12 + 4 * 4 + 4 * 4 * 1 == 320


def test_algorithmic_bytes_4clique_on_complete_dag():
    # DAG on 6 vertices: 15 seeds with min count 5 - b (20 proposals, 20
    # triangles written as 3-tuples); 20 triangles (a, b, c) with 3 binding
    # lists and min count 5 - c (15 proposals, 2 probes each).
    c, w = _work(6, "4-clique")
    assert c == 15 and (w.proposals[2], w.produced[3], w.proposals[3]) == (20, 20, 15)
    level2 = 4 * 2 * 15 + 16 * 30 + 4 * 20 + 4 * 20 * 1 + 4 * 3 * 20
    level3 = 4 * 3 * 20 + 16 * 60 + 4 * 15 + 4 * 15 * 2
    assert bench.algorithmic_bytes(w, 4) == 8 * 15 + level2 + level3 == 2500


def test_golden_bytes_follow_the_cost_model():
    """The roofline's algorithmic bytes at full size come from the oracle's
    work units in the committed golden: for the triangle, 8 bytes per seed
    edge and, per seed, 4*2 + 16*2 + 4c + 4c bytes (two binding lists)."""
    gold = bench.golden_static(20)
    assert gold is not None and gold["edges"] == 16084904
    st = gold["queries"]["triangle"]["stats"]
    m, c = gold["edges"], st["proposals"][2]
    assert st["extended"][2] == m and st["nbind_sum"][2] == 2 * m
    assert bench.oracle_bytes(gold, "triangle") == 8 * m + 8 * m + 16 * 2 * m + 4 * c + 4 * c
    assert bench.golden_static(20, seed=2) is None and bench.golden_static(7) is None


def test_traffic_only_from_a_capture_of_the_current_kernel(tmp_path, monkeypatch):
    sha = bench.kernel_sources_sha()
    f = tmp_path / "p.md"
    monkeypatch.setattr(bench, "PROFILE", str(f))
    assert bench.profiled_traffic()[0] is None
    f.write_text("kernel_sources_sha256: %s\ntraffic_bytes_per_launch: 1234\n" % sha)
    assert bench.profiled_traffic()[0] == 1234
    f.write_text("kernel_sources_sha256: %s\ntraffic_bytes_per_launch: 1234\n" % ("0" * 64))
    assert bench.profiled_traffic() == (None, "kernel changed since the ncu capture")


def test_a_failing_sub_record_keeps_the_headline(capsys):
    """bench.sub_record returns the record, or on failure an error entry
    (and a stderr line) instead of raising, so the headline line is printed."""
    import bench

    assert bench.sub_record("delta", lambda x, y=1: {"v": x + y}, 2, y=3) == {"v": 5}

    def boom():
        raise RuntimeError("no box")

    r = bench.sub_record("serve", boom)
    assert r == {"error": "RuntimeError: no box"}
    assert "the serve record failed" in capsys.readouterr().err


def test_kernel_sha_ignores_comments_but_not_code():
    """The ncu capture stays valid across comment edits and not across code edits."""
    import bench

    src = "// layout\nint f(int x) { /* twice */ return 2 * x; }  // end\n\n"
    assert bench.code_only(src) == "int f(int x) {  return 2 * x; }"
    assert bench.code_only(src.replace("twice", "double").replace("layout", "the layout")) == bench.code_only(src)
    assert bench.code_only(src.replace("2 * x", "3 * x")) != bench.code_only(src)
