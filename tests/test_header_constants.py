"""The limits and defaults that include/gj.h documents are the ones the
sources use: the largest query, the delta-engine threshold, the bounded
wait's default, the prefix-buffer default, the seed-chunk range, the
no-allocation entry point's scratch and query limit and the serving
request's query limit. CPU only (reads text)."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1802_03760_b300", "csrc")
HEADER = open(os.path.join(ROOT, "include", "gj.h")).read()
HEADER_FLAT = " ".join(re.sub(r"[/*]", " ", HEADER).split())


def src(name):
    return open(os.path.join(CSRC, name)).read()


def value(pattern, text):
    m = re.search(pattern, text)
    assert m, pattern
    return int(m.group(1))


def test_query_size_limits():
    max_k = value(r"#define GJ_MAX_K (\d+)", src("gj_internal.cuh"))
    max_atoms = value(r"#define GJ_MAX_ATOMS (\d+)", src("gj_internal.cuh"))
    assert "k < 2 or > %d, n_atoms > %d" % (max_k, max_atoms) in HEADER_FLAT


def test_delta_engine_threshold():
    n = value(r"GJ_DELTA_FUSED_MIN = (\d+);", src("gj_internal.cuh"))
    assert "fewer than %d normalised changes" % n in HEADER_FLAT


def test_wait_default():
    ms = value(r"ctx->wait_ms \? ctx->wait_ms : (\d+)\)", src("gj_internal.cuh"))
    assert "wait_ms milliseconds; 0 = %d" % ms in HEADER_FLAT


def test_prefix_buffer_default():
    mib = value(r"prefix_buffer_bytes : \((\d+)ull << 20\)", src("engine_plain.cu"))
    assert HEADER_FLAT.count("0 = %d MiB" % mib) == 2


def test_seed_chunk_range():
    lo = value(r"t->seed_chunk < (\d+)", src("capi.cu"))
    hi = value(r"t->seed_chunk > (\d+)", src("capi.cu"))
    mult = value(r"t->seed_chunk % (\d+)\)", src("capi.cu"))
    assert "(%d..%d, multiple of %d" % (lo, hi, mult) in HEADER_FLAT


def test_no_allocation_entry_point_limits():
    fused = src("engine_fused.cu")
    kib = value(r"NOALLOC_SCRATCH_BYTES = (\d+) \* 1024;", fused)
    nq = value(r"NOALLOC_MAX_QUERIES = (\d+);", fused)
    assert "one %d KiB array" % kib in HEADER_FLAT
    assert "%d queries per call" % nq in HEADER_FLAT


def test_serving_request_limit():
    nq = value(r"WAVE_MAX_QUERIES = (\d+);", src("serve.cu"))
    assert "Queues a count of nq <= %d queries" % nq in HEADER_FLAT
