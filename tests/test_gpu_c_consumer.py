"""A plain C program drives the library end to end: it includes only
include/gj.h, links libgj.so, loads the transitive tournament on 12
vertices (edges i -> j for i < j), defines the triangle and 4-clique queries
and counts them on the GPU; the counts and checksums it prints equal the
oracle's (C(12, 3) and C(12, 4) matches). No Python is on the call path."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from paper_1802_03760_b300 import gj
from paper_1802_03760_b300.build import build
from paper_1802_03760_b300.inputs import QUERIES

PROGRAM = r'''
#include <stdio.h>
#include "gj.h"

static int fail(gj_ctx* ctx, int rc) {
    fprintf(stderr, "%s: %s\n", gj_strerror(rc), ctx ? gj_last_error(ctx) : "");
    return 1;
}

int main(void) {
    enum { N = 12 };
    uint32_t src[N * (N - 1) / 2], dst[N * (N - 1) / 2];
    uint64_t m = 0;
    for (uint32_t i = 0; i < N; i++)
        for (uint32_t j = i + 1; j < N; j++) { src[m] = i; dst[m] = j; m++; }
    const uint32_t triangle[] = {0, 1, 1, 2, 0, 2};                  /* E(a0,a1), E(a1,a2), E(a0,a2) */
    const uint32_t clique4[] = {0, 1, 0, 2, 0, 3, 1, 2, 1, 3, 2, 3};  /* every pair a_i < a_j */
    gj_ctx* ctx = NULL;
    gj_graph* g = NULL;
    gj_query* q[2] = {NULL, NULL};
    int rc = gj_create(0, NULL, &ctx);
    if (rc) return fail(NULL, rc);
    if ((rc = gj_graph_load(ctx, src, dst, m, N, &g)) ||
        (rc = gj_query_define(ctx, 3, triangle, 3, NULL, &q[0])) ||
        (rc = gj_query_define(ctx, 4, clique4, 6, NULL, &q[1])))
        return fail(ctx, rc);
    int64_t counts[2];
    uint64_t chks[2];
    if ((rc = gj_count_many(g, (const gj_query* const*)q, 2, GJ_ENGINE_FUSED, counts, chks))) return fail(ctx, rc);
    printf("%lld %llu %lld %llu\n", (long long)counts[0], (unsigned long long)chks[0], (long long)counts[1],
           (unsigned long long)chks[1]);
    gj_query_free(q[0]);
    gj_query_free(q[1]);
    gj_graph_free(g);
    gj_destroy(ctx);
    return 0;
}
'''


@pytest.mark.gpu
def test_c_program_counts_on_the_gpu(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("gcc is not installed")
    libdir = os.path.dirname(build())
    src = tmp_path / "count.c"
    src.write_text(PROGRAM)
    exe = tmp_path / "count"
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I",
                           os.path.dirname(gj.HEADER), str(src), "-L", libdir, "-lgj", "-Wl,-rpath," + libdir,
                           "-o", str(exe)])
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    c3, h3, c4, h4 = (int(x) for x in out.stdout.split())
    n = 12
    s, d = np.triu_indices(n, 1)
    og = oracle.Graph(n, s.astype(np.uint32), d.astype(np.uint32))
    assert (c3, h3) == og.count(oracle.Query(*QUERIES["triangle"])) and c3 == 220
    assert (c4, h4) == og.count(oracle.Query(*QUERIES["4-clique"])) and c4 == 495
