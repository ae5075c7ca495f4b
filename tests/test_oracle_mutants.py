"""The pins reject a wrong oracle: each case plants one plausible mistake (a
dropped term, a wrong sign, index or bound, a transposed operand, swapped
versions) in a copy of oracle/gj_oracle.c, compiles the copy with gcc and
runs the oracle's pin tests (tests/test_oracle.py and
tests/test_oracle_specialisations.py) against it; every mutant must make
them fail. A control copy with no change must pass, so a failure is the
mutant's and not the harness's. Everything runs on the CPU; the copies live
in a temporary directory and the committed oracle is never changed."""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "gj_oracle.c")
PINS = ["tests/test_oracle.py", "tests/test_oracle_specialisations.py"]

# name -> (text in gj_oracle.c, replacement, the paper passage whose rule it breaks)
MUTANTS = {
    "duplicates-kept": (
        "if (u == 0 || keys[i] != keys[u - 1]) keys[u++] = keys[i];", "keys[u++] = keys[i];",
        "Section 2.1: a relation is a set of distinct tuples"),
    "self-loops-kept": (
        "if (hi[i] != lo[i]) keys[c++] =", "keys[c++] =",
        "Section 2.1: the edge relation of a simple graph"),
    "membership-misses-last": (
        "return lo < len && a[lo] == e;", "return lo + 1 < len && a[lo] == e;",
        "Section 2.2 (iii): membership in an extension set"),
    "extension-set-transposed": (
        "if (q->ad[t] == A) { s.a = g->fn + g->fo[vb];", "if (q->as[t] == A) { s.a = g->fn + g->fo[vb];",
        "Section 2.2: Ext for E(B, A) is out(B), for E(A, B) in(B)"),
    "largest-set-proposes": (
        "sets[nsets] = ext_set(r, t, A, j);\n        if (sets[nsets].len < sets[*imin].len)",
        "sets[nsets] = ext_set(r, t, A, j);\n        if (sets[nsets].len > sets[*imin].len)",
        "Fig. 1: the smallest extension set proposes (min-c)"),
    "intersection-skipped": (
        "if (!in_list(sets[s].a, sets[s].len, e)) return 0;", "(void)0;",
        "Fig. 1: a proposal is kept only if every other set holds it"),
    "first-level-range-off-by-one": (
        "if (j == 0 && (e < r->first_lo || e >= r->first_hi)) continue;",
        "if (j == 0 && (e < r->first_lo || e > r->first_hi)) continue;",
        "Theorem 2.1: counts add up over disjoint first-attribute ranges"),
    "hash-salt-index": (
        "(uint64_t)(a + 1) * 0x9e3779b97f4a7c15ULL", "(uint64_t)a * 0x9e3779b97f4a7c15ULL",
        "the match checksum's attribute salts"),
    "hash-factor-even": (
        "h *= mix64((uint64_t)x_by_attr[a] ^ salt) | 1u;", "h *= mix64((uint64_t)x_by_attr[a] ^ salt);",
        "the match checksum's odd factors"),
    "negative-matches-add": (
        "r->chk += (r->sign > 0) ? h : (uint64_t)(0 - h);", "r->chk += h;",
        "Section 3.3.1: a match seeded by a deletion counts negatively"),
    "delta-versions-swapped": (
        "(t < i) ? g_new : (t > i ? g_old : NULL)", "(t < i) ? g_old : (t > i ? g_new : NULL)",
        "Section 3.3.1: dQ_i reads new versions before i, old after i"),
    "first-update-decides": (
        "if (i + 1 < c && u[i + 1].key == u[i].key) continue;", "if (i > 0 && u[i - 1].key == u[i].key) continue;",
        "Section 3.3.1: updates apply in batch order, the last one decides"),
    "deletion-not-applied": (
        "if (lo < g->fo[u + 1] && d[lo] == ddst[i]) gone[lo] = 1;", "(void)lo;",
        "Section 3.3.1: R' = R + Delta R"),
    "seed-filter-dropped": (
        "if (ps <= 1 && pd <= 1) ok = has_edge(g, r.x[q.as[t]], r.x[q.ad[t]]);", "(void)ps; (void)pd;",
        "Section 4.1: further atoms over the seed pair filter the seeds"),
    "inequality-not-strict": (
        "!(e < r->x[q->lb[t]])", "!(e <= r->x[q->lb[t]])",
        "Section 5.4: symmetry breaking by strict inequalities"),
    "triangle-edge-reversed": (
        "edge_slot(g, r->x[q->ta[t]], r->x[q->tb[t]])", "edge_slot(g, r->x[q->tb[t]], r->x[q->ta[t]])",
        "Section 5.4: tri(a, b, c) is indexed by (a, b)"),
    "triangle-merge-misses-equal": (
        "if (g->fn[i] < g->fn[k]) i++;", "if (g->fn[i] <= g->fn[k]) i++;",
        "Section 5.4: the triangles on edge a -> b are out(a) intersected with out(b)"),
    "factorised-product-short": (
        "for (uint64_t i = 0; i < lens[j]; i++) {", "for (uint64_t i = 0; i + 1 < lens[j]; i++) {",
        "Section 5.4: factorised output is the Cartesian product of the trailing sets"),
    "degree-order-descending": (
        "for (uint32_t i = 0; i < g->n; i++) new_of_old[(uint32_t)key[i]] = i;",
        "for (uint32_t i = 0; i < g->n; i++) new_of_old[(uint32_t)key[i]] = g->n - 1 - i;",
        "Section 5.4: new ids ascend with degree"),
    "orientation-dropped": (
        "if (orient && !(u < w)) continue;", "(void)orient;",
        "Section 5.4: edges kept from the lower to the higher id"),
    "projection-transposed": (
        "if (q->as[t] == A) { s.a = g->srcs; s.len = g->nsrcs; }", "if (q->as[t] == A) { s.a = g->dsts; s.len = g->ndsts; }",
        "Section 2.2: a relation whose other attribute is unbound extends by its projection"),
    "inequality-lower-not-strict": (
        "!(r->x[q->la[t]] < e)", "!(r->x[q->la[t]] <= e)",
        "Section 5.4: symmetry breaking by strict inequalities"),
    "deep-inequalities-dropped": (
        "    return lt_ok(r, A, e, j);\n}", "    return 1;\n}",
        "Section 5.4: inequality filters on every level"),
    "seed-inequalities-dropped": (
        "if (r.pos[q.la[t]] <= 1 && r.pos[q.lb[t]] <= 1) ok = r.x[q.la[t]] < r.x[q.lb[t]];", "(void)ok;",
        "Section 5.4: inequalities between the seed attributes filter the seeds"),
    "seed-endpoints-swapped": (
        "seed = (int)t; sa = q.as[t]; sd = q.ad[t];", "seed = (int)t; sa = q.ad[t]; sd = q.as[t];",
        "Section 4.1: the seed atom's edges bind (source, target)"),
    "signed-count-dropped": (
        "r->count += r->sign;", "r->count += 1;",
        "Section 3.3.1: a match seeded by a deletion counts negatively"),
    "delta-seed-filter-old-version": (
        "ok = has_edge(v.view[t], r.x[s], r.x[d]);", "ok = has_edge(g_old, r.x[s], r.x[d]);",
        "Section 3.3.1: atoms before i read the new version"),
    "factorised-intersection-skipped": (
        "if (keep_candidate(r, j, A, e, sets, nsets, imin)) lists[j][lens[j]++] = e;", "lists[j][lens[j]++] = e;",
        "Section 5.4: each factorised set is still an intersection"),
    "factorised-tri-join-ignored": (
        "joins(pos, q->ta[t], q->tc[t], p, f) ||\n                joins(pos, q->tb[t], q->tc[t], p, f)",
        "joins(pos, q->ta[t], q->tc[t], p, f)",
        "Section 5.4: only attributes that constrain one another in no way factorise"),
    "factorised-prefixes-miscounted": (
        "if (j > r->fact_from && r->st) r->st->prefixes[j]++;", "if (j >= r->fact_from && r->st) r->st->prefixes[j]++;",
        "Section 2.2: prefix counts of the cost model"),
    "symmetrised-not-reversed": (
        "s[g->m + i] = d[i]; d[g->m + i] = s[i];", "s[g->m + i] = s[i]; d[g->m + i] = d[i];",
        "Section 5.4: symmetry breaking runs on the undirected graph"),
    "degree-ties-unbroken": (
        "(((uint64_t)(h->fo[v + 1] - h->fo[v]) << 32) | v)", "((uint64_t)(h->fo[v + 1] - h->fo[v]) << 32)",
        "Section 5.4: renaming by degree, ties by old id"),
    "probes-uncounted": (
        "if (r->st) r->st->probes[j]++;", "(void)0;",
        "Section 2.2: one membership test per proposal per other set"),
    "bindings-miscounted": (
        "r->st->nbind_sum[j] += nsets;", "r->st->nbind_sum[j] += nsets - 1;",
        "Section 2.2: one size lookup per binding relation"),
    "seed-range-off-by-one": (
        "if (r.x[a0] < first_lo || r.x[a0] >= first_hi) continue;", "if (r.x[a0] < first_lo || r.x[a0] > first_hi) continue;",
        "Theorem 2.1: counts add up over disjoint first-attribute ranges"),
    "listing-in-execution-order": (
        "r->out[r->written * q->k + a] = r->x[a];", "r->out[r->written * q->k + a] = r->x[r->order[a]];",
        "Section 2.1: a match is a tuple over the query's attributes"),
    "reverse-index-not-transposed": (
        "uint64_t mr = sorted_keys(dst, src, m, keys);", "uint64_t mr = sorted_keys(src, dst, m, keys);",
        "Section 4.1: the reverse index holds in-neighbours"),
    "insertions-not-applied": (
        "if (dsign[i] > 0) { s[m] = dsrc[i]; d[m] = ddst[i]; m++; }", "(void)0;",
        "Section 3.3.1: R' = R + Delta R"),
    "unchanged-edges-kept-as-changes": (
        "if ((u[i].sign > 0) == present) continue;", "(void)present;",
        "Section 3.3.1: only updates that change the relation are changes"),
    "factorisation-reaches-seed": (
        "    while (f > 2) {", "    while (f > 1) {",
        "Section 5.4: the seed attributes are not factorised"),
    "factorisation-needs-three": (
        "return (q->k - f >= 2) ? f : q->k;", "return (q->k - f >= 3) ? f : q->k;",
        "Section 5.4: two independent trailing attributes factorise"),
    "tri-order-unchecked": (
        "if (r.pos[q.tc[t]] < r.pos[q.ta[t]] || r.pos[q.tc[t]] < r.pos[q.tb[t]]) return OG_E_INVALID;", "(void)0;",
        "Section 5.4: tri binds its third attribute after its first two"),
    "unused-attribute-accepted": (
        "if (used != (1u << k) - 1) return OG_E_INVALID;", "(void)used;",
        "Section 2.1: every attribute appears in some atom"),
    "unbound-level-accepted": (
        "                if (r.pos[q.tc[t]] == j) ok = 1;\n            if (!ok) return OG_E_INVALID;",
        "                if (r.pos[q.tc[t]] == j) ok = 1;\n            (void)ok;",
        "Section 4.1: every later attribute is bound by an atom over earlier ones"),
    "sign-unchecked": (
        "if (sign[i] != 1 && sign[i] != -1) { free(u); return OG_E_INVALID; }", "(void)0;",
        "Section 3.3.1: an update inserts (+1) or deletes (-1)"),
    "equal-attribute-atom-accepted": (
        "if (q->as[t] >= k || q->ad[t] >= k || q->as[t] == q->ad[t]) return OG_E_INVALID;",
        "if (q->as[t] >= k || q->ad[t] >= k) return OG_E_INVALID;",
        "Section 2.1: an edge atom joins two distinct attributes"),
    "tri-seed-one-way": (
        "if ((q.ta[t] == a0 && q.tb[t] == a1) || (q.ta[t] == a1 && q.tb[t] == a0))",
        "if (q.ta[t] == a0 && q.tb[t] == a1)",
        "Section 5.4: a tri atom's key pair seeds in either order"),
    "degree-is-in-degree": (
        "key[v] = degree_order ? (((uint64_t)(h->fo[v + 1] - h->fo[v]) << 32) | v) : (uint64_t)v;",
        "key[v] = degree_order ? (((uint64_t)(h->ro[v + 1] - h->ro[v]) << 32) | v) : (uint64_t)v;",
        "Section 5.4: renaming by (out-)degree"),
    "edge-seed-one-way": (
        "if ((q.as[t] == a0 && q.ad[t] == a1) || (q.as[t] == a1 && q.ad[t] == a0))",
        "if (q.as[t] == a0 && q.ad[t] == a1)",
        "Section 4.2: an edge atom over the first two attributes seeds in either direction"),
    "delta-seed-ignores-sign": (
        "            r.sign = dsign[c];", "            r.sign = 1;",
        "Section 3.3.1: each match counts with its seed's sign"),
}


def _compile(src_text, path):
    with open(path + ".c", "w") as f:
        f.write(src_text)
    subprocess.check_call(["gcc", "-O1", "-w", "-fPIC", "-shared", "-o", path, path + ".c"])


def _run_pins(lib):
    env = dict(os.environ, GJ_ORACLE_LIB=lib)
    p = subprocess.run([sys.executable, "-m", "pytest", *PINS, "-x", "-q", "-m", "not gpu",
                        "-p", "no:cacheprovider"], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    return p.returncode, (p.stdout + p.stderr)[-2000:]


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    if shutil.which("gcc") is None:
        pytest.skip("gcc is not installed")
    src = open(SRC).read()
    d = tmp_path_factory.mktemp("mutants")
    libs = {"control": str(d / "libcontrol.so")}
    _compile(src, libs["control"])
    for name, (old, new, _) in MUTANTS.items():
        assert src.count(old) == 1, f"{name}: the planted text must occur once in gj_oracle.c"
        libs[name] = str(d / f"lib{name}.so")
        _compile(src.replace(old, new), libs[name])
    with ThreadPoolExecutor(max_workers=max(2, os.cpu_count() or 2)) as ex:
        res = dict(zip(libs, ex.map(_run_pins, libs.values())))
    return res


def test_control_copy_passes(outcomes):
    rc, tail = outcomes["control"]
    assert rc == 0, tail


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_reject_mutant(outcomes, name):
    rc, tail = outcomes[name]
    # exit code 1: tests ran and at least one failed (not a collection or usage error)
    assert rc == 1, f"mutant {name} ({MUTANTS[name][2]}) survived or broke the harness:\n{tail}"
