/*
 * CPU oracle for the Generic Join prefix-extension method. TEST
 * INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg
 * of the benchmark call it; the library path never does.
 *
 * Plain, slow and single threaded on purpose. It shares no code with the
 * CUDA path. Every function says which part of the paper it follows:
 *   - relations and queries: Section 1 and Section 2.1 (a subgraph query is
 *     a multiway self-join of the edge relation under join semantics);
 *   - extension indices Ext^i_j with size, enumeration and membership:
 *     Section 2.2;
 *   - Generic Join from P0 = {()} to Pm, proposing from the smallest
 *     extension set and intersecting with the others: Fig. 1, Section 2.2;
 *   - delta queries dQ_1..dQ_n with new versions before i and old versions
 *     after i, seeded from the signed changes Delta R_i: Section 3.3.1
 *     (Delta-GJ) and Section 4.3;
 *   - update semantics R' = R + Delta R (a deletion removes the tuple):
 *     Section 3.3.1;
 *   - the specialisations of Section 5.4: inequality constraints between
 *     attributes (filters on prefixes), vertex ids renamed by degree with
 *     edges kept from the lower to the higher new id (symmetry breaking),
 *     the ternary relation tri(a_i, a_j, a_k) of the graph's triangles
 *     indexed by (a_i, a_j), and factorised output for trailing attributes
 *     that do not constrain one another.
 *
 * The match checksum is not from the paper; it is the order-independent sum
 * (mod 2^64) over matches of H(x_0..x_{k-1}) = q(k) * f_0(x_0) * ... *
 * f_{k-1}(x_{k-1}) (mod 2^64), with f_a(v) = m(v ^ s_a) | 1, q(k) = m(k) | 1,
 * s_a = (a + 1) * 0x9e3779b97f4a7c15 and m the SplitMix64 output function
 * (Steele, Lea, Flood, OOPSLA 2014); x_a is the value of query attribute a.
 * Every factor is odd, so H is a product in the group of odd residues and
 * the sum over a set of matches that agree on some attributes factorises
 * (the factorised output of Section 5.4 sums it without listing the set).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OG_MAX_K 8
#define OG_MAX_ATOMS 16

enum { OG_OK = 0, OG_E_INVALID = -1, OG_E_RANGE = -2, OG_E_NOMEM = -3, OG_E_TRUNCATED = -5 };

/* ---------------------------------------------------------------- graph */

typedef struct {
    uint32_t n;          /* vertices are 0..n-1 */
    uint64_t m;          /* distinct edges, no self-loops */
    uint64_t* fo;        /* forward offsets [n+1] */
    uint32_t* fn;        /* out-neighbours, sorted per vertex */
    uint64_t* ro;        /* reverse offsets [n+1] */
    uint32_t* rn;        /* in-neighbours, sorted per vertex */
    uint32_t* srcs;      /* vertices with out-degree > 0, ascending */
    uint64_t nsrcs;
    uint32_t* dsts;      /* vertices with in-degree > 0, ascending */
    uint64_t ndsts;
    /* ternary relation tri (Section 5.4), built on first use: for the
     * forward edge in slot e (u -> fn[e]), the vertices c with u -> c and
     * fn[e] -> c, ascending, are tn[to[e] .. to[e+1]) */
    uint64_t* to;
    uint32_t* tn;
} og_graph;

static int cmp_u64(const void* a, const void* b) {
    uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
    return (x > y) - (x < y);
}

/* Sorted distinct keys (hi << 32 | lo) from the pairs, self-loops dropped. */
static uint64_t sorted_keys(const uint32_t* hi, const uint32_t* lo, uint64_t m, uint64_t* keys) {
    uint64_t c = 0;
    for (uint64_t i = 0; i < m; i++)
        if (hi[i] != lo[i]) keys[c++] = ((uint64_t)hi[i] << 32) | lo[i];
    qsort(keys, c, sizeof(uint64_t), cmp_u64);
    uint64_t u = 0;
    for (uint64_t i = 0; i < c; i++)
        if (u == 0 || keys[i] != keys[u - 1]) keys[u++] = keys[i];
    return u;
}

/* Adjacency lists keyed by the high half of each key (an extension index, Section 2.2). */
static void lists_from_keys(uint32_t n, const uint64_t* keys, uint64_t m, uint64_t* off, uint32_t* nbr) {
    memset(off, 0, sizeof(uint64_t) * ((size_t)n + 1));
    for (uint64_t i = 0; i < m; i++) off[(keys[i] >> 32) + 1]++;
    for (uint32_t v = 0; v < n; v++) off[v + 1] += off[v];
    for (uint64_t i = 0; i < m; i++) nbr[i] = (uint32_t)keys[i];
}

void og_graph_free(og_graph* g) {
    if (!g) return;
    free(g->fo); free(g->fn); free(g->ro); free(g->rn); free(g->srcs); free(g->dsts);
    free(g->to); free(g->tn);
    free(g);
}

/*
 * The edge relation: distinct (src, dst) pairs, self-loops dropped, with a
 * forward index (out-neighbours of each vertex) and a reverse index
 * (in-neighbours), the two indices of Section 4.1. Returns NULL on a vertex
 * id >= n (*err = OG_E_RANGE) or when memory runs out.
 */
og_graph* og_graph_new(uint32_t n, const uint32_t* src, const uint32_t* dst, uint64_t m, int* err) {
    *err = OG_OK;
    for (uint64_t i = 0; i < m; i++)
        if (src[i] >= n || dst[i] >= n) { *err = OG_E_RANGE; return NULL; }
    og_graph* g = (og_graph*)calloc(1, sizeof(og_graph));
    uint64_t* keys = (uint64_t*)malloc(sizeof(uint64_t) * (m ? m : 1));
    if (!g || !keys) { free(g); free(keys); *err = OG_E_NOMEM; return NULL; }
    g->n = n;
    g->fo = (uint64_t*)malloc(sizeof(uint64_t) * ((size_t)n + 1));
    g->ro = (uint64_t*)malloc(sizeof(uint64_t) * ((size_t)n + 1));
    uint64_t mf = sorted_keys(src, dst, m, keys);
    g->m = mf;
    g->fn = (uint32_t*)malloc(sizeof(uint32_t) * (mf ? mf : 1));
    g->rn = (uint32_t*)malloc(sizeof(uint32_t) * (mf ? mf : 1));
    if (!g->fo || !g->ro || !g->fn || !g->rn) { free(keys); og_graph_free(g); *err = OG_E_NOMEM; return NULL; }
    lists_from_keys(n, keys, mf, g->fo, g->fn);
    uint64_t mr = sorted_keys(dst, src, m, keys);
    (void)mr; /* mr == mf: the same pair set, transposed */
    lists_from_keys(n, keys, mf, g->ro, g->rn);
    free(keys);
    g->srcs = (uint32_t*)malloc(sizeof(uint32_t) * ((size_t)n + 1));
    g->dsts = (uint32_t*)malloc(sizeof(uint32_t) * ((size_t)n + 1));
    if (!g->srcs || !g->dsts) { og_graph_free(g); *err = OG_E_NOMEM; return NULL; }
    for (uint32_t v = 0; v < n; v++) {
        if (g->fo[v + 1] > g->fo[v]) g->srcs[g->nsrcs++] = v;
        if (g->ro[v + 1] > g->ro[v]) g->dsts[g->ndsts++] = v;
    }
    return g;
}

uint64_t og_graph_num_edges(const og_graph* g) { return g->m; }

/* The distinct edges in (src, dst) order. */
void og_graph_edges(const og_graph* g, uint32_t* src, uint32_t* dst) {
    for (uint32_t v = 0; v < g->n; v++)
        for (uint64_t i = g->fo[v]; i < g->fo[v + 1]; i++) { src[i] = v; dst[i] = g->fn[i]; }
}

/* Membership of e in a sorted list (binary search): property (iii) of Section 2.2. */
static int in_list(const uint32_t* a, uint64_t len, uint32_t e) {
    uint64_t lo = 0, hi = len;
    while (lo < hi) {
        uint64_t mid = lo + (hi - lo) / 2;
        if (a[mid] < e) lo = mid + 1; else hi = mid;
    }
    return lo < len && a[lo] == e;
}

static int has_edge(const og_graph* g, uint32_t u, uint32_t v) {
    return in_list(g->fn + g->fo[u], g->fo[u + 1] - g->fo[u], v);
}

/* Slot of the edge u -> v in the forward index, or -1 if it is not an edge. */
static int64_t edge_slot(const og_graph* g, uint32_t u, uint32_t v) {
    uint64_t lo = g->fo[u], hi = g->fo[u + 1];
    while (lo < hi) {
        uint64_t mid = lo + (hi - lo) / 2;
        if (g->fn[mid] < v) lo = mid + 1; else hi = mid;
    }
    return (lo < g->fo[u + 1] && g->fn[lo] == v) ? (int64_t)lo : -1;
}

/* Size of out(a) intersected with out(b); with dst, also writes it, ascending. */
static uint64_t merge_out(const og_graph* g, uint32_t a, uint32_t b, uint32_t* dst) {
    uint64_t i = g->fo[a], ie = g->fo[a + 1], k = g->fo[b], ke = g->fo[b + 1], c = 0;
    while (i < ie && k < ke) {
        if (g->fn[i] < g->fn[k]) i++;
        else if (g->fn[i] > g->fn[k]) k++;
        else { if (dst) dst[c] = g->fn[i]; c++; i++; k++; }
    }
    return c;
}

/*
 * The ternary relation of the triangle-indexing specialisation (Section
 * 5.4): tri(a, b, c) holds when a -> b, a -> c and b -> c are edges, and it
 * is indexed by its first two attributes. For the forward edge in slot e
 * (a = the owner of the list holding e, b = fn[e]), the list of c is the
 * merge-intersection of out(a) and out(b), ascending. Built once per graph.
 */
static int build_tri(og_graph* g) {
    if (g->to) return OG_OK;
    uint64_t* to = (uint64_t*)malloc(sizeof(uint64_t) * (g->m + 1));
    if (!to) return OG_E_NOMEM;
    to[0] = 0;
    for (uint32_t a = 0; a < g->n; a++)
        for (uint64_t e = g->fo[a]; e < g->fo[a + 1]; e++) to[e + 1] = to[e] + merge_out(g, a, g->fn[e], NULL);
    uint32_t* tn = (uint32_t*)malloc(sizeof(uint32_t) * (to[g->m] ? to[g->m] : 1));
    if (!tn) { free(to); return OG_E_NOMEM; }
    for (uint32_t a = 0; a < g->n; a++)
        for (uint64_t e = g->fo[a]; e < g->fo[a + 1]; e++) merge_out(g, a, g->fn[e], tn + to[e]);
    g->to = to;
    g->tn = tn;
    return OG_OK;
}

/* Number of tuples of tri (0 on allocation failure). */
uint64_t og_graph_num_triangles(og_graph* g) { return build_tri(g) == OG_OK ? g->to[g->m] : 0; }

/* ---------------------------------------------------------------- query */

typedef struct {
    uint32_t k, natoms, ntri, nlt;
    uint32_t as[OG_MAX_ATOMS], ad[OG_MAX_ATOMS];  /* edge atom t is E(a_as[t], a_ad[t]) */
    uint32_t ta[OG_MAX_ATOMS], tb[OG_MAX_ATOMS], tc[OG_MAX_ATOMS];  /* tri atom t is tri(a_ta, a_tb, a_tc) */
    uint32_t la[OG_MAX_ATOMS], lb[OG_MAX_ATOMS];  /* inequality t: x_la[t] < x_lb[t] (vertex ids) */
    uint32_t order[OG_MAX_K];                     /* global attribute order */
} og_query;

/*
 * A query Q(a_0..a_{k-1}) := E(a_s, a_d), ..., tri(a_i, a_j, a_l), ...
 * (Section 2.1; tri atoms and inequalities from Section 5.4) with the
 * constraints x_a < x_b. 0 or OG_E_INVALID.
 */
static int make_query(uint32_t k, const uint32_t* atoms, uint32_t natoms, const uint32_t* tris, uint32_t ntri,
                      const uint32_t* lts, uint32_t nlt, const uint32_t* order, og_query* q) {
    if (k < 1 || k > OG_MAX_K || natoms > OG_MAX_ATOMS || ntri > OG_MAX_ATOMS || nlt > OG_MAX_ATOMS) return OG_E_INVALID;
    if (natoms + ntri < 1 || (natoms && !atoms) || (ntri && !tris) || (nlt && !lts)) return OG_E_INVALID;
    q->k = k; q->natoms = natoms; q->ntri = ntri; q->nlt = nlt;
    uint32_t used = 0;
    for (uint32_t t = 0; t < natoms; t++) {
        q->as[t] = atoms[2 * t]; q->ad[t] = atoms[2 * t + 1];
        if (q->as[t] >= k || q->ad[t] >= k || q->as[t] == q->ad[t]) return OG_E_INVALID;
        used |= (1u << q->as[t]) | (1u << q->ad[t]);
    }
    for (uint32_t t = 0; t < ntri; t++) {
        q->ta[t] = tris[3 * t]; q->tb[t] = tris[3 * t + 1]; q->tc[t] = tris[3 * t + 2];
        if (q->ta[t] >= k || q->tb[t] >= k || q->tc[t] >= k) return OG_E_INVALID;
        if (q->ta[t] == q->tb[t] || q->ta[t] == q->tc[t] || q->tb[t] == q->tc[t]) return OG_E_INVALID;
        used |= (1u << q->ta[t]) | (1u << q->tb[t]) | (1u << q->tc[t]);
    }
    for (uint32_t t = 0; t < nlt; t++) {
        q->la[t] = lts[2 * t]; q->lb[t] = lts[2 * t + 1];
        if (q->la[t] >= k || q->lb[t] >= k || q->la[t] == q->lb[t]) return OG_E_INVALID;
    }
    if (used != (1u << k) - 1) return OG_E_INVALID;  /* every attribute is in some atom */
    uint32_t seen = 0;
    for (uint32_t j = 0; j < k; j++) {
        uint32_t a = order ? order[j] : j;
        if (a >= k || (seen & (1u << a))) return OG_E_INVALID;
        seen |= 1u << a;
        q->order[j] = a;
    }
    return OG_OK;
}

/* ------------------------------------------------------------ checksum */

static uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

/* H of a match, tuple in query attribute order a_0..a_{k-1}: the query's
 * odd factor times one odd factor per attribute value, each salted by its
 * attribute so that the same value at two attributes weighs differently. */
static uint64_t tuple_hash(uint32_t k, const uint32_t* x_by_attr) {
    uint64_t h = mix64(k) | 1u;
    for (uint32_t a = 0; a < k; a++) {
        const uint64_t salt = (uint64_t)(a + 1) * 0x9e3779b97f4a7c15ULL;
        h *= mix64((uint64_t)x_by_attr[a] ^ salt) | 1u;
    }
    return h;
}

uint64_t og_mix64(uint64_t z) { return mix64(z); }
uint64_t og_tuple_hash(uint32_t k, const uint32_t* x) { return tuple_hash(k, x); }

/* ---------------------------------------------------------- Generic Join */

/*
 * Instrumentation of the prefix-extension work, in the units of the cost
 * model of Section 2.2 / Theorem 2.1 (one size lookup per binding relation
 * per prefix, one proposal per element of the smallest extension set, one
 * membership test per proposal per other binding relation). Index j is the
 * prefix length being extended.
 */
typedef struct {
    int64_t prefixes[OG_MAX_K + 1];   /* |P_j| reached */
    int64_t extended[OG_MAX_K + 1];   /* prefixes of length j that were extended */
    int64_t nbind_sum[OG_MAX_K + 1];  /* sum over those of the number of binding relations */
    int64_t proposals[OG_MAX_K + 1];  /* sum of min-c */
    int64_t probes[OG_MAX_K + 1];     /* membership tests */
} og_stats;

/* The relations (atoms) that one dQ_i evaluation sees (Section 3.3.1). */
typedef struct {
    const og_graph* view[OG_MAX_ATOMS];  /* graph each atom reads; NULL for the Delta atom */
} og_views;

typedef struct {
    const og_query* q;
    const og_views* v;
    const og_graph* g;          /* graph of the tri atoms (static evaluation only) */
    uint32_t order[OG_MAX_K];   /* execution order (attribute ids) */
    uint32_t pos[OG_MAX_K];     /* pos[a] = position of attribute a in the execution order */
    uint32_t x[OG_MAX_K];       /* x[a] = value bound to attribute a */
    uint32_t first_lo, first_hi;/* value range allowed for the first attribute */
    int sign;                   /* +1, or the sign of the Delta tuple that seeded this run */
    int bound_only;             /* 1: only atoms whose other attribute is bound bind a level (Section 4.1) */
    uint32_t fact_from;         /* first position of the factorised trailing attributes (k: none) */
    int64_t count;
    uint64_t chk;
    og_stats* st;
    uint32_t* out; uint64_t cap, written;  /* optional listing, tuples in query order */
} og_run;

/* One extension set Ext^t_j(p) for attribute A of atom t: a sorted list. */
typedef struct { const uint32_t* a; uint64_t len; } og_set;

static og_set ext_set(const og_run* r, uint32_t t, uint32_t A, uint32_t j) {
    const og_query* q = r->q;
    const og_graph* g = r->v->view[t];
    og_set s;
    uint32_t B = (q->as[t] == A) ? q->ad[t] : q->as[t];
    if (r->pos[B] < j) {
        uint32_t vb = r->x[B];
        if (q->ad[t] == A) { s.a = g->fn + g->fo[vb]; s.len = g->fo[vb + 1] - g->fo[vb]; }   /* E(B, A): out(B) */
        else { s.a = g->rn + g->ro[vb]; s.len = g->ro[vb + 1] - g->ro[vb]; }                  /* E(A, B): in(B) */
    } else {
        /* B comes later: the relation restricted to the first j+1 attributes is its projection on A */
        if (q->as[t] == A) { s.a = g->srcs; s.len = g->nsrcs; }
        else { s.a = g->dsts; s.len = g->ndsts; }
    }
    return s;
}

/* Extension set of tri atom t for its third attribute: the list indexed by
 * the bound values of its first two (empty when they are not an edge). */
static og_set tri_set(const og_run* r, uint32_t t) {
    const og_query* q = r->q;
    const og_graph* g = r->g;
    og_set s = {NULL, 0};
    int64_t e = edge_slot(g, r->x[q->ta[t]], r->x[q->tb[t]]);
    if (e >= 0) { s.a = g->tn + g->to[e]; s.len = g->to[e + 1] - g->to[e]; }
    return s;
}

/* The inequality constraints (Section 5.4) between attribute A, taking
 * value e at level j, and the attributes bound before it. */
static int lt_ok(const og_run* r, uint32_t A, uint32_t e, uint32_t j) {
    const og_query* q = r->q;
    for (uint32_t t = 0; t < q->nlt; t++) {
        if (q->la[t] == A && r->pos[q->lb[t]] < j && !(e < r->x[q->lb[t]])) return 0;
        if (q->lb[t] == A && r->pos[q->la[t]] < j && !(r->x[q->la[t]] < e)) return 0;
    }
    return 1;
}

static void emit(og_run* r) {
    const og_query* q = r->q;
    r->count += r->sign;
    uint64_t h = tuple_hash(q->k, r->x);
    r->chk += (r->sign > 0) ? h : (uint64_t)(0 - h);
    if (r->out) {
        if (r->written < r->cap)
            for (uint32_t a = 0; a < q->k; a++) r->out[r->written * q->k + a] = r->x[a];
        r->written++;
    }
}

/*
 * The extension sets of attribute A at level j: one per relation that
 * contains A (for tri atoms: A is the third attribute and the first two are
 * bound; with bound_only, edge atoms whose other attribute is bound). The
 * index of the smallest (ties: the first found, edge atoms before tri
 * atoms, each in definition order) goes to *imin; the work is counted.
 */
static uint32_t collect_sets(og_run* r, uint32_t j, uint32_t A, og_set* sets, uint32_t* imin) {
    const og_query* q = r->q;
    uint32_t nsets = 0;
    *imin = 0;
    for (uint32_t t = 0; t < q->natoms; t++) {
        if (r->v->view[t] == NULL) continue;            /* the Delta atom was consumed by the seed */
        if (q->as[t] != A && q->ad[t] != A) continue;   /* does not contain a_{j+1} */
        if (r->bound_only) {
            uint32_t B = (q->as[t] == A) ? q->ad[t] : q->as[t];
            if (r->pos[B] >= j) continue;                /* its other attribute is not bound yet */
        }
        sets[nsets] = ext_set(r, t, A, j);
        if (sets[nsets].len < sets[*imin].len) *imin = nsets;
        nsets++;
    }
    for (uint32_t t = 0; t < q->ntri; t++) {
        if (q->tc[t] != A) continue;
        sets[nsets] = tri_set(r, t);
        if (sets[nsets].len < sets[*imin].len) *imin = nsets;
        nsets++;
    }
    if (nsets && r->st) {
        r->st->extended[j]++;
        r->st->nbind_sum[j] += nsets;
        r->st->proposals[j] += (int64_t)sets[*imin].len;
    }
    return nsets;
}

/* Whether proposal e of sets[imin] is in every other set and meets the
 * inequalities with the bound attributes. */
static int keep_candidate(og_run* r, uint32_t j, uint32_t A, uint32_t e, const og_set* sets, uint32_t nsets,
                          uint32_t imin) {
    for (uint32_t s = 0; s < nsets; s++) {
        if (s == imin) continue;
        if (r->st) r->st->probes[j]++;
        if (!in_list(sets[s].a, sets[s].len, e)) return 0;
    }
    return lt_ok(r, A, e, j);
}

static void extend_factorised(og_run* r);

/*
 * Extend every prefix of length j (attributes order[0..j-1] bound) by
 * attribute order[j], as in Fig. 1: the relations that contain the new
 * attribute each give an extension set; the smallest one proposes (ties go
 * to the lowest atom index), and each proposal is kept only if it is a
 * member of every other set. Relations not yet joined at this level (none
 * of their attributes bound) do not constrain it.
 */
static void gj_extend(og_run* r, uint32_t j) {
    const og_query* q = r->q;
    if (r->st) r->st->prefixes[j]++;
    if (j == q->k) { emit(r); return; }
    if (j == r->fact_from) { extend_factorised(r); return; }
    uint32_t A = r->order[j];
    og_set sets[2 * OG_MAX_ATOMS];
    uint32_t imin = 0;
    uint32_t nsets = collect_sets(r, j, A, sets, &imin);
    if (nsets == 0) return;  /* cannot happen for a validated query */
    for (uint64_t c = 0; c < sets[imin].len; c++) {
        uint32_t e = sets[imin].a[c];
        if (j == 0 && (e < r->first_lo || e >= r->first_hi)) continue;
        if (!keep_candidate(r, j, A, e, sets, nsets, imin)) continue;
        r->x[A] = e;
        gj_extend(r, j + 1);
    }
}

/* The Cartesian product of the factorised extension sets, from position j. */
static void emit_product(og_run* r, uint32_t j, uint32_t* const* lists, const uint64_t* lens) {
    if (j > r->fact_from && r->st) r->st->prefixes[j]++;
    if (j == r->q->k) { emit(r); return; }
    for (uint64_t i = 0; i < lens[j]; i++) {
        r->x[r->order[j]] = lists[j][i];
        emit_product(r, j + 1, lists, lens);
    }
}

/*
 * Factorised output (Section 5.4, the house query): the attributes at
 * positions f..k-1 of the order are joined to one another by no atom and
 * no inequality, so each extends the prefix on its own. Their extension
 * sets are computed once for the prefix (the work counted once per
 * prefix), and the matches that extend it are their Cartesian product.
 */
static void extend_factorised(og_run* r) {
    const og_query* q = r->q;
    const uint32_t f = r->fact_from;
    uint32_t* lists[OG_MAX_K] = {0};
    uint64_t lens[OG_MAX_K] = {0};
    int ok = 1;
    for (uint32_t j = f; j < q->k && ok; j++) {
        uint32_t A = r->order[j];
        og_set sets[2 * OG_MAX_ATOMS];
        uint32_t imin = 0;
        uint32_t nsets = collect_sets(r, j, A, sets, &imin);
        if (nsets == 0) { ok = 0; break; }
        lists[j] = (uint32_t*)malloc(sizeof(uint32_t) * (sets[imin].len ? sets[imin].len : 1));
        if (!lists[j]) { ok = 0; break; }
        for (uint64_t c = 0; c < sets[imin].len; c++) {
            uint32_t e = sets[imin].a[c];
            if (keep_candidate(r, j, A, e, sets, nsets, imin)) lists[j][lens[j]++] = e;
        }
    }
    if (ok) emit_product(r, f, lists, lens);
    for (uint32_t j = f; j < q->k; j++) free(lists[j]);
}

/* Whether atom-or-inequality (u, v) joins position p to a position >= f. */
static int joins(const uint32_t* pos, uint32_t u, uint32_t v, uint32_t p, uint32_t f) {
    return (pos[u] == p && pos[v] >= f) || (pos[v] == p && pos[u] >= f);
}

/*
 * First position of the longest trailing run of at least two attributes of
 * the order that no atom (edge or tri) and no inequality joins to one
 * another; k if there is none. Positions 0 and 1 (the seed) never belong
 * to it.
 */
static uint32_t factor_start(const og_query* q, const uint32_t* pos) {
    uint32_t f = q->k;
    while (f > 2) {
        const uint32_t p = f - 1;
        int ok = 1;
        for (uint32_t t = 0; t < q->natoms && ok; t++)
            if (joins(pos, q->as[t], q->ad[t], p, f)) ok = 0;
        for (uint32_t t = 0; t < q->nlt && ok; t++)
            if (joins(pos, q->la[t], q->lb[t], p, f)) ok = 0;
        for (uint32_t t = 0; t < q->ntri && ok; t++)
            if (joins(pos, q->ta[t], q->tb[t], p, f) || joins(pos, q->ta[t], q->tc[t], p, f) ||
                joins(pos, q->tb[t], q->tc[t], p, f))
                ok = 0;
        if (!ok) break;
        f = p;
    }
    return (q->k - f >= 2) ? f : q->k;
}

static void run_init(og_run* r, const og_query* q, const og_views* v, const uint32_t* order) {
    memset(r, 0, sizeof(*r));
    r->q = q; r->v = v; r->sign = 1;
    for (uint32_t j = 0; j < q->k; j++) { r->order[j] = order[j]; r->pos[order[j]] = j; }
    r->first_lo = 0; r->first_hi = UINT32_MAX;
    r->fact_from = q->k;
}

/*
 * Static evaluation: count and checksum of Q over g.
 *
 * mode 0 follows Fig. 1 and Section 2.2 literally: GJ from P0 = {()}, every
 * relation containing the next attribute gives an extension set (its
 * projection when its other attribute is not bound yet), so P_j is exactly
 * the result of Q with every relation restricted to the first j attributes.
 * Queries with tri atoms are not accepted in mode 0.
 *
 * mode 1 follows the paper's implementation (Section 4.1, Section 4.2):
 * the length-2 prefixes are the edges of the first atom over the first two
 * attributes of the order (an edge atom, else a tri atom whose first two
 * attributes they are: its triangles lie on edges), kept if every other
 * edge atom and inequality over those two attributes holds, and a level is
 * bound only by the atoms whose other attributes are already bound. A tri
 * atom binds its third attribute, which must come after its first two in
 * the order. Both modes give the same matches; their intermediate prefix
 * sets differ. Mode 1 needs an order whose first two attributes share an
 * atom and whose later attributes each share an atom with earlier ones.
 *
 * mode 2 is mode 1 with factorised output (Section 5.4) for the trailing
 * attributes that constrain one another in no way (factor_start).
 *
 * Only matches whose first attribute (in execution order) lies in
 * [first_lo, first_hi) are counted; the count is additive over such ranges.
 * stats and out may be NULL. If out is given, up to cap tuples (query
 * attribute order) are written and *written receives the total.
 */
int og_count_ex(og_graph* g, uint32_t k, const uint32_t* atoms, uint32_t natoms, const uint32_t* tris,
                uint32_t ntri, const uint32_t* lts, uint32_t nlt, const uint32_t* order, uint32_t first_lo,
                uint32_t first_hi, int mode, int64_t* count, uint64_t* chk, og_stats* stats, uint32_t* out,
                uint64_t cap, uint64_t* written) {
    og_query q;
    int rc = make_query(k, atoms, natoms, tris, ntri, lts, nlt, order, &q);
    if (rc) return rc;
    if (mode < 0 || mode > 2 || (mode == 0 && ntri)) return OG_E_INVALID;
    if (ntri && (rc = build_tri(g)) != OG_OK) return rc;
    og_views v;
    for (uint32_t t = 0; t < q.natoms; t++) v.view[t] = g;
    og_run r;
    run_init(&r, &q, &v, q.order);
    r.g = g;
    r.first_lo = first_lo; r.first_hi = first_hi;
    r.st = stats;
    if (stats) memset(stats, 0, sizeof(*stats));
    r.out = out; r.cap = cap;
    if (mode == 0) {
        gj_extend(&r, 0);
    } else {
        /* seed: the first edge atom over the first two attributes of the order, else the
         * first tri atom whose first two attributes they are; (sa, sd) = (source, target) */
        uint32_t a0 = q.order[0], a1 = q.order[1];
        int seed = -1;
        uint32_t sa = 0, sd = 0;
        for (uint32_t t = 0; t < q.natoms && seed < 0; t++)
            if ((q.as[t] == a0 && q.ad[t] == a1) || (q.as[t] == a1 && q.ad[t] == a0)) { seed = (int)t; sa = q.as[t]; sd = q.ad[t]; }
        for (uint32_t t = 0; t < q.ntri && seed < 0; t++)
            if ((q.ta[t] == a0 && q.tb[t] == a1) || (q.ta[t] == a1 && q.tb[t] == a0)) { seed = OG_MAX_ATOMS + (int)t; sa = q.ta[t]; sd = q.tb[t]; }
        if (seed < 0) return OG_E_INVALID;
        for (uint32_t t = 0; t < q.ntri; t++)
            if (r.pos[q.tc[t]] < r.pos[q.ta[t]] || r.pos[q.tc[t]] < r.pos[q.tb[t]]) return OG_E_INVALID;
        for (uint32_t j = 2; j < q.k; j++) {
            int ok = 0;
            for (uint32_t t = 0; t < q.natoms; t++) {
                uint32_t ps = r.pos[q.as[t]], pd = r.pos[q.ad[t]];
                if ((ps == j && pd < j) || (pd == j && ps < j)) ok = 1;
            }
            for (uint32_t t = 0; t < q.ntri; t++)
                if (r.pos[q.tc[t]] == j) ok = 1;
            if (!ok) return OG_E_INVALID;
        }
        r.bound_only = 1;
        if (mode == 2) r.fact_from = factor_start(&q, r.pos);
        for (uint32_t u = 0; u < g->n; u++) {
            for (uint64_t e = g->fo[u]; e < g->fo[u + 1]; e++) {
                uint32_t w = g->fn[e];
                r.x[sa] = u;
                r.x[sd] = w;
                if (r.x[a0] < first_lo || r.x[a0] >= first_hi) continue;
                int ok = 1;
                for (uint32_t t = 0; t < q.natoms && ok; t++) {
                    if ((int)t == seed) continue;
                    uint32_t ps = r.pos[q.as[t]], pd = r.pos[q.ad[t]];
                    if (ps <= 1 && pd <= 1) ok = has_edge(g, r.x[q.as[t]], r.x[q.ad[t]]);
                }
                for (uint32_t t = 0; t < q.nlt && ok; t++)
                    if (r.pos[q.la[t]] <= 1 && r.pos[q.lb[t]] <= 1) ok = r.x[q.la[t]] < r.x[q.lb[t]];
                if (ok) gj_extend(&r, 2);
            }
        }
    }
    *count = r.count;
    *chk = r.chk;
    if (written) *written = r.written;
    return (out && r.written > cap) ? OG_E_TRUNCATED : OG_OK;
}

/* og_count_ex for queries of edge atoms only. */
int og_count(og_graph* g, uint32_t k, const uint32_t* atoms, uint32_t natoms, const uint32_t* order,
             uint32_t first_lo, uint32_t first_hi, int mode, int64_t* count, uint64_t* chk, og_stats* stats,
             uint32_t* out, uint64_t cap, uint64_t* written) {
    return og_count_ex(g, k, atoms, natoms, NULL, 0, NULL, 0, order, first_lo, first_hi, mode, count, chk, stats,
                       out, cap, written);
}

/*
 * Symmetry breaking's input transformation (Section 5.4): optionally adds
 * the reverse of every edge (the undirected graph), optionally gives the
 * vertices new ids that ascend with degree (out-degree after the optional
 * symmetrisation, ties broken by the old id), and optionally keeps only
 * the edges that point from a lower to a higher new id. new_of_old[v]
 * receives v's new id (v itself without renaming). NULL on failure.
 */
og_graph* og_graph_transform(const og_graph* g, int symmetrize, int degree_order, int orient, uint32_t* new_of_old,
                             int* err) {
    const uint64_t m2 = symmetrize ? 2 * g->m : g->m;
    uint32_t* s = (uint32_t*)malloc(sizeof(uint32_t) * (m2 ? m2 : 1));
    uint32_t* d = (uint32_t*)malloc(sizeof(uint32_t) * (m2 ? m2 : 1));
    uint64_t* key = (uint64_t*)malloc(sizeof(uint64_t) * ((size_t)g->n + 1));
    if (!s || !d || !key) { free(s); free(d); free(key); *err = OG_E_NOMEM; return NULL; }
    og_graph_edges(g, s, d);
    if (symmetrize)
        for (uint64_t i = 0; i < g->m; i++) { s[g->m + i] = d[i]; d[g->m + i] = s[i]; }
    og_graph* h = og_graph_new(g->n, s, d, m2, err);
    if (!h) { free(s); free(d); free(key); return NULL; }
    /* rank by (degree, old id): the position of (deg << 32 | v) in ascending order */
    for (uint32_t v = 0; v < g->n; v++)
        key[v] = degree_order ? (((uint64_t)(h->fo[v + 1] - h->fo[v]) << 32) | v) : (uint64_t)v;
    qsort(key, g->n, sizeof(uint64_t), cmp_u64);
    for (uint32_t i = 0; i < g->n; i++) new_of_old[(uint32_t)key[i]] = i;
    uint64_t mk = 0;
    og_graph_edges(h, s, d);
    for (uint64_t i = 0; i < h->m; i++) {
        uint32_t u = new_of_old[s[i]], w = new_of_old[d[i]];
        if (orient && !(u < w)) continue;
        s[mk] = u; d[mk] = w; mk++;
    }
    og_graph* out = og_graph_new(g->n, s, d, mk, err);
    og_graph_free(h);
    free(s); free(d); free(key);
    return out;
}

/* ------------------------------------------------------------- updates */

typedef struct { uint64_t key; uint64_t idx; int8_t sign; } og_upd;

static int cmp_upd(const void* a, const void* b) {
    const og_upd* x = (const og_upd*)a; const og_upd* y = (const og_upd*)b;
    if (x->key != y->key) return (x->key > y->key) - (x->key < y->key);
    return (x->idx > y->idx) - (x->idx < y->idx);
}

/*
 * Normalises a batch of signed edge updates against g under the set
 * semantics R' = R + Delta R of Section 3.3.1: updates apply in batch
 * order, so the last update of an edge decides whether it is present
 * afterwards; self-loops are dropped; an edge's change is +1 if it was
 * absent and ends present, -1 if it was present and ends absent, and it is
 * dropped otherwise. Writes the changes sorted by (src, dst) and returns
 * their number, or OG_E_RANGE / OG_E_INVALID (sign not +-1) / OG_E_NOMEM.
 */
int64_t og_normalize(const og_graph* g, const uint32_t* src, const uint32_t* dst, const int8_t* sign, uint64_t b,
                     uint32_t* osrc, uint32_t* odst, int8_t* osign) {
    og_upd* u = (og_upd*)malloc(sizeof(og_upd) * (b ? b : 1));
    if (!u) return OG_E_NOMEM;
    uint64_t c = 0;
    for (uint64_t i = 0; i < b; i++) {
        if (src[i] >= g->n || dst[i] >= g->n) { free(u); return OG_E_RANGE; }
        if (sign[i] != 1 && sign[i] != -1) { free(u); return OG_E_INVALID; }
        if (src[i] == dst[i]) continue;
        u[c].key = ((uint64_t)src[i] << 32) | dst[i]; u[c].idx = i; u[c].sign = sign[i]; c++;
    }
    qsort(u, c, sizeof(og_upd), cmp_upd);
    int64_t nout = 0;
    for (uint64_t i = 0; i < c; i++) {
        if (i + 1 < c && u[i + 1].key == u[i].key) continue;  /* a later update of this edge decides */
        uint32_t s = (uint32_t)(u[i].key >> 32), d = (uint32_t)u[i].key;
        int present = has_edge(g, s, d);
        if ((u[i].sign > 0) == present) continue;              /* no change */
        osrc[nout] = s; odst[nout] = d; osign[nout] = u[i].sign; nout++;
    }
    free(u);
    return nout;
}

/* The graph after applying normalised changes (R' = R + Delta R). */
og_graph* og_graph_apply(const og_graph* g, const uint32_t* dsrc, const uint32_t* ddst, const int8_t* dsign,
                         uint64_t nd, int* err) {
    uint64_t cap = g->m + nd;
    uint32_t* s = (uint32_t*)malloc(sizeof(uint32_t) * (cap ? cap : 1));
    uint32_t* d = (uint32_t*)malloc(sizeof(uint32_t) * (cap ? cap : 1));
    if (!s || !d) { free(s); free(d); *err = OG_E_NOMEM; return NULL; }
    uint8_t* gone = (uint8_t*)calloc(g->m ? g->m : 1, 1);
    if (!gone) { free(s); free(d); *err = OG_E_NOMEM; return NULL; }
    og_graph_edges(g, s, d);
    /* find each deleted edge in the (sorted) edge list and flag it */
    for (uint64_t i = 0; i < nd; i++) {
        if (dsign[i] > 0) continue;
        uint32_t u = dsrc[i];
        uint64_t lo = g->fo[u], hi = g->fo[u + 1];
        while (lo < hi) { uint64_t mid = lo + (hi - lo) / 2; if (d[mid] < ddst[i]) lo = mid + 1; else hi = mid; }
        if (lo < g->fo[u + 1] && d[lo] == ddst[i]) gone[lo] = 1;
    }
    uint64_t m = 0;
    for (uint64_t i = 0; i < g->m; i++)
        if (!gone[i]) { s[m] = s[i]; d[m] = d[i]; m++; }
    free(gone);
    for (uint64_t i = 0; i < nd; i++)
        if (dsign[i] > 0) { s[m] = dsrc[i]; d[m] = ddst[i]; m++; }
    og_graph* out = og_graph_new(g->n, s, d, m, err);
    free(s); free(d);
    return out;
}

/*
 * Delta-GJ (Section 3.3.1): the change of Q's matches caused by the
 * normalised changes Delta (dsrc, ddst, dsign) that turn g_old into g_new,
 * as the sum of the delta queries
 *     dQ_i := R'_1, ..., R'_{i-1}, Delta R_i, R_{i+1}, ..., R_n
 * with atoms numbered in query definition order. Each dQ_i runs GJ with an
 * attribute order that starts with the attributes of atom i (source, then
 * destination) followed by the remaining attributes in the query's order
 * (or in ascending attribute id when order is NULL), seeded from each
 * signed change; every match counts with its seed's sign. each_count and
 * each_chk (may be NULL) receive the result of each dQ_i, i = 0..natoms-1.
 */
int og_delta_each(const og_graph* g_old, const og_graph* g_new, const uint32_t* dsrc, const uint32_t* ddst,
                  const int8_t* dsign, uint64_t nd, uint32_t k, const uint32_t* atoms, uint32_t natoms,
                  const uint32_t* order, int64_t* dcount, uint64_t* dchk, int64_t* each_count,
                  uint64_t* each_chk) {
    og_query q;
    int rc = make_query(k, atoms, natoms, NULL, 0, NULL, 0, order, &q);
    if (rc) return rc;
    int64_t total = 0;
    uint64_t tchk = 0;
    for (uint32_t i = 0; i < q.natoms; i++) {
        og_views v;
        for (uint32_t t = 0; t < q.natoms; t++) v.view[t] = (t < i) ? g_new : (t > i ? g_old : NULL);
        uint32_t ord[OG_MAX_K], n = 0;
        ord[n++] = q.as[i];
        ord[n++] = q.ad[i];
        for (uint32_t j = 0; j < q.k; j++)
            if (q.order[j] != q.as[i] && q.order[j] != q.ad[i]) ord[n++] = q.order[j];
        og_run r;
        run_init(&r, &q, &v, ord);
        for (uint64_t c = 0; c < nd; c++) {
            r.x[q.as[i]] = dsrc[c];
            r.x[q.ad[i]] = ddst[c];
            r.sign = dsign[c];
            /* the remaining atoms over the same two attributes filter the seed in their own versions */
            int ok = 1;
            for (uint32_t t = 0; t < q.natoms && ok; t++) {
                if (t == i) continue;
                uint32_t s = q.as[t], d = q.ad[t];
                if ((s == q.as[i] || s == q.ad[i]) && (d == q.as[i] || d == q.ad[i]))
                    ok = has_edge(v.view[t], r.x[s], r.x[d]);
            }
            if (ok) gj_extend(&r, 2);
        }
        if (each_count) each_count[i] = r.count;
        if (each_chk) each_chk[i] = r.chk;
        total += r.count;
        tchk += r.chk;
    }
    *dcount = total;
    *dchk = tchk;
    return OG_OK;
}

/* The sum of the delta queries only (og_delta_each without the parts). */
int og_delta(const og_graph* g_old, const og_graph* g_new, const uint32_t* dsrc, const uint32_t* ddst,
             const int8_t* dsign, uint64_t nd, uint32_t k, const uint32_t* atoms, uint32_t natoms,
             const uint32_t* order, int64_t* dcount, uint64_t* dchk) {
    return og_delta_each(g_old, g_new, dsrc, ddst, dsign, nd, k, atoms, natoms, order, dcount, dchk, NULL, NULL);
}
