/*
 * gj.h -- C ABI of libgj, a single-GPU (B300, sm_103a) implementation of the
 * worst-case optimal Generic Join prefix-extension step and its delta-query
 * form, after "Distributed Evaluation of Subgraph Queries Using Worst-case
 * Optimal Low-Memory Dataflows" (Ammar, McSherry, Salihoglu, Joglekar).
 *
 * Problem statement (Section 1, Section 2.1): a subgraph query over a
 * directed graph is a multiway self-join of the edge relation,
 *     Q(a_0, ..., a_{k-1}) := E(a_s1, a_d1), ..., E(a_sn, a_dn),
 * evaluated under join (homomorphism) semantics: a match is any assignment
 * of vertex ids to the attributes such that every atom is an edge. Generic
 * Join (Fig. 1, Section 2.2) fixes a global attribute order and extends
 * prefixes one attribute at a time: for each prefix, every atom binding the
 * next attribute gives an extension set (count), the smallest set proposes
 * candidates (propose), and each candidate is kept only if it is in all the
 * other sets (intersect).
 *
 * Conventions for every call:
 *   - Return value: GJ_OK (0) or a negative GJ_E_* code; gj_strerror() names
 *     it and gj_last_error() gives the context's last message. On error no
 *     output argument is written unless stated.
 *   - Vertex ids are uint32 in [0, num_vertices). Match counts are exact
 *     int64; checksums are uint64 sums modulo 2^64.
 *   - Input arrays are owned by the caller and are copied (or fully
 *     consumed) before the call returns; they may be host or device
 *     pointers (the library asks the CUDA runtime which). Output arrays are
 *     owned by the caller and must be host memory.
 *   - Handles (gj_ctx, gj_graph, gj_query) are owned by the library and
 *     released by their *_free / gj_destroy call; free a context's graphs
 *     and queries before destroying the context.
 *   - A context and the graphs and queries made from it are used by one host
 *     thread at a time.
 *
 * Match checksum (not from the paper; fixed by this library so that listed
 * matches can be compared without sorting): H(x) = q(k) * f_0(x_0) * ... *
 * f_{k-1}(x_{k-1}) modulo 2^64, x_a the value of query attribute a, with
 * f_a(v) = m(v ^ s_a) | 1, q(k) = m(k) | 1, s_a = (a + 1) *
 * 0x9e3779b97f4a7c15 and m the SplitMix64 output function (Steele, Lea,
 * Flood, OOPSLA 2014); the checksum of a set of matches is the sum of H over
 * it modulo 2^64. All factors are odd (units modulo 2^64), and the sum over
 * matches that share some attributes factorises, so factorised output
 * (Section 5.4) is checked without listing its matches. Delta checksums add
 * H for gained matches and subtract it for lost ones.
 */
#ifndef GJ_H
#define GJ_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    GJ_OK = 0,
    GJ_E_INVALID = -1,    /* null pointer, malformed query, bad sign, bad option */
    GJ_E_RANGE = -2,      /* vertex id >= num_vertices */
    GJ_E_NOMEM = -3,      /* device or host allocation failed */
    GJ_E_ADMIT = -4,      /* request needs more device memory than the budget allows */
    GJ_E_TRUNCATED = -5,  /* more matches than the output capacity */
    GJ_E_TIMEOUT = -6,    /* a bounded wait expired */
    GJ_E_OVERFLOW = -7,   /* a match count passed 2^63 - 1 (the int64 result would wrap) */
    GJ_E_CUDA = -8,       /* a CUDA runtime call failed (gj_last_error has the text) */
    GJ_E_PENDING = -9,    /* request not finished yet */
    GJ_E_NOTFOUND = -10,  /* unknown request id */
    GJ_E_CHECK = -11,     /* checked build only: a device bounds check failed (gj_last_error names it) */
    GJ_E_CANCELLED = -12  /* the request was withdrawn by gj_cancel before it started */
};

typedef struct gj_ctx gj_ctx;
typedef struct gj_graph gj_graph;
typedef struct gj_query gj_query;

/* Engines for gj_count_ex / gj_count_many. */
enum {
    /* Level-synchronous evaluation: separate count, scan, propose+intersect
     * kernels per level over bounded prefix buffers, the host choosing the
     * deepest level with pending work after every launch (Section 3.1.1,
     * Section 3.2; the "plain" one-query-at-a-time path). */
    GJ_ENGINE_PLAIN = 0,
    /* One fused launch per call: each warp extends a bounded batch of
     * prefixes depth-first through all levels (the batching rule of
     * Section 3.1.2 with B' = one warp's batch), warps take seed ranges from
     * a shared work counter. */
    GJ_ENGINE_FUSED = 1
};

/* Option flags for the delta queries of update batches. By default a batch
 * of fewer than 8192 normalised changes runs on the level-synchronous
 * engine (which spreads a small batch's fan-out over the whole GPU at once)
 * and a larger one on the fused engine (which balances its work by
 * donation). GJ_FLAG_DELTA_FUSED / GJ_FLAG_DELTA_PLAIN force one of them. */
enum { GJ_FLAG_DELTA_FUSED = 1, GJ_FLAG_DELTA_PLAIN = 2 };

typedef struct {
    uint64_t prefix_buffer_bytes; /* cap on device prefix buffers of one evaluation; 0 = 512 MiB */
    uint64_t window;              /* plain engine: candidates per propose+intersect launch; 0 = from the cap */
    uint32_t engine;              /* default engine of gj_count (GJ_ENGINE_*) */
    uint32_t flags;               /* GJ_FLAG_* */
    void* stream;                 /* cudaStream_t for all launches; NULL = the context creates one */
} gj_options;

/* Units of work of the last gj_count_ex / gj_count_many call on a context,
 * in the terms of the cost model of Section 2.2 and Theorem 2.1. Index j is
 * a prefix length; entries j < 2 are zero because evaluation starts from
 * the length-2 prefixes read off the edges (Section 4.2). */
typedef struct {
    int64_t seeds;                /* seed edges read */
    int64_t extended[9];          /* prefixes of length j that were extended */
    int64_t nbind[9];             /* sum over those of the number of binding atoms */
    int64_t proposals[9];         /* sum over those of the smallest extension-set size */
    int64_t produced[9];          /* prefixes of length j produced (j = k: matches) */
} gj_work_stats;

/* Creates a context on CUDA device `cuda_device`. opt may be NULL
 * (defaults). Errors: GJ_E_INVALID (negative or out-of-range device index,
 * bad engine), GJ_E_CUDA (no usable CUDA driver or device; a failed set-up). */
int gj_create(int cuda_device, const gj_options* opt, gj_ctx** out);
/* Stops a request loop on ctx, waits for its stream and frees its memory
 * and (if the context created it) its stream. ctx's graphs and queries must
 * be freed first. NULL is ignored. */
void gj_destroy(gj_ctx* ctx);
/* A static English name of an error code ("unknown error" for others). */
const char* gj_strerror(int code);
/* Last error message recorded on ctx (empty string if none); valid until the next call. */
const char* gj_last_error(const gj_ctx* ctx);

/*
 * Loads the edge relation E from m pairs (src[i], dst[i]) on vertices
 * [0, num_vertices), host or device arrays. Self-loops are dropped and
 * duplicate pairs collapse (E is a set, Section 2.1). Builds, on the
 * device, the forward index (out-neighbours of each vertex, sorted) and
 * the reverse index (in-neighbours, sorted), the only two indices every
 * atom shares (Section 4.1). Errors: GJ_E_INVALID (null pointer with m >
 * 0, num_vertices == 0 or > 2^32 - 1), GJ_E_RANGE, GJ_E_NOMEM, GJ_E_CUDA.
 */
int gj_graph_load(gj_ctx* ctx, const uint32_t* src, const uint32_t* dst, uint64_t m, uint32_t num_vertices,
                  gj_graph** out);
/* Flags of gj_graph_load_ex: the input transformation of symmetry breaking
 * (Section 5.4). GJ_LOAD_SYMMETRIZE adds the reverse of every edge (the
 * undirected graph). GJ_LOAD_DEGREE_ORDER gives the vertices new ids that
 * ascend with their out-degree (after the optional symmetrisation; ties
 * keep the order of the old ids); the indices, queries and results then
 * use the new ids (gj_graph_relabel_map gives them). GJ_LOAD_ORIENT keeps
 * only the edges from a lower to a higher (new) id, so that a clique query
 * with atoms E(a_i, a_j), i < j, finds each undirected clique once. */
enum { GJ_LOAD_SYMMETRIZE = 1, GJ_LOAD_DEGREE_ORDER = 2, GJ_LOAD_ORIENT = 4 };
/* gj_graph_load with the GJ_LOAD_* flags above (0: gj_graph_load). Host
 * or device arrays; device arrays must be on the context's device and
 * complete (written by work that has finished, or is ordered before the
 * context's stream). Errors: as gj_graph_load, and GJ_E_INVALID (unknown
 * flag, an array in another device's memory). */
int gj_graph_load_ex(gj_ctx* ctx, const uint32_t* src, const uint32_t* dst, uint64_t m, uint32_t num_vertices,
                     uint32_t flags, gj_graph** out);
/* new_of_old[v] = the id that input vertex v has in g's indices (v itself
 * unless g was loaded with GJ_LOAD_DEGREE_ORDER); host array of
 * num_vertices. Errors: GJ_E_INVALID, GJ_E_CUDA. */
int gj_graph_relabel_map(const gj_graph* g, uint32_t* new_of_old);
/*
 * Builds g's triangle index, the ternary relation tri(a, b, c) of triangle
 * indexing (Section 5.4): the tuples with a -> b, a -> c and b -> c, indexed
 * by (a, b), i.e. for every edge a -> b the sorted list of the c that
 * complete a triangle on it. Queries with tri atoms read it; counting such
 * a query builds it when it is missing, and applying an update batch drops
 * it (it describes one version of the graph). *count (may be NULL) receives
 * the number of tuples. Errors: GJ_E_INVALID (null g, serving), GJ_E_NOMEM,
 * GJ_E_CUDA.
 */
int gj_graph_build_triangles(gj_graph* g, uint64_t* count);
/* Number of distinct edges and the committed version (0 after load, +1 per applied batch). */
int gj_graph_stats(const gj_graph* g, uint64_t* num_edges, uint64_t* version);
/* Copies the forward index to host arrays: offsets [num_vertices + 1], neighbours [num_edges]. */
int gj_graph_export(const gj_graph* g, int64_t* offsets, uint32_t* neighbours);
/* Stops a request loop serving g, waits for the context's stream and frees
 * g's device indices. NULL is ignored. */
void gj_graph_free(gj_graph* g);

/*
 * Defines Q(a_0..a_{k-1}) := E(a_atoms[0], a_atoms[1]), E(a_atoms[2],
 * a_atoms[3]), ... with n_atoms atoms, and the global attribute order
 * `order` (k attribute ids; NULL = 0, 1, ..., k-1). Evaluation starts from
 * the edges of an atom over the first two attributes of the order, as the
 * paper's implementation does (Section 4.2), so those two attributes must
 * share an atom, and every later attribute must share an atom with an
 * earlier one. Errors: GJ_E_INVALID (k < 2 or > 8, n_atoms > 16, an atom
 * with equal or out-of-range attributes, order not a permutation, an
 * attribute in no atom, or the connectivity rule above broken).
 */
int gj_query_define(gj_ctx* ctx, uint32_t k, const uint32_t* atoms, uint32_t n_atoms, const uint32_t* order,
                    gj_query** out);
/*
 * gj_query_define with the specialisations of Section 5.4. tri_atoms holds
 * n_tri triples (i, j, l): the atom tri(a_i, a_j, a_l) holds when a_i ->
 * a_j, a_i -> a_l and a_j -> a_l are edges (the triangle index, indexed by
 * (a_i, a_j)); a_l must come after a_i and a_j in the order, and a tri atom
 * whose first two attributes are the first two of the order can seed the
 * evaluation (every edge between them is a seed). lt_pairs holds n_lt pairs
 * (a, b): matches must have x_a < x_b (vertex ids; symmetry breaking).
 * atoms may be NULL when n_atoms is 0. Queries with tri atoms cannot be
 * used in update batches or serving requests (GJ_E_INVALID there). When the
 * last attributes of the order do not depend on every earlier one (for
 * example the diamond in order a2, a3, a1, a4, or the house query of
 * Section 5.4), the fused engine extends prefixes that agree on what the
 * last level reads once for all of them (aggregation of identical lookups,
 * Section 3.4.2) and hashes the matches of each. Errors: as
 * gj_query_define, and a tri atom or inequality with equal or out-of-range
 * attributes, or a tri atom whose third attribute comes too early.
 */
int gj_query_define_ex(gj_ctx* ctx, uint32_t k, const uint32_t* atoms, uint32_t n_atoms, const uint32_t* tri_atoms,
                       uint32_t n_tri, const uint32_t* lt_pairs, uint32_t n_lt, const uint32_t* order,
                       gj_query** out);
/* Frees q (host memory only). A query passed to a serving request must stay
 * alive until that request is polled. NULL is ignored. */
void gj_query_free(gj_query* q);

/* Count and checksum of the matches of q in the committed graph, default engine.
 * GJ_E_TIMEOUT: a bounded wait of the fused engine's work queue expired
 * (the result is not reported). */
int gj_count(gj_graph* g, const gj_query* q, int64_t* count, uint64_t* checksum);

/*
 * As gj_count with an explicit engine, restricted to the matches whose first
 * attribute in the global order has a value in [v_lo, v_hi) (the counts of
 * disjoint ranges add up). stats may be NULL. Errors: GJ_E_INVALID,
 * GJ_E_NOMEM, GJ_E_CUDA.
 */
int gj_count_ex(gj_graph* g, const gj_query* q, uint32_t engine, uint32_t v_lo, uint32_t v_hi, int64_t* count,
                uint64_t* checksum, gj_work_stats* stats);

/*
 * Counts nq queries over the committed graph. With GJ_ENGINE_FUSED all of
 * them run in one persistent launch whose warps share one seed counter (the
 * batched path); with GJ_ENGINE_PLAIN they run one after another. counts
 * and checksums are host arrays of nq. Errors: GJ_E_INVALID, GJ_E_NOMEM,
 * GJ_E_CUDA.
 */
int gj_count_many(gj_graph* g, const gj_query* const* qs, uint32_t nq, uint32_t engine, int64_t* counts,
                  uint64_t* checksums);

/*
 * gj_count_many with the fused engine, for callers that must not allocate
 * device memory during the call: for example a host application whose
 * device memory is entirely owned by another framework's pool, or a
 * latency-critical loop where cudaMalloc/cudaFree would stall other streams
 * by synchronizing the device. The paper has no counterpart; this is an
 * interface convenience of this library.
 *
 * g and the queries are created beforehand (gj_graph_load allocates); the
 * call itself allocates nothing. Its scratch (plans, seed ranges, counters)
 * is one 64 KiB array in the library's device memory, resident on every GPU
 * that loads the library until the process exits. The first call on a
 * device looks up that array's address (cudaGetSymbolAddress) and caches
 * it, so make the first call on each device before any stream capture.
 * Every call on a device shares the array: calls that overlap on the GPU
 * (from different contexts or streams) race and give wrong counts. At most
 * 64 queries per call (GJ_E_INVALID above that, with a message in
 * gj_last_error). counts and checksums are host arrays of nq. Errors:
 * GJ_E_INVALID, GJ_E_CUDA.
 */
int gj_count_noalloc(gj_graph* g, const gj_query* const* qs, uint32_t nq, int64_t* counts, uint64_t* checksums);

/* gj_count_many restricted to matches whose first attribute (in each
 * query's global order) lies in [v_lo, v_hi). */
int gj_count_many_ex(gj_graph* g, const gj_query* const* qs, uint32_t nq, uint32_t engine, uint32_t v_lo,
                     uint32_t v_hi, int64_t* counts, uint64_t* checksums);

/* Launch settings of a context. */
typedef struct {
    uint32_t seed_chunk;           /* fused engine: seeds a warp takes per grab (8..4096, multiple of 8;
                                    * delta launches take at most 8) */
    uint32_t blocks_per_sm;        /* fused engine: resident blocks per SM, 0 = as many as fit */
    uint64_t prefix_buffer_bytes;  /* level-synchronous engine: prefix-buffer budget, 0 = 512 MiB */
    double fused_ms, plain_ms;     /* gj_autotune: the sample's time with the chosen settings */
    /* fused engine work donation (the balance step of Section 3.4 at warp
     * granularity): a warp about to extend a batch of >= 32 new prefixes
     * hands it to a queue that idle warps take from. 0: only while some warp
     * is idle (default), 1: whenever a queue slot is free (stress setting),
     * 2: off. Results never depend on it. */
    uint32_t donation;
    /* The fused engine's end-of-launch wait (warps without work waiting for
     * donations until no warp holds work) gives up with GJ_E_TIMEOUT once the
     * donation queue has shown no progress for wait_ms milliseconds; 0 =
     * 10000. Working warps interact with the queue at least every ~1000
     * candidates, so the bound only ends waits that cannot end otherwise. */
    uint32_t wait_ms;
    /* Failure injection for tests; 0 = off. 1: the end-of-launch wait counts
     * a working warp that never finishes, so it can only end by its time bound
     * (the count call returns GJ_E_TIMEOUT; the context stays usable). 2: the
     * fused engine's per-query counts start at 2^63 - 1024, so a query with
     * more than 1023 matches returns GJ_E_OVERFLOW. 3 (checked build only,
     * GJ_E_INVALID otherwise): the graph views the kernels get claim one
     * vertex fewer than the graph has, so the first access to the last
     * vertex's lists trips a bounds check and the call returns GJ_E_CHECK.
     * 4: the library's device allocations after the first fault_count
     * (counted from this setting) fail as if the device were out of memory:
     * the call returns GJ_E_NOMEM and leaves the graph as it was (a failed
     * load creates no graph, a failed update batch commits nothing). */
    uint32_t fault;
    uint32_t fault_count;
} gj_tuning;
/* Copies the context's current settings to *out (fused_ms and plain_ms are
 * 0: only gj_autotune's output carries them). Errors: GJ_E_INVALID (null pointer). */
int gj_get_tuning(const gj_ctx* ctx, gj_tuning* out);
/* Replaces the context's settings (fused_ms and plain_ms are ignored); results
 * never depend on them (except for the failure-injection field). Errors:
 * GJ_E_INVALID (seed_chunk out of range or not a multiple of 8, budget under
 * 1 MiB, donation > 2, fault > 4). */
int gj_set_tuning(gj_ctx* ctx, const gj_tuning* t);
/*
 * Chooses the context's launch settings by timing the given queries on the
 * first-attribute range [v_lo, v_hi) of g (a sample of the workload): seeds
 * per grab in {8, 32, 128} x {all, all but one} resident blocks per SM
 * x donation when warps idle or whenever a queue slot is free for the fused
 * engine, and a prefix-buffer budget in {64 MiB, 256 MiB,
 * 1 GiB, 2 GiB} up to prefix_cap_bytes (0 = 2 GiB) for the level-synchronous
 * engine (the memory/runtime trade-off of the paper's batch size). Applies
 * the fastest settings to g's context and returns them. Errors:
 * GJ_E_INVALID (null pointer, nq == 0, serving), and any error of the timed
 * counts; on an error the context keeps its previous settings.
 */
int gj_autotune(gj_graph* g, const gj_query* const* qs, uint32_t nq, uint64_t prefix_cap_bytes, uint32_t v_lo,
                uint32_t v_hi, gj_tuning* out);

/* Work units of the last gj_count, gj_count_ex or gj_count_many call on ctx
 * (summed over queries). */
int gj_last_work(const gj_ctx* ctx, gj_work_stats* out);

/*
 * Lists matches: writes up to cap tuples (k uint32 each, query attribute
 * order, in no particular tuple order) to host memory out_tuples, the
 * number written to *written, the total to *total and the checksum of all
 * matches to *checksum. Returns GJ_E_TRUNCATED (outputs still written) if
 * total > cap.
 */
int gj_list(gj_graph* g, const gj_query* q, uint32_t* out_tuples, uint64_t cap, uint64_t* written, int64_t* total,
            uint64_t* checksum);

/*
 * Applies a batch of b signed edge updates (src[i], dst[i], sign[i] = +1
 * insert / -1 delete; host or device arrays) to g and returns, for each of
 * the nq queries, the change of its match count and checksum (host arrays
 * delta_count[nq], delta_checksum[nq]; checksums add H of gained matches
 * and subtract H of lost ones, mod 2^64).
 *
 * Batch semantics (R' = R + Delta R, Section 3.3.1): updates apply in batch
 * order, so the last update of an edge decides whether it is present
 * afterwards; self-loops are ignored; an insert of a present edge or a
 * delete of an absent one changes nothing. The change is computed with the
 * delta queries dQ_1..dQ_n of Delta-GJ (Section 3.3.1): dQ_i is seeded from
 * the changed edges under atom i, atoms before i (definition order) read
 * the new graph and atoms after i the old one (Section 4.3), and the signed
 * sum over all dQ_i is exactly count(after) - count(before). The batch is
 * then committed: the version advances and later counts see it. On error
 * the graph is unchanged. Errors: GJ_E_INVALID (null pointer, sign not +-1,
 * b >= 2^32), GJ_E_RANGE, GJ_E_NOMEM, GJ_E_CUDA.
 */
int gj_apply_batch(gj_graph* g, const uint32_t* src, const uint32_t* dst, const int8_t* sign, uint64_t b,
                   const gj_query* const* qs, uint32_t nq, int64_t* delta_count, uint64_t* delta_checksum);
/* Number of edges whose presence the last gj_apply_batch on g changed. */
int gj_graph_last_batch(const gj_graph* g, uint64_t* changes);

/* ------------------------------------------------------------------ serving
 *
 * A request loop on one graph: count requests and update batches are
 * submitted from any thread and run in submission order, each seeing the
 * graph versions it would see if the requests ran one by one. Count
 * requests that are queued together run as one fused launch (continuous
 * batching); an update batch overlaps with count launches already running,
 * which keep reading the previous version of the index. Requests are
 * admitted against a device-memory budget. While serving, use only
 * gj_submit_count, gj_submit_batch, gj_poll and gj_serve_stop on the
 * context; other calls on it return GJ_E_INVALID. Queries passed to a
 * request must stay alive until the request is polled. Each count launch
 * (a wave) balances its warps through a work-donation queue of its own, set
 * by the context's donation and wait_ms settings at the time of the launch.
 */
typedef struct {
    uint64_t req_id;
    int32_t status;          /* GJ_OK, or the request's own error: GJ_E_ADMIT, GJ_E_OVERFLOW (a
                              * count of its wave passed 2^63 - 1), GJ_E_TIMEOUT (its wave's
                              * bounded donation wait expired), GJ_E_CUDA */
    uint32_t kind;           /* 0 = count request, 1 = update batch */
    uint32_t nq;
    uint32_t reserved;
    int64_t counts[64];      /* count request: counts; batch: delta counts */
    uint64_t checksums[64];  /* count request: checksums; batch: delta checksums */
    uint64_t version;        /* count: the version it read; batch: the version it committed */
    double submit_ms, start_ms, end_ms;  /* host times since gj_serve_start */
} gj_result;

/* Starts the request loop on g. memory_budget_bytes = 0: 80% of the free
 * device memory. Errors: GJ_E_INVALID (already serving), GJ_E_CUDA. */
int gj_serve_start(gj_ctx* ctx, gj_graph* g, uint64_t memory_budget_bytes);
/* Finishes every submitted request, then stops the loop. */
int gj_serve_stop(gj_ctx* ctx);
/* Queues a count of nq <= 64 queries; *req_id identifies it for gj_poll. */
int gj_submit_count(gj_ctx* ctx, const gj_query* const* qs, uint32_t nq, uint64_t* req_id);
/* Queues an update batch (copied before return; host or device arrays) and
 * the nq <= 64 queries whose deltas it reports (see gj_apply_batch). */
int gj_submit_batch(gj_ctx* ctx, const uint32_t* src, const uint32_t* dst, const int8_t* sign, uint64_t b,
                    const gj_query* const* qs, uint32_t nq, uint64_t* req_id);
/* Withdraws a request that has not started: GJ_OK, and the request is
 * finished with status GJ_E_CANCELLED (collect it with gj_poll). A cancelled
 * update batch is never applied: later requests see the graph without it.
 * GJ_E_PENDING if the request has started or finished (it keeps its
 * result), GJ_E_NOTFOUND for an unknown or retired id. */
int gj_cancel(gj_ctx* ctx, uint64_t req_id);
/* Waits up to wait_ms (-1: without limit, 0: not at all) for a request; on
 * GJ_OK *out holds its result and the request is retired. GJ_E_PENDING if
 * it is still running, GJ_E_NOTFOUND for an unknown or retired id. */
int gj_poll(gj_ctx* ctx, uint64_t req_id, int wait_ms, gj_result* out);

/* Kernel timing: when enabled, the launches of the dominant kernel of each
 * count call are bracketed by CUDA events on the context's stream and their
 * durations summed. gj_profile_read returns and clears the totals. */
int gj_profile_enable(gj_ctx* ctx, int enabled);
int gj_profile_read(gj_ctx* ctx, double* total_ms, uint64_t* launches);
/* Number of kernels the library has launched on ctx since it was created. */
uint64_t gj_launch_count(const gj_ctx* ctx);
/* 1 in the checked build of the library (libgj_checks.so, compiled with
 * GJ_CHECKS), 0 otherwise. The checked build guards every vertex id, list
 * extent, edge slot, prefix-buffer slot and donated bundle its kernels
 * use; a failed check skips the access (the kernel finishes) and the count,
 * list or update call returns GJ_E_CHECK instead of its results (an update
 * batch is then not committed). Served requests and gj_count_noalloc do not
 * report checks; the next checked call on the context does. */
int gj_checked_build(void);
/* The cudaStream_t all launches of ctx go to. */
void* gj_ctx_stream(gj_ctx* ctx);
/* Waits for all work on ctx's stream. */
int gj_sync(gj_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* GJ_H */
