// Internal declarations shared by the CUDA translation units of libgj.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>
#include <string>
#include <cstring>
#include <climits>
#include <vector>
#include <mutex>
#include <atomic>
#include <cstdio>
#include <nvtx3/nvToolsExt.h>

#include "../../include/gj.h"

#define GJ_MAX_K 8
#define GJ_MAX_ATOMS 16

// ------------------------------------------------------------------ errors

struct gj_status_error {
    int code;
    std::string msg;
};

void gj_set_error(gj_ctx* ctx, int code, const std::string& msg);

#define GJ_CUDA_TRY(ctx, call)                                                              \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) {                                                            \
            gj_set_error((ctx), GJ_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
            return e_ == cudaErrorMemoryAllocation ? GJ_E_NOMEM : GJ_E_CUDA;                \
        }                                                                                   \
    } while (0)

#define GJ_TRY(call)              \
    do {                          \
        int rc_ = (call);         \
        if (rc_ != GJ_OK) return rc_; \
    } while (0)

// ------------------------------------------------------------------ graph

// Adjacency index in CSR form: off[v] .. off[v+1] delimit v's sorted list in
// nbr; key[e] is the vertex whose list holds slot e (so (key[e], nbr[e]) is
// an edge of the index, in index order). Lists of at least GJ_HASH_MIN_DEG
// entries also get an open-addressing hash set in tab (2^ceil(log2(2 len))
// slots from tab_off[v], empty slots all ones, probed in groups of eight
// slots; see gj_tab_member) for constant-time membership.
struct gj_csr {
    int64_t* off = nullptr;      // [n + 1]
    uint32_t* nbr = nullptr;     // [m]
    uint32_t* key = nullptr;     // [m]
    int64_t* tab_off = nullptr;  // [n + 1]
    uint32_t* tab = nullptr;     // [tab_off[n]]
    // allocated lengths of nbr/key and tab (0: exactly m and tab_off[n]); an
    // index kept as the spare of an update can take a larger one in place
    uint64_t cap_m = 0, cap_tab = 0;
};

constexpr uint32_t GJ_HASH_MIN_DEG = 16;
constexpr uint32_t GJ_EMPTY = 0xffffffffu;

// Device view of a graph handed to kernels by value.
struct GraphView {
    uint32_t n;
    uint64_t m;
    const int64_t* __restrict__ fo;
    const uint32_t* __restrict__ fn;
    const uint32_t* __restrict__ fk;
    const int64_t* __restrict__ ro;
    const uint32_t* __restrict__ rn;
    const uint32_t* __restrict__ rk;
    const int64_t* __restrict__ fto;  // hash sets of the forward lists
    const uint32_t* __restrict__ ft;
    const int64_t* __restrict__ rto;  // hash sets of the reverse lists
    const uint32_t* __restrict__ rt;
    const int64_t* __restrict__ to;   // triangle lists per forward slot (null until built)
    const uint32_t* __restrict__ tn;
    const int64_t* __restrict__ tto;  // their hash sets
    const uint32_t* __restrict__ tt;
    const uint4* __restrict__ em;     // edge (a, b) -> its forward slot: {a, b, slot, 0}, 2^ebits entries
    uint32_t ebits;
    uint64_t tcount = 0;               // entries of the triangle lists
    unsigned long long* chk = nullptr;  // checked build: the bounds-check word (see GJ_CHECK)
};

// Bounds checks of the checked build (compiled with -DGJ_CHECKS). Each
// guards one access: a vertex id against the view's vertex count, a list's
// extent against its array, an edge slot against the edge count, a
// prefix-buffer slot against the buffer, a donated bundle's size and level.
// A failed check records (site << 56 | index) in the word chk once and
// makes the guarded access a no-op (an empty list, a non-member, a dropped
// prefix), so the kernel runs to its end; the API call then returns
// GJ_E_CHECK. In the normal build GJ_CHECK is the constant true and the
// condition is not evaluated.
enum { GJ_SITE_VERTEX = 1, GJ_SITE_LIST = 2, GJ_SITE_EDGE = 3, GJ_SITE_PREFIX = 4, GJ_SITE_BUNDLE = 5 };
#ifdef GJ_CHECKS
constexpr bool GJ_CHECKED_BUILD = true;
__device__ __forceinline__ bool gj_check(unsigned long long* w, bool ok, uint32_t site, uint64_t idx) {
    if (!ok && w) atomicCAS(w, 0ull, ((unsigned long long)site << 56) | (idx & ((1ull << 56) - 1)));
    return ok;
}
#define GJ_CHECK(w, cond, site, idx) gj_check((w), (cond), (site), (uint64_t)(idx))
#else
constexpr bool GJ_CHECKED_BUILD = false;
#define GJ_CHECK(w, cond, site, idx) true
#endif

// The ternary relation tri(a, b, c) (a -> b, a -> c, b -> c; Section 5.4)
// indexed by its first two attributes: for the forward slot e of the edge
// a -> b, the c are nbr[off[e] .. off[e+1]), ascending.
struct gj_tri {
    int64_t* off = nullptr;      // [m + 1]
    uint32_t* nbr = nullptr;     // [count]
    int64_t* tab_off = nullptr;  // [m + 1] hash sets of the lists of at least GJ_HASH_MIN_DEG entries
    uint32_t* tab = nullptr;
    // open-addressing map from an edge (a, b) to its forward slot, so that the
    // list of a tri atom is found with one probe instead of a search of out(a)
    uint4* emap = nullptr;
    uint32_t ebits = 0;
    uint64_t count = 0;
};

struct gj_graph {
    gj_ctx* ctx = nullptr;
    uint32_t n = 0;
    uint64_t m = 0;
    uint64_t version = 0;
    uint64_t last_changes = 0;  // normalised changes of the last applied batch
    gj_csr fwd;  // out-neighbours
    gj_csr rev;  // in-neighbours
    gj_tri tri;  // triangle index (built on request; dropped when the graph changes)
    gj_csr spare_fwd, spare_rev;  // the previous version's arrays, reused by the next update's commit
    uint32_t* relabel = nullptr;  // new id of each input id (degree renaming), null = identity
    uint32_t load_flags = 0;
    GraphView view() const;  // the arrays the kernels read (defined after gj_ctx)
};

// ------------------------------------------------------------------ plan

// Execution plan of one query. Positions are places in the execution
// (global attribute) order; x[p] is the value bound at position p.
constexpr uint32_t GJ_MAX_LT = 8;     // inequality filters per level
constexpr uint32_t GJ_MAX_BIND = 12;  // relations binding one level
enum { GJ_BIND_FWD = 0, GJ_BIND_REV = 1, GJ_BIND_TRI = 2 };
struct Plan {
    uint32_t k;
    uint32_t natoms;
    uint32_t qpos[GJ_MAX_K];    // qpos[a] = position of query attribute a (hash in query order)
    uint32_t order[GJ_MAX_K];   // order[p] = query attribute at position p
    // Seed: edges (x0, x1) of the relation over the first two positions.
    // seed_dir 0: edges x0 -> x1, read from the forward index keyed by x0;
    // 1: edges x1 -> x0, read from the reverse index keyed by x0.
    // seed_atom: the edge atom that gives them (delta plans: the atom whose
    // changes seed dQ_i).
    uint32_t seed_atom;
    uint32_t seed_dir;
    uint32_t nsf;                     // further edge atoms over {x0, x1}: membership filters
    uint8_t sf_dir[GJ_MAX_ATOMS];     // 0: edge x0->x1 must exist, 1: edge x1->x0
    // Level p = 2..k-1 extends prefixes of length p by x_p. Binding b gives
    // the list of x[bpos] in the forward index (bdir GJ_BIND_FWD: atom
    // E(x_bpos, x_p)), in the reverse index (GJ_BIND_REV: atom E(x_p,
    // x_bpos)), or the triangle list of the edge x[bpos] -> x[bpos2]
    // (GJ_BIND_TRI: atom tri(x_bpos, x_bpos2, x_p), Section 5.4).
    uint32_t nb[GJ_MAX_K];
    uint8_t bpos[GJ_MAX_K][GJ_MAX_BIND];
    uint8_t bpos2[GJ_MAX_K][GJ_MAX_BIND];
    uint8_t bdir[GJ_MAX_K][GJ_MAX_BIND];
    // Delta queries (Section 3.3.1): which version each atom reads, 0 = the
    // committed graph (old), 1 = the committed graph plus the batch (new).
    // Static plans leave these 0.
    uint8_t bview[GJ_MAX_K][GJ_MAX_BIND];
    uint8_t sf_view[GJ_MAX_ATOMS];
    // Inequality filters (Section 5.4) of level p: the new value x_p must be
    // below (lt_less 1) or above (0) x[lt_pos]. Level 1 holds the filters
    // between x1 and x0 (applied to the seeds).
    uint8_t nlt[GJ_MAX_K];
    uint8_t lt_pos[GJ_MAX_K][GJ_MAX_LT];
    uint8_t lt_less[GJ_MAX_K][GJ_MAX_LT];
    // Aggregation of identical lookups at the last level (the aggregation of
    // requests with equal keys of Section 3.4.2): bit p is set if the last
    // level's lists or filters read x_p. Prefixes that agree on those
    // positions have the same extensions, so consecutive ones are extended
    // once. 0: off (some list reads every earlier position, or delta plans).
    uint32_t agg;
    // Factorised output (Section 5.4): 1 if the last level reads every
    // position before k-2 and not position k-2 itself (k >= 4, static
    // plans). Then the extensions of a level-(k-2) prefix are never
    // materialised: the fused engine counts them (n) and sums their hash
    // factors (S) per level-(k-3) parent, extends each parent once at the
    // last level and weighs its matches by n (count) and S (checksum).
    uint32_t fact;
    uint32_t delta;  // 1: seeds are the batch's signed changes of atom seed_atom
};

enum { GJ_VIEW_OLD = 0, GJ_VIEW_NEW = 1 };

// The normalised changes of one batch, on the device. chg_* are sorted by
// (src, dst); per index direction, ins/del hold the inserted / deleted
// entries sorted by (list owner, neighbour).
struct DeltaSide {
    const uint32_t* ins_key;
    const uint32_t* ins_nbr;
    uint32_t nins;
    const uint32_t* del_key;
    const uint32_t* del_nbr;
    uint32_t ndel;
    // vertex -> its [ins_lo, ins_hi, del_lo, del_hi) ranges, open addressing
    // over the vertices the batch touches (keys all ones when empty)
    const uint32_t* hkey;
    const uint4* hval;
    uint32_t hbits;
};

struct DeltaView {
    DeltaSide fwd, rev;
};

struct DeltaBatch {
    const uint32_t* chg_src = nullptr;
    const uint32_t* chg_dst = nullptr;
    const int8_t* chg_sign = nullptr;
    uint64_t n = 0;
    DeltaView view{};
};

struct gj_query {
    gj_ctx* ctx = nullptr;
    uint32_t k = 0, natoms = 0, ntri = 0, nlt = 0;
    uint32_t as[GJ_MAX_ATOMS], ad[GJ_MAX_ATOMS];
    uint32_t ta[GJ_MAX_ATOMS], tb[GJ_MAX_ATOMS], tc[GJ_MAX_ATOMS];  // tri atoms
    uint32_t la[GJ_MAX_ATOMS], lb[GJ_MAX_ATOMS];                    // x_la < x_lb
    uint32_t order[GJ_MAX_K];
    Plan plan;
    Plan dplan[GJ_MAX_ATOMS];  // delta queries dQ_i, one per atom (edge-atom queries only)
};

// Plan of q's static evaluation in q->order (q's atoms, tri atoms and
// inequalities set; q->order the global order).
int gj_plan_compile(const gj_query* q, Plan* out, std::string* why);
// Plan of delta query dQ_i of q (Section 3.3.1): seeded from the changes of
// atom i, atoms before i read the new version, atoms after i the old one.
int gj_plan_compile_delta(const gj_query* q, uint32_t i, Plan* out, std::string* why);

// ------------------------------------------------------------------ context

struct ScratchArena {
    void* ptr = nullptr;
    size_t bytes = 0;
};

struct KernelTimer {
    bool enabled = false;
    std::vector<cudaEvent_t> pending;  // start/stop pairs recorded in the current call
    std::vector<cudaEvent_t> pool;
    double total_ms = 0.0;
    uint64_t launches = 0;
};

struct gj_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    gj_options opt{};
    int sm_count = 0;
    ScratchArena scratch[6];
    KernelTimer timer;
    uint64_t* d_acc = nullptr;   // small device accumulators (count, checksum, counters)
    uint64_t* h_acc = nullptr;   // pinned host mirror
    std::string last_error;
    std::mutex mu;
    gj_work_stats work{};        // units processed by the last count call
    uint64_t launches = 0;       // kernels launched on this context (host-side count)
    struct gj_server* server = nullptr;  // request loop, while serving
    uint32_t seed_chunk = 32;    // fused engine: seeds per grab
    uint32_t blocks_per_sm = 0;  // fused engine: resident blocks per SM, 0 = as many as fit
    uint32_t donation = 0;       // fused engine work donation: 0 when warps idle, 1 always, 2 off
    uint32_t wait_ms = 0;        // bound of the fused engine's end-of-launch wait without progress, 0 = 10 s
    uint32_t fault = 0;          // failure injection for tests (GJ_FAULT_*)
    uint32_t fault_count = 0;    // GJ_FAULT_ALLOC: allocations that still succeed
    std::atomic<uint64_t> allocs{0};  // device allocations since the settings were applied
};

// Failure injection (gj_tuning.fault): the fused engine's end-of-launch wait
// misses one warp (it ends by its time bound), or its counts start just
// below 2^63 (they overflow), or (checked build only) the graph views the
// kernels get claim one vertex fewer than the graph has, so that the first
// access to the last vertex trips the vertex bounds check.
enum { GJ_FAULT_NONE = 0, GJ_FAULT_WAIT = 1, GJ_FAULT_COUNT = 2, GJ_FAULT_NARROW_VIEW = 3, GJ_FAULT_ALLOC = 4 };

// Every device allocation of the library goes through these two, so that
// failure injection 4 can make the allocations after the first fault_count
// fail (as cudaErrorMemoryAllocation). On failure *p is null.
cudaError_t gj_malloc(gj_ctx* ctx, void** p, size_t bytes);
cudaError_t gj_malloc_async(gj_ctx* ctx, void** p, size_t bytes, cudaStream_t st);
template <typename T>
inline cudaError_t gj_malloc(gj_ctx* ctx, T** p, size_t bytes) {
    return gj_malloc(ctx, reinterpret_cast<void**>(p), bytes);
}
template <typename T>
inline cudaError_t gj_malloc_async(gj_ctx* ctx, T** p, size_t bytes, cudaStream_t st) {
    return gj_malloc_async(ctx, reinterpret_cast<void**>(p), bytes, st);
}

// The bounds-check word of the checked build: the last word of the
// context's accumulators, which no engine clears.
inline unsigned long long* gj_check_word(const gj_ctx* ctx) {
    return GJ_CHECKED_BUILD ? reinterpret_cast<unsigned long long*>(ctx->d_acc + 63) : nullptr;
}

inline GraphView gj_graph::view() const {
    GraphView v{n, m, fwd.off, fwd.nbr, fwd.key, rev.off, rev.nbr, rev.key,
                fwd.tab_off, fwd.tab, rev.tab_off, rev.tab, tri.off, tri.nbr, tri.tab_off, tri.tab,
                tri.emap, tri.ebits};
    v.tcount = tri.count;
    v.chk = gj_check_word(ctx);
    if (GJ_CHECKED_BUILD && ctx->fault == GJ_FAULT_NARROW_VIEW && v.n > 0) v.n--;
    return v;
}

// Checked build: GJ_E_CHECK (with the site and index in the context's
// error text) if a bounds check failed since the last call, and the word
// cleared; GJ_OK otherwise. The normal build returns GJ_OK at once.
int gj_check_status(gj_ctx* ctx);

// Engine of a batch's delta queries: the level-synchronous one spreads a
// small batch's fan-out over the whole GPU at once, the fused one balances
// a large batch's work better; GJ_FLAG_DELTA_PLAIN / _FUSED force either.
constexpr uint64_t GJ_DELTA_FUSED_MIN = 8192;  // normalised changes from which the fused engine runs
inline uint32_t gj_delta_engine(const gj_ctx* ctx, uint64_t changes) {
    if (ctx->opt.flags & GJ_FLAG_DELTA_PLAIN) return GJ_ENGINE_PLAIN;
    if (ctx->opt.flags & GJ_FLAG_DELTA_FUSED) return GJ_ENGINE_FUSED;
    return changes >= GJ_DELTA_FUSED_MIN ? GJ_ENGINE_FUSED : GJ_ENGINE_PLAIN;
}

inline uint64_t gj_wait_ns(const gj_ctx* ctx) { return (uint64_t)(ctx->wait_ms ? ctx->wait_ms : 10000) * 1000000ull; }

// Counts one kernel launch of ctx (gj_launch_count reports the total).
#define GJ_LAUNCHED(ctx) ((ctx)->launches++)

// NVTX range over a scope (host-side: the API call, a level step of the
// level-synchronous engine, a served wave or batch); it costs nothing
// unless a profiler is attached. The name may be printf-formatted.
struct GjRange {
    template <typename... T>
    explicit GjRange(const char* fmt, T... args) {
        if constexpr (sizeof...(T) == 0) {
            nvtxRangePushA(fmt);
        } else {
            char buf[96];
            snprintf(buf, sizeof buf, fmt, args...);
            nvtxRangePushA(buf);
        }
    }
    ~GjRange() { nvtxRangePop(); }
    GjRange(const GjRange&) = delete;
    GjRange& operator=(const GjRange&) = delete;
};
#define GJ_CAT2(a, b) a##b
#define GJ_CAT(a, b) GJ_CAT2(a, b)
#define GJ_RANGE(...) GjRange GJ_CAT(gj_range_, __LINE__)(__VA_ARGS__)

// Grow-only device scratch buffer `slot` of at least `bytes`.
int gj_scratch(gj_ctx* ctx, int slot, size_t bytes, void** out);

// Kernel timing (enabled by gj_profile_enable): wrap launches of the
// dominant kernel.
void gj_timer_begin(gj_ctx* ctx);
void gj_timer_end(gj_ctx* ctx);
int gj_timer_collect(gj_ctx* ctx);

// ------------------------------------------------------------------ host helpers

// Exclusive prefix sum of n values into out[0..n] (out[n] = total), int64.
int gj_scan_u32(gj_ctx* ctx, const uint32_t* in, int64_t* out, uint64_t n);
int gj_scan_i64(gj_ctx* ctx, const int64_t* in, int64_t* out, uint64_t n);

// Sorts n 64-bit keys whose significant bits are [0, bits). keys and tmp
// are n long; the sorted keys end in *result (keys or tmp).
int gj_radix_sort_u64(gj_ctx* ctx, uint64_t* keys, uint64_t* tmp, uint64_t n, int bits, uint64_t** result);
// Stable key-value variant: vals move with their keys (equal keys keep input order).
int gj_radix_sort_kv(gj_ctx* ctx, uint64_t* keys, uint64_t* ktmp, uint32_t* vals, uint32_t* vtmp, uint64_t n, int bits,
                     uint64_t** kresult, uint32_t** vresult);

int gj_csr_build(gj_ctx* ctx, const uint32_t* d_src, const uint32_t* d_dst, uint64_t m, uint32_t n, gj_graph* g);
// Symmetry breaking's input transformation (Section 5.4) on a built graph:
// rebuilds g with the flags of gj_graph_load_ex (symmetrise, rename by
// degree, orient from lower to higher id).
int gj_graph_transform(gj_ctx* ctx, gj_graph* g, uint32_t flags);
// Builds g's triangle index (Section 5.4) if it is missing.
int gj_tri_build(gj_ctx* ctx, gj_graph* g);
void gj_tri_release(gj_tri& t);
// Offsets and hash sets of an index whose key/nbr arrays (mu sorted slots) are set.
int gj_csr_finish(gj_ctx* ctx, uint32_t n, uint64_t mu, gj_csr* out);

// Engines: count (and checksum) of a query over the matches whose x0 lies in [v_lo, v_hi).
int gj_engine_plain(gj_ctx* ctx, const gj_graph* g, const gj_query* q, uint32_t v_lo, uint32_t v_hi,
                    int64_t* count, uint64_t* checksum, uint32_t* out_tuples, uint64_t cap, uint64_t* written);
// The same for an explicit plan; with delta non-null the seeds are the
// batch's changes and every match counts with its seed's sign.
int gj_engine_plain_plan(gj_ctx* ctx, const gj_graph* g, const Plan& P, uint32_t v_lo, uint32_t v_hi,
                         const DeltaBatch* delta, int64_t* count, uint64_t* checksum, uint32_t* out_tuples,
                         uint64_t cap, uint64_t* written);

// Device buffers of one normalised batch (owned; released by gj_delta_free).
struct DeltaBuf {
    void* mem = nullptr;
    DeltaBatch batch;
};
// Normalises an update batch against g (R' = R + Delta R, Section 3.3.1):
// per edge the last update decides, self-loops are dropped, only edges
// whose presence changes remain. Inputs may be host or device arrays.
int gj_delta_prepare(gj_ctx* ctx, const gj_graph* g, const uint32_t* src, const uint32_t* dst, const int8_t* sign,
                     uint64_t b, DeltaBuf* out);
void gj_delta_free(gj_ctx* ctx, DeltaBuf* d);
// Replaces g's indices by those of g + delta (the commit). With old_fwd /
// old_rev given, the previous index arrays are handed back instead of freed
// (readers still in flight keep using them).
int gj_delta_commit(gj_ctx* ctx, gj_graph* g, const DeltaBatch& d, gj_csr* old_fwd = nullptr,
                    gj_csr* old_rev = nullptr);
void gj_csr_release(gj_csr& c);
// Delta queries of a batch on the fused engine: np plans in launches of <= 64.
int gj_engine_fused_delta(gj_ctx* ctx, const gj_graph* g, const DeltaBatch& batch, const Plan* plans, uint32_t np,
                          int64_t* counts, uint64_t* checksums);
// Signed change of each query's count and checksum under a normalised
// batch: the sum over its delta queries dQ_i, on the given engine.
int gj_delta_eval(gj_ctx* ctx, const gj_graph* g, const DeltaBatch& batch, const gj_query* const* qs, uint32_t nq,
                  uint32_t engine, int64_t* counts, uint64_t* checksums);

// One launch over nq queries; counts/checksums are host arrays of nq.
int gj_engine_fused(gj_ctx* ctx, const gj_graph* g, const gj_query* const* qs, uint32_t nq, uint32_t v_lo,
                    uint32_t v_hi, int64_t* counts, uint64_t* checksums);
size_t gj_fused_async_bytes(uint32_t nq);
// Device bytes of one served wave of nq plans (gj_fused_enqueue): the
// launch's arguments and its own donation queue.
size_t gj_fused_wave_bytes(uint32_t nq);
// Resident blocks per SM of the static fused kernel for queries of up to kmax
// attributes (ext: the variant for tri atoms, inequalities or aggregation).
int gj_fused_occupancy(gj_ctx* ctx, uint32_t kmax, bool ext);
// Whether a plan needs the fused kernel's extended variant (tri atoms,
// inequality filters or an aggregated last level).
bool gj_plan_ext(const Plan& p);
int gj_fused_enqueue(gj_ctx* ctx, const GraphView& G, const Plan* hp, uint32_t nq, cudaStream_t st, void* dscratch,
                     unsigned long long** results);

// ------------------------------------------------------------------ device helpers

__host__ __device__ __forceinline__ uint64_t gj_mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

// Factors of the match hash H(x) = q(k) * prod_a f_a(x_a) mod 2^64 (the
// checksum's summand, defined in gj.h): the query's factor and attribute
// a's factor of the value v, all odd.
__host__ __device__ __forceinline__ uint64_t gj_hq(uint32_t k) { return gj_mix64((uint64_t)k) | 1ull; }
__host__ __device__ __forceinline__ uint64_t gj_hf(uint32_t a, uint32_t v) {
    return gj_mix64((uint64_t)v ^ ((uint64_t)(a + 1) * 0x9e3779b97f4a7c15ULL)) | 1ull;
}

// Membership of e in the sorted list a[0..len): branch-free binary search
// (the membership property of an extension index, Section 2.2).
__device__ __forceinline__ bool gj_contains(const uint32_t* __restrict__ a, int64_t len, uint32_t e) {
    if (len <= 0) return false;
    const uint32_t* base = a;
    int64_t n = len;
    while (n > 1) {
        int64_t half = n >> 1;
        base = (__ldg(base + half) <= e) ? base + half : base;
        n -= half;
    }
    return __ldg(base) == e;
}

// Slot count exponent of the hash set of a list of len entries:
// 2^ceil(log2(2 len)) slots, so the load factor stays in (1/4, 1/2].
__host__ __device__ __forceinline__ uint32_t gj_tab_bits(uint32_t len) {
#ifdef __CUDA_ARCH__
    return 32u - __clz(2u * len - 1u);
#else
    uint32_t b = 0;
    while ((1ull << b) < 2ull * len) b++;
    return b;
#endif
}

// Home slot of e in a set of 2^bits slots: multiplicative hashing with
// the 32-bit golden-ratio constant (Knuth, TAOCP vol. 3, Section 6.4).
__device__ __forceinline__ uint32_t gj_tab_home(uint32_t e, uint32_t bits) {
    return (e * 0x9e3779b1u) >> (32u - bits);
}

// Hash sets are read a group of eight slots (one 32-byte sector) at a time:
// a set has at least 32 slots, a power of two, and starts on a 128-byte
// boundary. A key's probe sequence starts at the first slot of its home
// group and runs slot by slot (linear probing, no deletions, never full),
// so a key that is not in its home group was inserted only after that
// group had filled up. Hence, scanning group by group from the home group,
// a group that holds e answers yes and a group with an empty slot answers
// no.
static_assert(GJ_HASH_MIN_DEG >= 4, "a hash set must span whole groups of eight slots");
__device__ __forceinline__ uint32_t gj_tab_start(uint32_t e, uint32_t bits) { return gj_tab_home(e, bits) & ~7u; }

// Reads group g and compares its slots with e: hit if one holds e, emp if
// one is empty.
__device__ __forceinline__ void gj_tab_group(const uint32_t* __restrict__ tab, uint32_t g, uint32_t e, bool& hit,
                                             bool& emp) {
    const uint4 a = __ldg(reinterpret_cast<const uint4*>(tab + g));
    const uint4 b = __ldg(reinterpret_cast<const uint4*>(tab + g) + 1);
    hit = (a.x == e) | (a.y == e) | (a.z == e) | (a.w == e) | (b.x == e) | (b.y == e) | (b.z == e) | (b.w == e);
    emp = (a.x == GJ_EMPTY) | (a.y == GJ_EMPTY) | (a.z == GJ_EMPTY) | (a.w == GJ_EMPTY) | (b.x == GJ_EMPTY) |
          (b.y == GJ_EMPTY) | (b.z == GJ_EMPTY) | (b.w == GJ_EMPTY);
}

// Membership of e in a hash set of 2^bits slots.
__device__ __forceinline__ bool gj_tab_member(const uint32_t* __restrict__ tab, uint32_t bits, uint32_t e) {
    const uint32_t mask = (1u << bits) - 1u;
    uint32_t g = gj_tab_start(e, bits);
    while (true) {
        bool hit, emp;
        gj_tab_group(tab, g, e, hit, emp);
        if (hit) return true;
        if (emp) return false;
        g = (g + 8u) & mask;
    }
}

// Membership of e in the list of v in index (off, nbr, tab_off, tab): the
// hash set for long lists, binary search for short ones.
__device__ __forceinline__ bool gj_list_member(const int64_t* __restrict__ off, const uint32_t* __restrict__ nbr,
                                               const int64_t* __restrict__ tab_off, const uint32_t* __restrict__ tab,
                                               uint32_t v, uint32_t e) {
    const int64_t s = __ldg(off + v);
    const uint32_t len = (uint32_t)(__ldg(off + v + 1) - s);
    if (len >= GJ_HASH_MIN_DEG) return gj_tab_member(tab + __ldg(tab_off + v), gj_tab_bits(len), e);
    return gj_contains(nbr + s, len, e);
}

// [lo, hi) of the entries owned by v in a key-sorted array.
__device__ __forceinline__ void gj_key_range(const uint32_t* __restrict__ key, uint32_t n, uint32_t v, uint32_t& lo,
                                             uint32_t& hi) {
    uint32_t a = 0, b = n;
    while (a < b) {
        uint32_t mid = (a + b) >> 1;
        if (__ldg(key + mid) < v) a = mid + 1; else b = mid;
    }
    lo = a;
    b = n;
    while (a < b) {
        uint32_t mid = (a + b) >> 1;
        if (__ldg(key + mid) <= v) a = mid + 1; else b = mid;
    }
    hi = a;
}

// A list of vertex v as seen by one view: the committed list, plus (new
// view only) the batch's inserted entries and the deleted ones to skip.
// Enumeration space: [0, base_len) committed entries, then the inserts.
struct ViewList {
    const uint32_t* base;
    uint32_t base_len;
    const uint32_t* ins;
    uint32_t nins;
    const uint32_t* del;
    uint32_t ndel;
    __device__ uint32_t degree() const { return base_len + nins - ndel; }
    __device__ uint32_t space() const { return base_len + nins; }
};

// The batch's insert and delete ranges of vertex v in one direction (empty
// when the batch does not touch v).
__device__ __forceinline__ uint4 gj_delta_ranges(const DeltaSide& S, uint32_t v) {
    if (S.hbits == 0) return make_uint4(0, 0, 0, 0);
    const uint32_t mask = (1u << S.hbits) - 1u;
    uint32_t h = gj_tab_home(v, S.hbits);
    while (true) {
        const uint32_t k = __ldg(S.hkey + h);
        if (k == v) return S.hval[h];
        if (k == GJ_EMPTY) return make_uint4(0, 0, 0, 0);
        h = (h + 1u) & mask;
    }
}

__device__ __forceinline__ ViewList gj_view_list(const GraphView& G, const DeltaView* D, uint32_t dir, uint32_t view,
                                                 uint32_t v) {
    if (!GJ_CHECK(G.chk, v < G.n, GJ_SITE_VERTEX, v)) return ViewList{G.fn, 0, nullptr, 0, nullptr, 0};
    const int64_t* off = dir ? G.ro : G.fo;
    const int64_t s = __ldg(off + v);
    ViewList L{(dir ? G.rn : G.fn) + s, (uint32_t)(__ldg(off + v + 1) - s), nullptr, 0, nullptr, 0};
    if (!GJ_CHECK(G.chk, (uint64_t)s + L.base_len <= G.m, GJ_SITE_LIST, v)) L.base_len = 0;
    if (view == GJ_VIEW_NEW && D) {
        const DeltaSide& S = dir ? D->rev : D->fwd;
        const uint4 r = gj_delta_ranges(S, v);
        L.ins = S.ins_nbr + r.x;
        L.nins = r.y - r.x;
        L.del = S.del_nbr + r.z;
        L.ndel = r.w - r.z;
    }
    return L;
}

// Membership of x in v's list under a view: the committed index first,
// then one of the batch's change lists of v. The batch is normalised
// (inserts are absent from the committed list, deletes present), so a
// committed member is a member unless deleted, and any other x only if
// inserted.
__device__ __forceinline__ bool gj_view_member(const GraphView& G, const DeltaView* D, uint32_t dir, uint32_t view,
                                               uint32_t v, uint32_t x) {
    if (!GJ_CHECK(G.chk, v < G.n, GJ_SITE_VERTEX, v)) return false;
    const bool c = dir ? gj_list_member(G.ro, G.rn, G.rto, G.rt, v, x) : gj_list_member(G.fo, G.fn, G.fto, G.ft, v, x);
    if (view == GJ_VIEW_NEW && D) {
        const DeltaSide& S = dir ? D->rev : D->fwd;
        const uint4 r = gj_delta_ranges(S, v);
        return c ? !gj_contains(S.del_nbr + r.z, r.w - r.z, x) : gj_contains(S.ins_nbr + r.x, r.y - r.x, x);
    }
    return c;
}

// The list a binding of a plan level reads for one prefix (static plans):
// the sorted list p[0, len) and, for long index lists, its hash set (bits
// > 0). v is x[bpos]; v2 is x[bpos2] (tri bindings only).
struct BindList {
    const uint32_t* p;
    uint32_t len;
    const uint32_t* tab;
    uint32_t bits;
};

// Home entry of the edge (a, b) in the edge map: multiplicative hashing of
// the 64-bit pair with the 64-bit golden-ratio constant (Knuth, TAOCP vol. 3,
// Section 6.4).
__host__ __device__ __forceinline__ uint32_t gj_edge_home(uint32_t a, uint32_t b, uint32_t bits) {
    return (uint32_t)(((((uint64_t)a << 32) | b) * 0x9e3779b97f4a7c15ULL) >> (64 - bits));
}

// Forward slot of the edge a -> b, or -1 (edge map lookup, linear probing).
__device__ __forceinline__ int64_t gj_edge_slot(const GraphView& G, uint32_t a, uint32_t b) {
    const uint32_t mask = (uint32_t)((1ull << G.ebits) - 1u);
    uint32_t h = gj_edge_home(a, b, G.ebits);
    while (true) {
        const uint4 E = __ldg(G.em + h);
        if (E.x == a && E.y == b) return (int64_t)E.z;
        if (E.x == GJ_EMPTY) return -1;
        h = (h + 1u) & mask;
    }
}

__device__ __forceinline__ BindList gj_bind_list(const GraphView& G, uint32_t dir, uint32_t v, uint32_t v2) {
    if (dir == GJ_BIND_TRI) {
        // the triangles on the edge v -> v2: its forward slot, then its list
        const int64_t e = gj_edge_slot(G, v, v2);
        if (e < 0 || !GJ_CHECK(G.chk, (uint64_t)e < G.m, GJ_SITE_EDGE, e)) return BindList{G.fn, 0u, nullptr, 0u};
        const int64_t a = __ldg(G.to + e);
        const uint32_t len = (uint32_t)(__ldg(G.to + e + 1) - a);
        if (!GJ_CHECK(G.chk, (uint64_t)a + len <= G.tcount, GJ_SITE_LIST, e)) return BindList{G.fn, 0u, nullptr, 0u};
        if (len >= GJ_HASH_MIN_DEG) return BindList{G.tn + a, len, G.tt + __ldg(G.tto + e), gj_tab_bits(len)};
        return BindList{G.tn + a, len, nullptr, 0u};
    }
    if (!GJ_CHECK(G.chk, v < G.n, GJ_SITE_VERTEX, v)) return BindList{G.fn, 0u, nullptr, 0u};
    const int64_t* off = dir ? G.ro : G.fo;
    const int64_t s = __ldg(off + v);
    const uint32_t len = (uint32_t)(__ldg(off + v + 1) - s);
    if (!GJ_CHECK(G.chk, (uint64_t)s + len <= G.m, GJ_SITE_LIST, v)) return BindList{G.fn, 0u, nullptr, 0u};
    const uint32_t* p = (dir ? G.rn : G.fn) + s;
    if (len >= GJ_HASH_MIN_DEG) return BindList{p, len, (dir ? G.rt : G.ft) + __ldg((dir ? G.rto : G.fto) + v), gj_tab_bits(len)};
    return BindList{p, len, nullptr, 0u};
}

__device__ __forceinline__ bool gj_bind_member(const BindList& L, uint32_t e) {
    return L.bits ? gj_tab_member(L.tab, L.bits, e) : gj_contains(L.p, L.len, e);
}

// Whether the value e of position j meets level j's inequality filters;
// val(p) gives the prefix's value at position p.
template <class F>
__device__ __forceinline__ bool gj_lt_ok(const Plan& P, uint32_t j, uint32_t e, F val) {
    for (uint32_t c = 0; c < P.nlt[j]; c++) {
        const uint32_t v = val(P.lt_pos[j][c]);
        if (P.lt_less[j][c] ? !(e < v) : !(e > v)) return false;
    }
    return true;
}

__device__ __forceinline__ uint32_t gj_lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

static inline unsigned gj_div_up(uint64_t a, uint64_t b) { return (unsigned)((a + b - 1) / b); }
