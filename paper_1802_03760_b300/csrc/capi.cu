// C ABI entry points of libgj (declared and documented in include/gj.h):
// context, graph and query handles, counting, listing and kernel timing.
#include "gj_internal.cuh"

#include <chrono>
#include <new>

void gj_set_error(gj_ctx* ctx, int code, const std::string& msg) {
    (void)code;
    if (ctx) ctx->last_error = msg;
}

static bool alloc_injected(gj_ctx* ctx) {
    return ctx && ctx->fault == GJ_FAULT_ALLOC && ctx->allocs.fetch_add(1) >= ctx->fault_count;
}

cudaError_t gj_malloc(gj_ctx* ctx, void** p, size_t bytes) {
    *p = nullptr;
    if (alloc_injected(ctx)) return cudaErrorMemoryAllocation;
    const cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) *p = nullptr;
    return e;
}

cudaError_t gj_malloc_async(gj_ctx* ctx, void** p, size_t bytes, cudaStream_t st) {
    *p = nullptr;
    if (alloc_injected(ctx)) return cudaErrorMemoryAllocation;
    const cudaError_t e = cudaMallocAsync(p, bytes, st);
    if (e != cudaSuccess) *p = nullptr;
    return e;
}

int gj_scratch(gj_ctx* ctx, int slot, size_t bytes, void** out) {
    ScratchArena& a = ctx->scratch[slot];
    if (a.bytes < bytes) {
        if (a.ptr) {
            GJ_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
            cudaFree(a.ptr);
            a.ptr = nullptr;
            a.bytes = 0;
        }
        size_t want = bytes + bytes / 8;
        GJ_CUDA_TRY(ctx, gj_malloc(ctx, &a.ptr, want));
        a.bytes = want;
    }
    *out = a.ptr;
    return GJ_OK;
}

void gj_timer_begin(gj_ctx* ctx) {
    KernelTimer& t = ctx->timer;
    if (!t.enabled) return;
    cudaEvent_t e;
    if (!t.pool.empty()) {
        e = t.pool.back();
        t.pool.pop_back();
    } else if (cudaEventCreate(&e) != cudaSuccess) {
        return;
    }
    cudaEventRecord(e, ctx->stream);
    t.pending.push_back(e);
}

void gj_timer_end(gj_ctx* ctx) {
    KernelTimer& t = ctx->timer;
    if (!t.enabled || t.pending.size() % 2 == 0) return;
    cudaEvent_t e;
    if (!t.pool.empty()) {
        e = t.pool.back();
        t.pool.pop_back();
    } else if (cudaEventCreate(&e) != cudaSuccess) {
        return;
    }
    cudaEventRecord(e, ctx->stream);
    t.pending.push_back(e);
}

int gj_timer_collect(gj_ctx* ctx) {
    KernelTimer& t = ctx->timer;
    if (t.pending.empty()) return GJ_OK;
    size_t n = t.pending.size() & ~(size_t)1;
    if (n) GJ_CUDA_TRY(ctx, cudaEventSynchronize(t.pending[n - 1]));
    for (size_t i = 0; i + 1 < n; i += 2) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, t.pending[i], t.pending[i + 1]) == cudaSuccess) {
            t.total_ms += ms;
            t.launches++;
        }
    }
    for (cudaEvent_t e : t.pending) t.pool.push_back(e);
    t.pending.clear();
    return GJ_OK;
}

int gj_check_status(gj_ctx* ctx) {
    if (!GJ_CHECKED_BUILD) return GJ_OK;
    unsigned long long* word = gj_check_word(ctx);
    unsigned long long w = 0;
    GJ_CUDA_TRY(ctx, cudaMemcpyAsync(&w, word, sizeof(w), cudaMemcpyDeviceToHost, ctx->stream));
    GJ_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    if (!w) return GJ_OK;
    GJ_CUDA_TRY(ctx, cudaMemsetAsync(word, 0, sizeof(w), ctx->stream));
    static const char* const site[] = {"?", "vertex id", "list extent", "edge slot", "prefix-buffer slot",
                                       "donated bundle"};
    const unsigned s = (unsigned)(w >> 56);
    char buf[160];
    snprintf(buf, sizeof buf, "checked build: a %s bounds check failed (index %llu); the access was skipped",
             site[s < 6 ? s : 0], (unsigned long long)(w & ((1ull << 56) - 1)));
    gj_set_error(ctx, GJ_E_CHECK, buf);
    return GJ_E_CHECK;
}

namespace {

// 1: device memory of device dev, 0: host memory, -1: another device's memory
int ptr_kind(const void* p, int dev) {
    if (!p) return 0;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) return 0;
    return at.device == dev ? 1 : -1;
}

// Queries with tri atoms read the graph's triangle index: build it if missing.
int ensure_tri(gj_ctx* ctx, gj_graph* g, const gj_query* const* qs, uint32_t nq) {
    for (uint32_t i = 0; i < nq; i++)
        if (qs[i]->ntri) return gj_tri_build(ctx, g);
    return GJ_OK;
}

int autotune_sweep(gj_graph* g, const gj_query* const* qs, uint32_t nq, uint64_t prefix_cap_bytes, uint32_t v_lo,
                   uint32_t v_hi, gj_tuning* out);

struct DevSet {
    int prev = -1;
    explicit DevSet(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DevSet() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace

extern "C" {

const char* gj_strerror(int code) {
    switch (code) {
        case GJ_OK: return "ok";
        case GJ_E_INVALID: return "invalid argument";
        case GJ_E_RANGE: return "vertex id out of range";
        case GJ_E_NOMEM: return "out of memory";
        case GJ_E_ADMIT: return "request exceeds the memory budget";
        case GJ_E_TRUNCATED: return "output truncated";
        case GJ_E_TIMEOUT: return "bounded wait expired";
        case GJ_E_OVERFLOW: return "count overflow";
        case GJ_E_CUDA: return "CUDA error";
        case GJ_E_PENDING: return "request pending";
        case GJ_E_NOTFOUND: return "unknown request";
        case GJ_E_CHECK: return "a device bounds check failed (checked build)";
        case GJ_E_CANCELLED: return "request cancelled";
        default: return "unknown error";
    }
}

const char* gj_last_error(const gj_ctx* ctx) { return ctx ? ctx->last_error.c_str() : ""; }

int gj_create(int cuda_device, const gj_options* opt, gj_ctx** out) {
    if (!out) return GJ_E_INVALID;
    *out = nullptr;
    if (cuda_device < 0) return GJ_E_INVALID;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) {  // no usable CUDA driver or device
        cudaGetLastError();
        return GJ_E_CUDA;
    }
    if (cuda_device >= ndev) return GJ_E_INVALID;
    if (opt && opt->engine > GJ_ENGINE_FUSED) return GJ_E_INVALID;
    gj_ctx* ctx = new (std::nothrow) gj_ctx();
    if (!ctx) return GJ_E_NOMEM;
    ctx->device = cuda_device;
    if (opt) ctx->opt = *opt;
    DevSet ds(cuda_device);
    cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, cuda_device);
    if (ctx->opt.stream) {
        ctx->stream = (cudaStream_t)ctx->opt.stream;
    } else {
        if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete ctx;
            return GJ_E_CUDA;
        }
        ctx->own_stream = true;
    }
    if (gj_malloc(ctx, &ctx->d_acc, 64 * sizeof(uint64_t)) != cudaSuccess ||
        cudaMallocHost(&ctx->h_acc, 64 * sizeof(uint64_t)) != cudaSuccess) {
        gj_destroy(ctx);
        return GJ_E_NOMEM;
    }
    if (cudaMemset(ctx->d_acc, 0, 64 * sizeof(uint64_t)) != cudaSuccess) {
        gj_destroy(ctx);
        return GJ_E_CUDA;
    }
    *out = ctx;
    return GJ_OK;
}

void gj_destroy(gj_ctx* ctx) {
    if (!ctx) return;
    if (ctx->server) gj_serve_stop(ctx);
    DevSet ds(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    for (auto& a : ctx->scratch)
        if (a.ptr) cudaFree(a.ptr);
    for (cudaEvent_t e : ctx->timer.pool) cudaEventDestroy(e);
    for (cudaEvent_t e : ctx->timer.pending) cudaEventDestroy(e);
    if (ctx->d_acc) cudaFree(ctx->d_acc);
    if (ctx->h_acc) cudaFreeHost(ctx->h_acc);
    if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

void* gj_ctx_stream(gj_ctx* ctx) { return ctx ? (void*)ctx->stream : nullptr; }

uint64_t gj_launch_count(const gj_ctx* ctx) { return ctx ? ctx->launches : 0; }

int gj_checked_build(void) { return GJ_CHECKED_BUILD ? 1 : 0; }

int gj_sync(gj_ctx* ctx) {
    if (!ctx) return GJ_E_INVALID;
    GJ_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    return GJ_OK;
}

int gj_profile_enable(gj_ctx* ctx, int enabled) {
    if (!ctx) return GJ_E_INVALID;
    ctx->timer.enabled = enabled != 0;
    return GJ_OK;
}

int gj_profile_read(gj_ctx* ctx, double* total_ms, uint64_t* launches) {
    if (!ctx) return GJ_E_INVALID;
    GJ_TRY(gj_timer_collect(ctx));
    if (total_ms) *total_ms = ctx->timer.total_ms;
    if (launches) *launches = ctx->timer.launches;
    ctx->timer.total_ms = 0;
    ctx->timer.launches = 0;
    return GJ_OK;
}

void gj_graph_free(gj_graph* g) {
    if (!g) return;
    if (g->ctx->server) gj_serve_stop(g->ctx);  // the loop may still read g
    DevSet ds(g->ctx->device);
    cudaStreamSynchronize(g->ctx->stream);
    for (gj_csr* c : {&g->fwd, &g->rev, &g->spare_fwd, &g->spare_rev}) gj_csr_release(*c);
    gj_tri_release(g->tri);
    if (g->relabel) cudaFree(g->relabel);
    delete g;
}

int gj_graph_load_ex(gj_ctx* ctx, const uint32_t* src, const uint32_t* dst, uint64_t m, uint32_t num_vertices,
                     uint32_t flags, gj_graph** out) {
    if (!ctx || !out || num_vertices == 0 || num_vertices == UINT32_MAX || (m > 0 && (!src || !dst)))
        return GJ_E_INVALID;
    if (flags & ~(uint32_t)(GJ_LOAD_SYMMETRIZE | GJ_LOAD_DEGREE_ORDER | GJ_LOAD_ORIENT)) return GJ_E_INVALID;
    *out = nullptr;
    DevSet ds(ctx->device);
    std::lock_guard<std::mutex> lk(ctx->mu);
    GJ_RANGE("gj_graph_load (%llu edges)", (unsigned long long)m);
    cudaStream_t st = ctx->stream;
    const int ks = ptr_kind(src, ctx->device), kd = ptr_kind(dst, ctx->device);
    if (m > 0 && (ks < 0 || kd < 0)) {
        gj_set_error(ctx, GJ_E_INVALID, "graph load: an edge array is in another device's memory");
        return GJ_E_INVALID;
    }
    const bool sym = flags & GJ_LOAD_SYMMETRIZE;
    const uint64_t mm = sym ? 2 * m : m;  // with symmetrisation: (src, dst) then (dst, src)
    const uint32_t* ds_ = src;
    const uint32_t* dd_ = dst;
    uint32_t* tmp = nullptr;
    if (m > 0 && (sym || ks == 0 || kd == 0)) {
        GJ_CUDA_TRY(ctx, gj_malloc_async(ctx, &tmp, 2 * mm * sizeof(uint32_t), st));
        cudaError_t e = cudaSuccess;
        ds_ = tmp;
        dd_ = tmp + mm;
        for (int half = 0; half < (sym ? 2 : 1) && e == cudaSuccess; half++) {
            const uint32_t* a = half ? dst : src;  // sources of this half
            const uint32_t* b = half ? src : dst;
            const int ka = half ? kd : ks, kb = half ? ks : kd;
            e = cudaMemcpyAsync(tmp + half * m, a, m * 4, ka ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(tmp + mm + half * m, b, m * 4,
                                    kb ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st);
        }
        if (e != cudaSuccess) {
            cudaFreeAsync(tmp, st);
            gj_set_error(ctx, GJ_E_CUDA, std::string("graph load: copy of the edge list: ") + cudaGetErrorString(e));
            return GJ_E_CUDA;
        }
    }
    gj_graph* g = new (std::nothrow) gj_graph();
    if (!g) {
        if (tmp) cudaFreeAsync(tmp, st);
        return GJ_E_NOMEM;
    }
    g->ctx = ctx;
    g->load_flags = flags;
    int rc = gj_csr_build(ctx, ds_, dd_, mm, num_vertices, g);
    if (tmp) cudaFreeAsync(tmp, st);
    if (rc == GJ_OK) rc = gj_graph_transform(ctx, g, flags);
    if (rc != GJ_OK) {
        gj_graph_free(g);
        return rc;
    }
    *out = g;
    return GJ_OK;
}

int gj_graph_load(gj_ctx* ctx, const uint32_t* src, const uint32_t* dst, uint64_t m, uint32_t num_vertices,
                  gj_graph** out) {
    return gj_graph_load_ex(ctx, src, dst, m, num_vertices, 0, out);
}

int gj_graph_relabel_map(const gj_graph* g, uint32_t* new_of_old) {
    if (!g || !new_of_old) return GJ_E_INVALID;
    gj_ctx* ctx = g->ctx;
    if (!g->relabel) {
        for (uint32_t v = 0; v < g->n; v++) new_of_old[v] = v;
        return GJ_OK;
    }
    DevSet ds(ctx->device);
    GJ_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    GJ_CUDA_TRY(ctx, cudaMemcpy(new_of_old, g->relabel, sizeof(uint32_t) * g->n, cudaMemcpyDeviceToHost));
    return GJ_OK;
}

int gj_graph_build_triangles(gj_graph* g, uint64_t* count) {
    if (!g) return GJ_E_INVALID;
    gj_ctx* ctx = g->ctx;
    if (ctx->server) return GJ_E_INVALID;
    DevSet ds(ctx->device);
    std::lock_guard<std::mutex> lk(ctx->mu);
    GJ_RANGE("gj_graph_build_triangles");
    GJ_TRY(gj_tri_build(ctx, g));
    if (count) *count = g->tri.count;
    return GJ_OK;
}

int gj_graph_stats(const gj_graph* g, uint64_t* num_edges, uint64_t* version) {
    if (!g) return GJ_E_INVALID;
    if (num_edges) *num_edges = g->m;
    if (version) *version = g->version;
    return GJ_OK;
}

int gj_graph_export(const gj_graph* g, int64_t* offsets, uint32_t* neighbours) {
    if (!g || !offsets || (!neighbours && g->m)) return GJ_E_INVALID;
    gj_ctx* ctx = g->ctx;
    DevSet ds(ctx->device);
    GJ_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    GJ_CUDA_TRY(ctx, cudaMemcpy(offsets, g->fwd.off, sizeof(int64_t) * ((size_t)g->n + 1), cudaMemcpyDeviceToHost));
    if (g->m) GJ_CUDA_TRY(ctx, cudaMemcpy(neighbours, g->fwd.nbr, sizeof(uint32_t) * g->m, cudaMemcpyDeviceToHost));
    return GJ_OK;
}

int gj_query_define_ex(gj_ctx* ctx, uint32_t k, const uint32_t* atoms, uint32_t n_atoms, const uint32_t* tri_atoms,
                       uint32_t n_tri, const uint32_t* lt_pairs, uint32_t n_lt, const uint32_t* order,
                       gj_query** out) {
    if (!ctx || !out || (n_atoms && !atoms) || (n_tri && !tri_atoms) || (n_lt && !lt_pairs)) return GJ_E_INVALID;
    *out = nullptr;
    if (n_atoms > GJ_MAX_ATOMS || n_tri > GJ_MAX_ATOMS || n_lt > GJ_MAX_ATOMS || k > GJ_MAX_K || k < 2) {
        gj_set_error(ctx, GJ_E_INVALID, "k must be in [2, 8] and each list hold at most 16 entries");
        return GJ_E_INVALID;
    }
    gj_query* q = new (std::nothrow) gj_query();
    if (!q) return GJ_E_NOMEM;
    q->ctx = ctx;
    q->k = k;
    q->natoms = n_atoms;
    q->ntri = n_tri;
    q->nlt = n_lt;
    for (uint32_t t = 0; t < n_atoms; t++) {
        q->as[t] = atoms[2 * t];
        q->ad[t] = atoms[2 * t + 1];
    }
    for (uint32_t t = 0; t < n_tri; t++) {
        q->ta[t] = tri_atoms[3 * t];
        q->tb[t] = tri_atoms[3 * t + 1];
        q->tc[t] = tri_atoms[3 * t + 2];
    }
    for (uint32_t t = 0; t < n_lt; t++) {
        q->la[t] = lt_pairs[2 * t];
        q->lb[t] = lt_pairs[2 * t + 1];
    }
    for (uint32_t j = 0; j < k; j++) q->order[j] = order ? order[j] : j;
    std::string why;
    int rc = gj_plan_compile(q, &q->plan, &why);
    if (rc != GJ_OK) {
        gj_set_error(ctx, rc, "query: " + why);
        delete q;
        return rc;
    }
    for (uint32_t i = 0; i < n_atoms && n_tri == 0; i++) {
        rc = gj_plan_compile_delta(q, i, &q->dplan[i], &why);
        if (rc != GJ_OK) {
            gj_set_error(ctx, rc, "query: " + why);
            delete q;
            return rc;
        }
    }
    *out = q;
    return GJ_OK;
}

int gj_query_define(gj_ctx* ctx, uint32_t k, const uint32_t* atoms, uint32_t n_atoms, const uint32_t* order,
                    gj_query** out) {
    if (!atoms) return GJ_E_INVALID;
    return gj_query_define_ex(ctx, k, atoms, n_atoms, nullptr, 0, nullptr, 0, order, out);
}

void gj_query_free(gj_query* q) { delete q; }

int gj_count_ex(gj_graph* g, const gj_query* q, uint32_t engine, uint32_t v_lo, uint32_t v_hi, int64_t* count,
                uint64_t* checksum, gj_work_stats* stats) {
    if (!g || !q || !count || !checksum || q->ctx != g->ctx || engine > GJ_ENGINE_FUSED) return GJ_E_INVALID;
    gj_ctx* ctx = g->ctx;
    if (ctx->server) return GJ_E_INVALID;
    DevSet ds(ctx->device);
    std::lock_guard<std::mutex> lk(ctx->mu);
    GJ_RANGE("gj_count (k=%u, %s engine)", q->k, engine == GJ_ENGINE_PLAIN ? "level-synchronous" : "fused");
    GJ_TRY(ensure_tri(ctx, g, &q, 1));
    int rc;
    if (engine == GJ_ENGINE_PLAIN)
        rc = gj_engine_plain(ctx, g, q, v_lo, v_hi, count, checksum, nullptr, 0, nullptr);
    else
        rc = gj_engine_fused(ctx, g, &q, 1, v_lo, v_hi, count, checksum);
    if (rc == GJ_OK) rc = gj_check_status(ctx);
    if (rc == GJ_OK && stats) *stats = ctx->work;
    return rc;
}

int gj_count_many_ex(gj_graph* g, const gj_query* const* qs, uint32_t nq, uint32_t engine, uint32_t v_lo,
                     uint32_t v_hi, int64_t* counts, uint64_t* checksums) {
    if (!g || (nq && (!qs || !counts || !checksums)) || engine > GJ_ENGINE_FUSED) return GJ_E_INVALID;
    for (uint32_t i = 0; i < nq; i++)
        if (!qs[i] || qs[i]->ctx != g->ctx) return GJ_E_INVALID;
    gj_ctx* ctx = g->ctx;
    if (ctx->server) return GJ_E_INVALID;
    DevSet ds(ctx->device);
    std::lock_guard<std::mutex> lk(ctx->mu);
    GJ_RANGE("gj_count_many (%u queries, %s engine)", nq, engine == GJ_ENGINE_PLAIN ? "level-synchronous" : "fused");
    GJ_TRY(ensure_tri(ctx, g, qs, nq));
    if (engine == GJ_ENGINE_FUSED) {
        GJ_TRY(gj_engine_fused(ctx, g, qs, nq, v_lo, v_hi, counts, checksums));
        return gj_check_status(ctx);
    }
    gj_work_stats sum{};
    for (uint32_t i = 0; i < nq; i++) {
        GJ_TRY(gj_engine_plain(ctx, g, qs[i], v_lo, v_hi, counts + i, checksums + i, nullptr, 0, nullptr));
        const gj_work_stats& w = ctx->work;
        sum.seeds += w.seeds;
        for (int j = 0; j < 9; j++) {
            sum.extended[j] += w.extended[j];
            sum.nbind[j] += w.nbind[j];
            sum.proposals[j] += w.proposals[j];
            sum.produced[j] += w.produced[j];
        }
    }
    ctx->work = sum;
    return gj_check_status(ctx);
}

int gj_count_many(gj_graph* g, const gj_query* const* qs, uint32_t nq, uint32_t engine, int64_t* counts,
                  uint64_t* checksums) {
    return gj_count_many_ex(g, qs, nq, engine, 0, UINT32_MAX, counts, checksums);
}

int gj_get_tuning(const gj_ctx* ctx, gj_tuning* out) {
    if (!ctx || !out) return GJ_E_INVALID;
    memset(out, 0, sizeof(*out));
    out->seed_chunk = ctx->seed_chunk;
    out->blocks_per_sm = ctx->blocks_per_sm;
    out->prefix_buffer_bytes = ctx->opt.prefix_buffer_bytes;
    out->donation = ctx->donation;
    out->wait_ms = ctx->wait_ms;
    out->fault = ctx->fault;
    out->fault_count = ctx->fault_count;
    return GJ_OK;
}

int gj_set_tuning(gj_ctx* ctx, const gj_tuning* t) {
    if (!ctx || !t || t->seed_chunk < 8 || t->seed_chunk > 4096 || t->seed_chunk % 8) return GJ_E_INVALID;
    if (t->prefix_buffer_bytes && t->prefix_buffer_bytes < (1ull << 20)) return GJ_E_INVALID;
    if (t->donation > 2 || t->fault > GJ_FAULT_ALLOC) return GJ_E_INVALID;
    if (t->fault == GJ_FAULT_NARROW_VIEW && !GJ_CHECKED_BUILD) {
        gj_set_error(ctx, GJ_E_INVALID, "failure injection 3 (narrowed graph views) needs the checked build");
        return GJ_E_INVALID;
    }
    ctx->seed_chunk = t->seed_chunk;
    ctx->wait_ms = t->wait_ms;
    ctx->fault = t->fault;
    ctx->fault_count = t->fault_count;
    ctx->allocs = 0;
    ctx->donation = t->donation;
    ctx->blocks_per_sm = t->blocks_per_sm;
    ctx->opt.prefix_buffer_bytes = t->prefix_buffer_bytes;
    return GJ_OK;
}

int gj_autotune(gj_graph* g, const gj_query* const* qs, uint32_t nq, uint64_t prefix_cap_bytes, uint32_t v_lo,
                uint32_t v_hi, gj_tuning* out) {
    if (!g || !qs || !nq || !out) return GJ_E_INVALID;
    gj_ctx* ctx = g->ctx;
    if (ctx->server) return GJ_E_INVALID;
    DevSet ds(ctx->device);
    // on any failure the context keeps the settings it had before the call
    const uint32_t old_chunk = ctx->seed_chunk, old_bps = ctx->blocks_per_sm, old_don = ctx->donation;
    const uint64_t old_bytes = ctx->opt.prefix_buffer_bytes;
    const int rc = autotune_sweep(g, qs, nq, prefix_cap_bytes, v_lo, v_hi, out);
    if (rc != GJ_OK) {
        ctx->seed_chunk = old_chunk;
        ctx->blocks_per_sm = old_bps;
        ctx->donation = old_don;
        ctx->opt.prefix_buffer_bytes = old_bytes;
    }
    return rc;
}

}  // extern "C"

namespace {

int autotune_sweep(gj_graph* g, const gj_query* const* qs, uint32_t nq, uint64_t prefix_cap_bytes, uint32_t v_lo,
                   uint32_t v_hi, gj_tuning* out) {
    gj_ctx* ctx = g->ctx;
    std::vector<int64_t> c(nq);
    std::vector<uint64_t> h(nq);
    auto timed = [&](uint32_t engine, double* ms) -> int {
        GJ_TRY(gj_count_many_ex(g, qs, nq, engine, v_lo, v_hi, c.data(), h.data()));  // warm
        auto t0 = std::chrono::steady_clock::now();
        GJ_TRY(gj_count_many_ex(g, qs, nq, engine, v_lo, v_hi, c.data(), h.data()));
        *ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        return GJ_OK;
    };
    // fused engine: seeds per grab x resident blocks per SM
    int per_sm_max = 0;
    {
        uint32_t kmax = 2;
        bool ext = false;
        for (uint32_t i = 0; i < nq; i++) {
            kmax = qs[i]->k > kmax ? qs[i]->k : kmax;
            ext = ext || gj_plan_ext(qs[i]->plan);
        }
        per_sm_max = gj_fused_occupancy(ctx, kmax, ext);
    }
    double best_f = 1e300;
    uint32_t best_chunk = 32, best_bps = 0, best_don = 0;
    for (uint32_t chunk : {8u, 32u, 128u}) {
        for (int bps : {0, per_sm_max - 1}) {  // 0: as many blocks as fit
            if (bps < 0) continue;
            for (uint32_t don : {0u, 1u}) {  // donate when warps idle / whenever a slot is free
                ctx->seed_chunk = chunk;
                ctx->blocks_per_sm = (uint32_t)bps;
                ctx->donation = don;
                double ms = 0;
                GJ_TRY(timed(GJ_ENGINE_FUSED, &ms));
                if (ms < best_f) {
                    best_f = ms;
                    best_chunk = chunk;
                    best_bps = (uint32_t)bps;
                    best_don = don;
                }
            }
        }
    }
    ctx->seed_chunk = best_chunk;
    ctx->blocks_per_sm = best_bps;
    ctx->donation = best_don;
    // plain engine: prefix-buffer budget, at most prefix_cap_bytes
    if (!prefix_cap_bytes) prefix_cap_bytes = 2ull << 30;
    double best_p = 1e300;
    uint64_t best_bytes = 0;
    for (uint64_t bytes : {64ull << 20, 256ull << 20, 1ull << 30, 2ull << 30}) {
        if (bytes > prefix_cap_bytes) continue;
        ctx->opt.prefix_buffer_bytes = bytes;
        double ms = 0;
        GJ_TRY(timed(GJ_ENGINE_PLAIN, &ms));
        if (ms < best_p) {
            best_p = ms;
            best_bytes = bytes;
        }
    }
    if (best_bytes) ctx->opt.prefix_buffer_bytes = best_bytes;
    GJ_TRY(gj_get_tuning(ctx, out));
    out->fused_ms = best_f;
    out->plain_ms = best_bytes ? best_p : 0;
    return GJ_OK;
}

}  // namespace

extern "C" {

int gj_last_work(const gj_ctx* ctx, gj_work_stats* out) {
    if (!ctx || !out) return GJ_E_INVALID;
    *out = ctx->work;
    return GJ_OK;
}

int gj_count(gj_graph* g, const gj_query* q, int64_t* count, uint64_t* checksum) {
    if (!g) return GJ_E_INVALID;
    return gj_count_ex(g, q, g->ctx->opt.engine, 0, UINT32_MAX, count, checksum, nullptr);
}

int gj_apply_batch(gj_graph* g, const uint32_t* src, const uint32_t* dst, const int8_t* sign, uint64_t b,
                   const gj_query* const* qs, uint32_t nq, int64_t* delta_count, uint64_t* delta_checksum) {
    if (!g || (b && (!src || !dst || !sign)) || (nq && (!qs || !delta_count || !delta_checksum)) || b > UINT32_MAX)
        return GJ_E_INVALID;
    for (uint32_t i = 0; i < nq; i++)
        if (!qs[i] || qs[i]->ctx != g->ctx) return GJ_E_INVALID;
    gj_ctx* ctx = g->ctx;
    if (ctx->server) return GJ_E_INVALID;
    for (uint32_t i = 0; i < nq; i++)
        if (qs[i]->ntri) {
            gj_set_error(ctx, GJ_E_INVALID, "update batch: queries with tri atoms have no delta queries");
            return GJ_E_INVALID;
        }
    DevSet ds(ctx->device);
    std::lock_guard<std::mutex> lk(ctx->mu);
    GJ_RANGE("gj_apply_batch (%llu updates, %u queries)", (unsigned long long)b, nq);
    DeltaBuf buf;
    // the deltas go to the caller's arrays only once the batch is committed
    std::vector<int64_t> dc(nq);
    std::vector<uint64_t> dh(nq);
    int rc = gj_delta_prepare(ctx, g, src, dst, sign, b, &buf);
    if (rc == GJ_OK) rc = gj_delta_eval(ctx, g, buf.batch, qs, nq,
                                         gj_delta_engine(ctx, buf.batch.n),
                                         dc.data(), dh.data());
    gj_work_stats sum = ctx->work;
    const uint64_t changes = buf.batch.n;
    if (rc == GJ_OK) rc = gj_check_status(ctx);  // the batch is not committed after a failed check
    if (rc == GJ_OK) rc = gj_delta_commit(ctx, g, buf.batch);
    gj_delta_free(ctx, &buf);
    if (rc == GJ_OK) {
        GJ_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
        g->last_changes = changes;
        ctx->work = sum;
        for (uint32_t i = 0; i < nq; i++) {
            delta_count[i] = dc[i];
            delta_checksum[i] = dh[i];
        }
    }
    return rc;
}

}  // extern "C"

int gj_delta_eval(gj_ctx* ctx, const gj_graph* g, const DeltaBatch& batch, const gj_query* const* qs, uint32_t nq,
                  uint32_t engine, int64_t* counts, uint64_t* checksums) {
    GJ_RANGE("delta: evaluate %u delta queries (%s engine)", nq, engine == GJ_ENGINE_FUSED ? "fused" : "level-synchronous");
    for (uint32_t qi = 0; qi < nq; qi++) {
        counts[qi] = 0;
        checksums[qi] = 0;
    }
    memset(&ctx->work, 0, sizeof(ctx->work));
    if (batch.n == 0 || nq == 0) return GJ_OK;
    if (engine == GJ_ENGINE_FUSED) {
        std::vector<Plan> plans;
        std::vector<uint32_t> owner;
        for (uint32_t qi = 0; qi < nq; qi++)
            for (uint32_t i = 0; i < qs[qi]->natoms; i++) {
                plans.push_back(qs[qi]->dplan[i]);
                owner.push_back(qi);
            }
        std::vector<int64_t> c(plans.size());
        std::vector<uint64_t> h(plans.size());
        GJ_TRY(gj_engine_fused_delta(ctx, g, batch, plans.data(), (uint32_t)plans.size(), c.data(), h.data()));
        for (size_t p = 0; p < plans.size(); p++) {
            counts[owner[p]] += c[p];
            checksums[owner[p]] += h[p];
        }
        return GJ_OK;
    }
    gj_work_stats sum{};
    for (uint32_t qi = 0; qi < nq; qi++) {
        const gj_query* q = qs[qi];
        for (uint32_t i = 0; i < q->natoms; i++) {
            int64_t ci = 0;
            uint64_t hi = 0;
            GJ_TRY(gj_engine_plain_plan(ctx, g, q->dplan[i], 0, UINT32_MAX, &batch, &ci, &hi, nullptr, 0, nullptr));
            counts[qi] += ci;
            checksums[qi] += hi;
            const gj_work_stats& w = ctx->work;
            sum.seeds += w.seeds;
            for (int j = 0; j < 9; j++) {
                sum.extended[j] += w.extended[j];
                sum.nbind[j] += w.nbind[j];
                sum.proposals[j] += w.proposals[j];
                sum.produced[j] += w.produced[j];
            }
        }
    }
    ctx->work = sum;
    return GJ_OK;
}

extern "C" {

int gj_graph_last_batch(const gj_graph* g, uint64_t* changes) {
    if (!g || !changes) return GJ_E_INVALID;
    *changes = g->last_changes;
    return GJ_OK;
}

int gj_list(gj_graph* g, const gj_query* q, uint32_t* out_tuples, uint64_t cap, uint64_t* written, int64_t* total,
            uint64_t* checksum) {
    if (!g || !q || !written || !total || !checksum || (cap && !out_tuples) || q->ctx != g->ctx)
        return GJ_E_INVALID;
    gj_ctx* ctx = g->ctx;
    if (ctx->server) return GJ_E_INVALID;
    DevSet ds(ctx->device);
    std::lock_guard<std::mutex> lk(ctx->mu);
    GJ_TRY(ensure_tri(ctx, g, &q, 1));
    int64_t c = 0;
    uint64_t h = 0;
    GJ_TRY(gj_engine_plain(ctx, g, q, 0, UINT32_MAX, &c, &h, out_tuples, cap, written));
    GJ_TRY(gj_check_status(ctx));
    *total = c;
    *checksum = h;
    return (uint64_t)c > cap ? GJ_E_TRUNCATED : GJ_OK;
}

}  // extern "C"
