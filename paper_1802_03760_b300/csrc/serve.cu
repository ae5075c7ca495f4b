// Request loop for serving count requests and update batches on one graph.
//
// A host thread takes requests in submission order. Count requests at the
// head of the queue are merged into one wave: a single fused persistent
// launch over all their queries on the count stream (continuous batching:
// whatever arrived while the previous wave ran joins the next one). An
// update batch at the head runs on the context's stream while earlier waves
// are still executing: it normalises the batch, evaluates the delta queries
// on the current version and builds the next version's index in new memory;
// waves already in flight keep reading the previous index, which is freed
// only after they complete. Every request therefore sees exactly the
// versions it would see if the requests ran one by one in submission order.
// Requests are admitted against a device-memory budget; a request that can
// never fit is failed with GJ_E_ADMIT.
#include <algorithm>

#include "gj_internal.cuh"

#include <chrono>
#include <condition_variable>
#include <deque>
#include <thread>
#include <unordered_map>

namespace {

enum { REQ_COUNT = 0, REQ_BATCH = 1 };

struct Request {
    uint64_t id = 0;
    uint32_t kind = REQ_COUNT;
    std::vector<const gj_query*> qs;
    std::vector<uint32_t> src, dst;
    std::vector<int8_t> sign;
    bool done = false;
    int status = GJ_E_PENDING;
    std::vector<int64_t> counts;
    std::vector<uint64_t> chks;
    uint64_t version = 0;
    double t_submit = 0, t_start = 0, t_end = 0;
};

struct Wave {
    std::vector<Request*> reqs;
    void* dscratch = nullptr;
    unsigned long long* dres = nullptr;
    unsigned long long* hres = nullptr;  // pinned
    cudaEvent_t done = nullptr;
    size_t mem = 0;
    uint64_t version = 0;
    uint32_t nq = 0;
};

struct Retired {
    gj_csr fwd, rev;
    std::vector<cudaEvent_t> waits;  // completion events of the waves that read it
};

}  // namespace

struct gj_server {
    gj_ctx* ctx = nullptr;
    gj_graph* g = nullptr;
    uint64_t budget = 0;
    uint64_t in_use = 0;
    std::thread th;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request*> pending;
    std::unordered_map<uint64_t, Request*> reqs;
    uint64_t next_id = 1;
    bool stop = false;
    cudaStream_t s_count = nullptr;
    std::vector<Wave*> inflight;
    std::vector<Retired> retired;
    std::chrono::steady_clock::time_point t0;
    double now() const {
        return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace {

constexpr uint32_t WAVE_MAX_QUERIES = 64;

size_t batch_need(const gj_graph* g, uint64_t b) {
    // batch arena + the next version's index + the index build's temporaries
    return 128 * (size_t)(b + 1) + 80 * (size_t)(g->m + b) + 32 * ((size_t)g->n + 1);
}

void finish(gj_server* S, Request* r, int status) {
    r->status = status;
    r->t_end = S->now();
    r->done = true;
}

// A retired index that no wave reads any more becomes the graph's spare
// arrays (the next commit writes the next version into them) when it has
// none; otherwise it is freed. Reusing it avoids a cudaFree, which would
// wait for every wave in flight, and the next commit's allocations.
void keep_or_release(gj_graph* g, Retired& rt) {
    if (!g->spare_fwd.off && !g->spare_rev.off) {
        g->spare_fwd = rt.fwd;
        g->spare_rev = rt.rev;
    } else {
        gj_csr_release(rt.fwd);
        gj_csr_release(rt.rev);
    }
    rt.fwd = gj_csr{};
    rt.rev = gj_csr{};
}

// Completes the waves whose launch finished; frees retired indices no wave reads.
void reap(gj_server* S) {
    for (size_t i = 0; i < S->inflight.size();) {
        Wave* w = S->inflight[i];
        cudaError_t q = cudaEventQuery(w->done);
        if (q == cudaErrorNotReady) {
            i++;
            continue;
        }
        int st = (q == cudaSuccess) ? GJ_OK : GJ_E_CUDA;
        if (q != cudaSuccess) cudaGetLastError();
        // the wave's flags: its donation queue's bounded wait gave up, a
        // count passed 2^63 - 1 (not known which: every request of the wave
        // is refused)
        const bool gave_up = st == GJ_OK && w->hres[2 * (size_t)w->nq] != 0;
        const bool wave_ovf = st == GJ_OK && w->hres[2 * (size_t)w->nq + 1] != 0;
        if (gave_up) st = GJ_E_TIMEOUT;
        uint32_t o = 0;
        {
            std::lock_guard<std::mutex> lk(S->mu);
            for (Request* r : w->reqs) {
                const uint32_t nq = (uint32_t)r->qs.size();
                r->counts.resize(nq);
                r->chks.resize(nq);
                bool ovf = false;
                for (uint32_t k = 0; k < nq; k++) {
                    r->counts[k] = (int64_t)w->hres[o + k];
                    r->chks[k] = w->hres[w->nq + o + k];
                    ovf = ovf || r->counts[k] < 0;  // a count past 2^63 - 1
                }
                o += nq;
                r->version = w->version;
                finish(S, r, (st == GJ_OK && (ovf || wave_ovf)) ? GJ_E_OVERFLOW : st);
            }
            S->in_use -= w->mem;
        }
        S->cv_done.notify_all();
        cudaFreeAsync(w->dscratch, S->s_count);
        cudaFreeHost(w->hres);
        // keep the event alive while a retired index still lists it
        bool referenced = false;
        for (Retired& rt : S->retired)
            for (cudaEvent_t e : rt.waits) referenced |= (e == w->done);
        if (!referenced) cudaEventDestroy(w->done);
        delete w;
        S->inflight.erase(S->inflight.begin() + i);
    }
    for (size_t i = 0; i < S->retired.size();) {
        Retired& rt = S->retired[i];
        bool ready = true;
        for (cudaEvent_t e : rt.waits) ready &= (cudaEventQuery(e) != cudaErrorNotReady);
        if (!ready) {
            i++;
            continue;
        }
        keep_or_release(S->g, rt);
        std::vector<cudaEvent_t> ws = rt.waits;
        S->retired.erase(S->retired.begin() + i);
        for (cudaEvent_t e : ws) {
            bool still = false;
            for (Wave* w : S->inflight) still |= (w->done == e);
            for (Retired& o : S->retired)
                for (cudaEvent_t x : o.waits) still |= (x == e);
            if (!still) cudaEventDestroy(e);
        }
    }
}

// Launches the count requests at the head of the queue as one wave. Returns
// false if the head is not a count request or the wave does not fit yet.
bool launch_wave(gj_server* S) {
    std::vector<Request*> take;
    std::vector<Plan> plans;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        uint32_t nq = 0;
        while (!S->pending.empty() && S->pending.front()->kind == REQ_COUNT) {
            Request* r = S->pending.front();
            if (nq + r->qs.size() > WAVE_MAX_QUERIES && nq > 0) break;
            const size_t need = gj_fused_wave_bytes(nq + (uint32_t)r->qs.size());
            if (S->in_use + need > S->budget && !take.empty()) break;
            if (S->in_use + need > S->budget && !S->inflight.empty()) break;
            S->pending.pop_front();
            take.push_back(r);
            nq += (uint32_t)r->qs.size();
        }
        if (take.empty()) return false;
        for (Request* r : take) {
            r->t_start = S->now();
            for (const gj_query* q : r->qs) plans.push_back(q->plan);
        }
    }
    GJ_RANGE("serve: wave of %zu requests", take.size());
    Wave* w = new Wave();
    w->reqs = take;
    w->nq = (uint32_t)plans.size();
    w->mem = gj_fused_wave_bytes(w->nq);
    w->version = S->g->version;
    gj_ctx* ctx = S->ctx;
    int rc = GJ_OK;
    if (gj_malloc_async(ctx, &w->dscratch, w->mem, S->s_count) != cudaSuccess ||
        cudaMallocHost(&w->hres, 16 * (size_t)w->nq + 16) != cudaSuccess ||
        cudaEventCreateWithFlags(&w->done, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        rc = GJ_E_NOMEM;
    }
    if (rc == GJ_OK) rc = gj_fused_enqueue(ctx, S->g->view(), plans.data(), w->nq, S->s_count, w->dscratch, &w->dres);
    if (rc == GJ_OK &&
        cudaMemcpyAsync(w->hres, w->dres, 16 * (size_t)w->nq + 16, cudaMemcpyDeviceToHost, S->s_count) != cudaSuccess)
        rc = GJ_E_CUDA;
    if (rc == GJ_OK && cudaEventRecord(w->done, S->s_count) != cudaSuccess) rc = GJ_E_CUDA;
    if (rc != GJ_OK) {
        std::lock_guard<std::mutex> lk(S->mu);
        for (Request* r : take) finish(S, r, rc);
        if (w->dscratch) cudaFreeAsync(w->dscratch, S->s_count);
        if (w->hres) cudaFreeHost(w->hres);
        if (w->done) cudaEventDestroy(w->done);
        delete w;
        S->cv_done.notify_all();
        return true;
    }
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->in_use += w->mem;
    }
    S->inflight.push_back(w);
    return true;
}

// Runs the update batch at the head of the queue (if it fits), overlapping
// with the waves in flight. Returns false if it must wait for memory.
bool run_batch(gj_server* S) {
    Request* r;
    size_t need;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->pending.empty() || S->pending.front()->kind != REQ_BATCH) return false;
        r = S->pending.front();
        need = batch_need(S->g, r->src.size());
        if (need > S->budget) {
            S->pending.pop_front();
            finish(S, r, GJ_E_ADMIT);
            S->cv_done.notify_all();
            return true;
        }
        if (S->in_use + need > S->budget && !S->inflight.empty()) return false;
        S->pending.pop_front();
        S->in_use += need;
        r->t_start = S->now();
    }
    gj_ctx* ctx = S->ctx;
    gj_graph* g = S->g;
    const uint32_t nq = (uint32_t)r->qs.size();
    GJ_RANGE("serve: update batch of %zu", r->src.size());
    std::vector<int64_t> c(nq, 0);
    std::vector<uint64_t> h(nq, 0);
    DeltaBuf buf;
    int rc = gj_delta_prepare(ctx, g, r->src.data(), r->dst.data(), r->sign.data(), r->src.size(), &buf);
    if (rc == GJ_OK) rc = gj_delta_eval(ctx, g, buf.batch, r->qs.data(), nq,
                                         gj_delta_engine(ctx, buf.batch.n),
                                         c.data(), h.data());
    Retired rt;
    const uint64_t changes = buf.batch.n;
    if (rc == GJ_OK) rc = gj_delta_commit(ctx, g, buf.batch, &rt.fwd, &rt.rev);
    gj_delta_free(ctx, &buf);
    if (rc == GJ_OK) {
        cudaStreamSynchronize(ctx->stream);
        g->last_changes = changes;
        if (rt.fwd.off) {
            for (Wave* w : S->inflight) rt.waits.push_back(w->done);
            if (rt.waits.empty()) {
                keep_or_release(g, rt);
            } else {
                S->retired.push_back(rt);
            }
        }
    }
    {
        std::lock_guard<std::mutex> lk(S->mu);
        r->counts = c;
        r->chks = h;
        r->version = g->version;
        finish(S, r, rc);
        S->in_use -= need;
    }
    S->cv_done.notify_all();
    return true;
}

void loop(gj_server* S) {
    cudaSetDevice(S->ctx->device);
    while (true) {
        {
            std::unique_lock<std::mutex> lk(S->mu);
            if (S->pending.empty() && S->inflight.empty()) {
                if (S->stop) break;
                S->cv_work.wait_for(lk, std::chrono::milliseconds(50));
                continue;
            }
        }
        reap(S);
        bool progressed = launch_wave(S);
        if (!progressed) progressed = run_batch(S);
        if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    for (Retired& rt : S->retired) {
        gj_csr_release(rt.fwd);
        gj_csr_release(rt.rev);
    }
    S->retired.clear();
}

}  // namespace

extern "C" {

int gj_serve_start(gj_ctx* ctx, gj_graph* g, uint64_t memory_budget_bytes) {
    if (!ctx || !g || g->ctx != ctx) return GJ_E_INVALID;
    if (ctx->server) {
        gj_set_error(ctx, GJ_E_INVALID, "already serving");
        return GJ_E_INVALID;
    }
    cudaSetDevice(ctx->device);
    GJ_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    gj_server* S = new (std::nothrow) gj_server();
    if (!S) return GJ_E_NOMEM;
    S->ctx = ctx;
    S->g = g;
    if (memory_budget_bytes == 0) {
        size_t fr = 0, tot = 0;
        cudaMemGetInfo(&fr, &tot);
        memory_budget_bytes = (uint64_t)(0.8 * (double)fr);
    }
    S->budget = memory_budget_bytes;
    S->t0 = std::chrono::steady_clock::now();
    if (cudaStreamCreateWithFlags(&S->s_count, cudaStreamNonBlocking) != cudaSuccess) {
        delete S;
        return GJ_E_CUDA;
    }
    ctx->server = S;
    S->th = std::thread(loop, S);
    return GJ_OK;
}

int gj_serve_stop(gj_ctx* ctx) {
    if (!ctx || !ctx->server) return GJ_E_INVALID;
    gj_server* S = ctx->server;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    S->th.join();
    cudaStreamSynchronize(S->s_count);
    cudaStreamDestroy(S->s_count);
    for (auto& kv : S->reqs) delete kv.second;
    delete S;
    ctx->server = nullptr;
    return GJ_OK;
}

int gj_submit_count(gj_ctx* ctx, const gj_query* const* qs, uint32_t nq, uint64_t* req_id) {
    if (!ctx || !ctx->server || !qs || !req_id || nq == 0 || nq > WAVE_MAX_QUERIES) return GJ_E_INVALID;
    gj_server* S = ctx->server;
    Request* r = new (std::nothrow) Request();
    if (!r) return GJ_E_NOMEM;
    for (uint32_t i = 0; i < nq; i++) {
        if (!qs[i] || qs[i]->ctx != ctx || qs[i]->ntri) {  // the triangle index is not versioned: no tri atoms
            delete r;
            return GJ_E_INVALID;
        }
        r->qs.push_back(qs[i]);
    }
    r->kind = REQ_COUNT;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        r->id = S->next_id++;
        r->t_submit = S->now();
        S->reqs[r->id] = r;
        S->pending.push_back(r);
    }
    S->cv_work.notify_all();
    *req_id = r->id;
    return GJ_OK;
}

int gj_submit_batch(gj_ctx* ctx, const uint32_t* src, const uint32_t* dst, const int8_t* sign, uint64_t b,
                    const gj_query* const* qs, uint32_t nq, uint64_t* req_id) {
    if (!ctx || !ctx->server || !req_id || (b && (!src || !dst || !sign)) || (nq && !qs) ||
        nq > WAVE_MAX_QUERIES || b > UINT32_MAX)
        return GJ_E_INVALID;
    gj_server* S = ctx->server;
    Request* r = new (std::nothrow) Request();
    if (!r) return GJ_E_NOMEM;
    for (uint32_t i = 0; i < nq; i++) {
        if (!qs[i] || qs[i]->ctx != ctx || qs[i]->ntri) {  // the triangle index is not versioned: no tri atoms
            delete r;
            return GJ_E_INVALID;
        }
        r->qs.push_back(qs[i]);
    }
    r->kind = REQ_BATCH;
    r->src.resize(b);
    r->dst.resize(b);
    r->sign.resize(b);
    // the caller's arrays may be reused once this returns: copy them (host or device)
    if (b) {
        if (cudaMemcpy(r->src.data(), src, 4 * b, cudaMemcpyDefault) != cudaSuccess ||
            cudaMemcpy(r->dst.data(), dst, 4 * b, cudaMemcpyDefault) != cudaSuccess ||
            cudaMemcpy(r->sign.data(), sign, b, cudaMemcpyDefault) != cudaSuccess) {
            cudaGetLastError();
            delete r;
            return GJ_E_CUDA;
        }
    }
    {
        std::lock_guard<std::mutex> lk(S->mu);
        r->id = S->next_id++;
        r->t_submit = S->now();
        S->reqs[r->id] = r;
        S->pending.push_back(r);
    }
    S->cv_work.notify_all();
    *req_id = r->id;
    return GJ_OK;
}

int gj_cancel(gj_ctx* ctx, uint64_t req_id) {
    if (!ctx || !ctx->server) return GJ_E_INVALID;
    gj_server* S = ctx->server;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->reqs.find(req_id);
        if (it == S->reqs.end()) return GJ_E_NOTFOUND;
        Request* r = it->second;
        auto p = std::find(S->pending.begin(), S->pending.end(), r);
        if (p == S->pending.end()) return GJ_E_PENDING;  // started or finished: it runs to its end
        S->pending.erase(p);
        r->t_start = S->now();
        finish(S, r, GJ_E_CANCELLED);
    }
    S->cv_done.notify_all();
    return GJ_OK;
}

int gj_poll(gj_ctx* ctx, uint64_t req_id, int wait_ms, gj_result* out) {
    if (!ctx || !ctx->server || !out) return GJ_E_INVALID;
    gj_server* S = ctx->server;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(req_id);
    if (it == S->reqs.end()) return GJ_E_NOTFOUND;
    Request* r = it->second;
    if (!r->done && wait_ms != 0) {
        auto pred = [&] { return r->done; };
        if (wait_ms < 0) S->cv_done.wait(lk, pred);
        else S->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), pred);
    }
    if (!r->done) return GJ_E_PENDING;
    memset(out, 0, sizeof(*out));
    out->req_id = r->id;
    out->status = r->status;
    out->kind = r->kind;
    out->nq = (uint32_t)r->qs.size();
    for (uint32_t i = 0; i < out->nq && i < r->counts.size(); i++) {
        out->counts[i] = r->counts[i];
        out->checksums[i] = r->chks[i];
    }
    out->version = r->version;
    out->submit_ms = r->t_submit;
    out->start_ms = r->t_start;
    out->end_ms = r->t_end;
    S->reqs.erase(it);
    delete r;
    return GJ_OK;
}

}  // extern "C"
