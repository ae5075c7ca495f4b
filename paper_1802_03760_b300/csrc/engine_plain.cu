// Plain engine: level-synchronous Generic Join, one query at a time.
//
// Every level j (prefixes of length j, extended by x_j) keeps a bounded
// prefix buffer. The steps of the dataflow primitive (Section 3.1.1) are
// separate kernels: Count computes, per prefix, the smallest extension-set
// size min-c and the atom that has it (min-i); an exclusive scan of min-c
// lays the candidates of all prefixes of the level out on one line; Propose
// + Intersect takes a window of that line (at most the next level's buffer
// capacity, Section 3.1.2's batch of proposals, the window start being the
// rem-ext cursor), resolves each candidate to its prefix and its element of
// the min-i list, tests membership in every other binding list, and appends
// survivors to the next level's buffer (or counts and hashes them at the
// last level). After each launch the host reads the sizes back and picks
// the deepest level with pending candidates (Section 3.2).
//
// The same kernels evaluate delta queries dQ_i (Section 3.3.1, Section 4.3):
// the seeds are a batch's signed changes, each atom reads the old or the
// new version of the graph, and every prefix carries its seed's sign.
#include "gj_internal.cuh"

namespace {

constexpr int PT = 256;  // threads per block

struct Cols {
    uint32_t* x[GJ_MAX_K];
    int8_t* sg;  // sign of the seed each prefix descends from (delta queries)
    uint64_t cap;  // slots of each column
};

struct Acc {
    unsigned long long* count;
    unsigned long long* chk;
    unsigned long long* n_out;  // append cursor of the next level's buffer
    unsigned long long* tup;    // slot cursor of listed matches
};

// H of the match whose value at position p is xs[p] (position p binds query
// attribute P.order[p]).
__device__ __forceinline__ uint64_t hash_positions(const Plan& P, const uint32_t* xs) {
    uint64_t h = gj_hq(P.k);
    for (uint32_t p = 0; p < P.k; p++) h *= gj_hf(P.order[p], xs[p]);
    return h;
}

__device__ __forceinline__ void warp_add(unsigned long long* dst, unsigned long long v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(dst, v);
}

// Reads seeds [e_lo, e_hi) and keeps those that pass the other atoms over
// (x0, x1). Static plans read the seed atom's index slots; delta plans read
// the batch's changes (sorted (src, dst) pairs with signs). k == 2 counts
// the seeds as matches.
__global__ void __launch_bounds__(PT) k_seed(Plan P, GraphView G, DeltaView D, DeltaBatch B, int64_t e_lo,
                                             int64_t e_hi, Cols out, Acc acc, int emit, uint32_t* __restrict__ tuples,
                                             uint64_t cap) {
    const int lane = threadIdx.x & 31;
    const uint32_t lt = gj_lanemask_lt();
    const DeltaView* Dv = P.delta ? &D : nullptr;
    const uint32_t* key = P.seed_dir ? G.rk : G.fk;
    const uint32_t* nbr = P.seed_dir ? G.rn : G.fn;
    unsigned long long cnt = 0, chk = 0;
    const int64_t stride = (int64_t)gridDim.x * PT;
    for (int64_t base = e_lo + (int64_t)blockIdx.x * PT + (threadIdx.x & ~31); base < e_hi; base += stride) {
        int64_t e = base + lane;
        bool keep = e < e_hi;
        uint32_t x0 = 0, x1 = 0;
        int sign = 1;
        if (keep) {
            if (P.delta) {
                x0 = B.chg_src[e];
                x1 = B.chg_dst[e];
                sign = B.chg_sign[e];
            } else {
                x0 = __ldg(key + e);
                x1 = __ldg(nbr + e);
            }
            for (uint32_t f = 0; f < P.nsf && keep; f++) {
                uint32_t u = P.sf_dir[f] ? x1 : x0, w = P.sf_dir[f] ? x0 : x1;
                keep = gj_view_member(G, Dv, 0, P.sf_view[f], u, w);
            }
            keep = keep && gj_lt_ok(P, 1, x1, [&](uint32_t) { return x0; });
        }
        if (emit) {
            if (keep) {
                uint32_t xs[2] = {x0, x1};
                const uint64_t h = hash_positions(P, xs);
                cnt += (unsigned long long)(long long)sign;
                chk += sign > 0 ? h : 0ull - h;
                if (tuples) {
                    unsigned long long slot = atomicAdd(acc.tup, 1ull);
                    if (slot < cap) {
                        tuples[slot * 2 + P.order[0]] = x0;
                        tuples[slot * 2 + P.order[1]] = x1;
                    }
                }
            }
            continue;
        }
        uint32_t mask = __ballot_sync(0xffffffffu, keep);
        if (!mask) continue;
        int leader = __ffs(mask) - 1;
        unsigned long long b0 = 0;
        if (lane == leader) b0 = atomicAdd(acc.n_out, (unsigned long long)__popc(mask));
        b0 = __shfl_sync(0xffffffffu, b0, leader);
        if (keep && GJ_CHECK(G.chk, b0 + __popc(mask & lt) < out.cap, GJ_SITE_PREFIX, b0 + __popc(mask & lt))) {
            uint64_t s = b0 + __popc(mask & lt);
            out.x[0][s] = x0;
            out.x[1][s] = x1;
            if (out.sg) out.sg[s] = (int8_t)sign;
        }
    }
    if (emit) {
        warp_add(acc.count, cnt);
        warp_add(acc.chk, chk);
    }
}

// Count: min-c and min-i of every prefix of a level (ties: first binding
// atom). cnt is the size of the chosen list's enumeration space (for a new
// view that includes the batch's deletions, which Propose skips).
__global__ void __launch_bounds__(PT) k_count(Plan P, GraphView G, DeltaView D, uint32_t j, Cols in, uint64_t n,
                                              uint32_t* __restrict__ cnt, uint8_t* __restrict__ mini) {
    const DeltaView* Dv = P.delta ? &D : nullptr;
    const uint64_t stride = (uint64_t)gridDim.x * PT;
    for (uint64_t i = (uint64_t)blockIdx.x * PT + threadIdx.x; i < n; i += stride) {
        uint32_t best = 0xffffffffu, space = 0, bi = 0;
        for (uint32_t b = 0; b < P.nb[j]; b++) {
            const uint32_t v = in.x[P.bpos[j][b]][i];
            uint32_t deg, sp;
            if (P.bdir[j][b] == GJ_BIND_TRI) {  // static plans only
                deg = sp = gj_bind_list(G, GJ_BIND_TRI, v, in.x[P.bpos2[j][b]][i]).len;
            } else {
                const ViewList L = gj_view_list(G, Dv, P.bdir[j][b], P.bview[j][b], v);
                deg = L.degree();
                sp = L.space();
            }
            if (deg < best) {
                best = deg;
                space = sp;
                bi = b;
            }
        }
        cnt[i] = space;
        mini[i] = (uint8_t)bi;
    }
}

// Propose + Intersect over candidates [c_lo, c_hi) of level j.
__global__ void __launch_bounds__(PT) k_extend(Plan P, GraphView G, DeltaView D, uint32_t j, Cols in, uint64_t n,
                                               const int64_t* __restrict__ coff, const uint8_t* __restrict__ mini,
                                               int64_t c_lo, int64_t c_hi, int last, Cols out, Acc acc,
                                               uint32_t* __restrict__ tuples, uint64_t cap) {
    const int lane = threadIdx.x & 31;
    const uint32_t lt = gj_lanemask_lt();
    const DeltaView* Dv = P.delta ? &D : nullptr;
    unsigned long long cnt = 0, chk = 0;
    const int64_t stride = (int64_t)gridDim.x * PT;
    for (int64_t base = c_lo + (int64_t)blockIdx.x * PT + (threadIdx.x & ~31); base < c_hi; base += stride) {
        int64_t t = base + lane;
        bool keep = t < c_hi;
        uint32_t xs[GJ_MAX_K];
        uint64_t i = 0;
        int sign = 1;
        if (keep) {
            // the prefix whose candidate range holds t: last i with coff[i] <= t
            uint64_t lo = 0, hi = n;
            while (hi - lo > 1) {
                uint64_t mid = (lo + hi) >> 1;
                if (__ldg(coff + mid) <= t) lo = mid; else hi = mid;
            }
            i = lo;
            const uint32_t r = (uint32_t)(t - __ldg(coff + i));
            const uint32_t b = mini[i];
            for (uint32_t p = 0; p < j; p++) xs[p] = in.x[p][i];
            if (in.sg) sign = in.sg[i];
            uint32_t e = 0;
            if (P.bdir[j][b] == GJ_BIND_TRI) {
                const BindList L = gj_bind_list(G, GJ_BIND_TRI, xs[P.bpos[j][b]], xs[P.bpos2[j][b]]);
                if (GJ_CHECK(G.chk, r < L.len, GJ_SITE_LIST, r)) e = __ldg(L.p + r);
                else keep = false;
            } else {
                const ViewList L = gj_view_list(G, Dv, P.bdir[j][b], P.bview[j][b], xs[P.bpos[j][b]]);
                if (GJ_CHECK(G.chk, r < L.space(), GJ_SITE_LIST, r)) {
                    e = r < L.base_len ? __ldg(L.base + r) : __ldg(L.ins + (r - L.base_len));
                    if (r < L.base_len && L.ndel) keep = !gj_contains(L.del, L.ndel, e);  // deleted in the new version
                } else {
                    keep = false;
                }
            }
            xs[j] = e;
            for (uint32_t bb = 0; bb < P.nb[j] && keep; bb++) {
                if (bb == b) continue;
                if (P.bdir[j][bb] == GJ_BIND_TRI)
                    keep = gj_bind_member(gj_bind_list(G, GJ_BIND_TRI, xs[P.bpos[j][bb]], xs[P.bpos2[j][bb]]), e);
                else
                    keep = gj_view_member(G, Dv, P.bdir[j][bb], P.bview[j][bb], xs[P.bpos[j][bb]], e);
            }
            if (keep && P.nlt[j]) keep = gj_lt_ok(P, j, e, [&](uint32_t p) { return xs[p]; });
        }
        if (last) {
            if (keep) {
                const uint64_t h = hash_positions(P, xs);
                cnt += (unsigned long long)(long long)sign;
                chk += sign > 0 ? h : 0ull - h;
                if (tuples) {
                    unsigned long long slot = atomicAdd(acc.tup, 1ull);
                    if (slot < cap)
                        for (uint32_t p = 0; p < P.k; p++) tuples[slot * P.k + P.order[p]] = xs[p];
                }
            }
            continue;
        }
        uint32_t mask = __ballot_sync(0xffffffffu, keep);
        if (!mask) continue;
        int leader = __ffs(mask) - 1;
        unsigned long long b0 = 0;
        if (lane == leader) b0 = atomicAdd(acc.n_out, (unsigned long long)__popc(mask));
        b0 = __shfl_sync(0xffffffffu, b0, leader);
        if (keep && GJ_CHECK(G.chk, b0 + __popc(mask & lt) < out.cap, GJ_SITE_PREFIX, b0 + __popc(mask & lt))) {
            uint64_t s = b0 + __popc(mask & lt);
            for (uint32_t p = 0; p <= j; p++) out.x[p][s] = xs[p];
            if (out.sg) out.sg[s] = (int8_t)sign;
        }
    }
    if (last) {
        warp_add(acc.count, cnt);
        warp_add(acc.chk, chk);
    }
}

struct Level {
    Cols cols{};
    uint32_t* cnt = nullptr;
    uint8_t* mini = nullptr;
    int64_t* coff = nullptr;
    uint64_t n = 0;
    int64_t total = 0;
    int64_t cursor = 0;
};

}  // namespace

int gj_engine_plain_plan(gj_ctx* ctx, const gj_graph* g, const Plan& P, uint32_t v_lo, uint32_t v_hi,
                         const DeltaBatch* delta, int64_t* count, uint64_t* checksum, uint32_t* out_tuples,
                         uint64_t cap, uint64_t* written) {
    const uint32_t k = P.k;
    cudaStream_t st = ctx->stream;
    GraphView G = g->view();
    DeltaView D = delta ? delta->view : DeltaView{};
    DeltaBatch B = delta ? *delta : DeltaBatch{};
    gj_work_stats& W = ctx->work;
    memset(&W, 0, sizeof(W));

    int64_t se[2] = {0, 0};
    if (P.delta) {
        se[1] = (int64_t)B.n;
    } else {
        if (v_hi > g->n) v_hi = g->n;
        if (v_lo > v_hi) v_lo = v_hi;
        // seed edge range: the index slots keyed by x0 in [v_lo, v_hi)
        const int64_t* soff = P.seed_dir ? g->rev.off : g->fwd.off;
        GJ_CUDA_TRY(ctx, cudaMemcpyAsync(&se[0], soff + v_lo, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        GJ_CUDA_TRY(ctx, cudaMemcpyAsync(&se[1], soff + v_hi, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        GJ_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    }

    // prefix buffers for levels 2..k-1, all with the same capacity
    uint64_t budget = ctx->opt.prefix_buffer_bytes ? ctx->opt.prefix_buffer_bytes : (512ull << 20);
    uint64_t per_slot = 0;
    for (uint32_t j = 2; j < k; j++) per_slot += 4ull * j + 4 + 1 + 8 + (P.delta ? 1 : 0);
    uint64_t capacity = per_slot ? budget / per_slot : 0;
    if (k > 2 && capacity < 1024) {
        gj_set_error(ctx, GJ_E_INVALID, "prefix_buffer_bytes too small");
        return GJ_E_INVALID;
    }
    if (capacity > (1ull << 31)) capacity = 1ull << 31;
    Level L[GJ_MAX_K];
    if (k > 2) {
        char* base = nullptr;
        GJ_TRY(gj_scratch(ctx, 0, per_slot * capacity + 16ull * (k + 1) * 256 + 4096, (void**)&base));
        auto take = [&](size_t bytes) {
            char* p = base;
            base += (bytes + 255) & ~(size_t)255;
            return (void*)p;
        };
        for (uint32_t j = 2; j < k; j++) {
            for (uint32_t p = 0; p < j; p++) L[j].cols.x[p] = (uint32_t*)take(4 * capacity);
            L[j].cols.sg = P.delta ? (int8_t*)take(capacity) : nullptr;
            L[j].cols.cap = capacity;
            L[j].cnt = (uint32_t*)take(4 * capacity);
            L[j].mini = (uint8_t*)take(capacity);
            L[j].coff = (int64_t*)take(8 * (capacity + 1));
        }
    }
    uint64_t window = ctx->opt.window ? ctx->opt.window : capacity;
    if (window > capacity && k > 2) window = capacity;

    unsigned long long* acc = (unsigned long long*)ctx->d_acc;
    GJ_CUDA_TRY(ctx, cudaMemsetAsync(acc, 0, 8 * sizeof(unsigned long long), st));
    Acc A{acc + 0, acc + 1, acc + 2, acc + 3};
    const unsigned grid = (unsigned)ctx->sm_count * 8;
    uint32_t* tuples = nullptr;
    if (out_tuples && cap) GJ_TRY(gj_scratch(ctx, 1, (size_t)cap * k * 4, (void**)&tuples));

    auto read_u64 = [&](unsigned long long* d, uint64_t* h) -> int {
        GJ_CUDA_TRY(ctx, cudaMemcpyAsync(h, d, 8, cudaMemcpyDeviceToHost, st));
        GJ_CUDA_TRY(ctx, cudaStreamSynchronize(st));
        return GJ_OK;
    };
    // count, scan and read back the candidate total of level j
    auto prepare = [&](uint32_t j) -> int {
        GJ_RANGE("level %u: count", j);
        Level& l = L[j];
        l.cursor = 0;
        l.total = 0;
        if (l.n == 0) return GJ_OK;
        k_count<<<gj_div_up(l.n, PT) < grid ? gj_div_up(l.n, PT) : grid, PT, 0, st>>>(P, G, D, j, l.cols, l.n, l.cnt,
                                                                                       l.mini);
        GJ_LAUNCHED(ctx);
        GJ_TRY(gj_scan_u32(ctx, l.cnt, l.coff, l.n));
        GJ_CUDA_TRY(ctx, cudaMemcpyAsync(&l.total, l.coff + l.n, 8, cudaMemcpyDeviceToHost, st));
        GJ_CUDA_TRY(ctx, cudaStreamSynchronize(st));
        W.extended[j] += (int64_t)l.n;
        W.nbind[j] += (int64_t)l.n * P.nb[j];
        W.proposals[j] += l.total;
        return GJ_OK;
    };

    W.seeds = se[1] - se[0];
    if (k == 2) {
        if (se[1] > se[0]) {
            gj_timer_begin(ctx);
            k_seed<<<grid, PT, 0, st>>>(P, G, D, B, se[0], se[1], Cols{}, A, 1, tuples, cap);
            GJ_LAUNCHED(ctx);
            gj_timer_end(ctx);
        }
    } else {
        int64_t seed_cursor = se[0];
        while (true) {
            int jd = -1;
            for (int j = (int)k - 1; j >= 2; j--)
                if (L[j].cursor < L[j].total) { jd = j; break; }
            if (jd < 0) {
                if (seed_cursor >= se[1]) break;
                int64_t chunk = se[1] - seed_cursor;
                if ((uint64_t)chunk > capacity) chunk = (int64_t)capacity;
                GJ_RANGE("level 2: seeds");
                GJ_CUDA_TRY(ctx, cudaMemsetAsync(A.n_out, 0, 8, st));
                k_seed<<<grid, PT, 0, st>>>(P, G, D, B, seed_cursor, seed_cursor + chunk, L[2].cols, A, 0, nullptr,
                                            0);
                GJ_LAUNCHED(ctx);
                GJ_CUDA_TRY(ctx, cudaGetLastError());
                seed_cursor += chunk;
                GJ_TRY(read_u64(A.n_out, &L[2].n));
                W.produced[2] += (int64_t)L[2].n;
                GJ_TRY(prepare(2));
                continue;
            }
            Level& l = L[jd];
            GJ_RANGE("level %d: propose and intersect", jd);
            if (jd == (int)k - 1) {
                gj_timer_begin(ctx);
                k_extend<<<grid, PT, 0, st>>>(P, G, D, jd, l.cols, l.n, l.coff, l.mini, l.cursor, l.total, 1, Cols{},
                                              A, tuples, cap);
                GJ_LAUNCHED(ctx);
                gj_timer_end(ctx);
                GJ_CUDA_TRY(ctx, cudaGetLastError());
                l.cursor = l.total;
                continue;
            }
            int64_t w = l.total - l.cursor;
            if ((uint64_t)w > window) w = (int64_t)window;
            GJ_CUDA_TRY(ctx, cudaMemsetAsync(A.n_out, 0, 8, st));
            k_extend<<<grid, PT, 0, st>>>(P, G, D, jd, l.cols, l.n, l.coff, l.mini, l.cursor, l.cursor + w, 0,
                                          L[jd + 1].cols, A, nullptr, 0);
            GJ_LAUNCHED(ctx);
            GJ_CUDA_TRY(ctx, cudaGetLastError());
            l.cursor += w;
            GJ_TRY(read_u64(A.n_out, &L[jd + 1].n));
            W.produced[jd + 1] += (int64_t)L[jd + 1].n;
            GJ_TRY(prepare(jd + 1));
        }
    }
    uint64_t h[4] = {0, 0, 0, 0};
    GJ_CUDA_TRY(ctx, cudaMemcpyAsync(h, acc, 4 * 8, cudaMemcpyDeviceToHost, st));
    GJ_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    GJ_TRY(gj_timer_collect(ctx));
    *count = (int64_t)h[0];
    *checksum = h[1];
    W.produced[k] = (int64_t)h[0];
    if (out_tuples && cap) {
        uint64_t wr = h[3] < cap ? h[3] : cap;
        if (wr) GJ_CUDA_TRY(ctx, cudaMemcpy(out_tuples, tuples, wr * k * 4, cudaMemcpyDeviceToHost));
        if (written) *written = wr;
    } else if (written) {
        *written = 0;
    }
    return GJ_OK;
}

int gj_engine_plain(gj_ctx* ctx, const gj_graph* g, const gj_query* q, uint32_t v_lo, uint32_t v_hi,
                    int64_t* count, uint64_t* checksum, uint32_t* out_tuples, uint64_t cap, uint64_t* written) {
    return gj_engine_plain_plan(ctx, g, q->plan, v_lo, v_hi, nullptr, count, checksum, out_tuples, cap, written);
}
