// The input-side specialisations of Section 5.4:
//
// - symmetry breaking's input transformation: the vertices get new ids that
//   ascend with degree (ties broken by the old id) and, optionally, only the
//   edges that point from a lower to a higher new id are kept, so that a
//   clique query finds each undirected clique once;
// - triangle indexing: the ternary relation tri(a, b, c) of the graph's
//   triangles (a -> b, a -> c, b -> c), indexed by its first two attributes.
//   For the forward slot e of the edge a -> b the list of c is the
//   intersection of out(a) and out(b), ascending; it is built by the same
//   propose-and-intersect step as the triangle query (the shorter list
//   proposes, the longer one is probed), in two passes: count, then write.
#include "gj_internal.cuh"

namespace {

unsigned grid_for(gj_ctx* ctx, uint64_t work) {
    uint64_t want = (work + 255) / 256;
    uint64_t cap = (uint64_t)ctx->sm_count * 16;
    if (want > cap) want = cap;
    return (unsigned)(want ? want : 1);
}

#define GRID_STRIDE(i, n) \
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += (uint64_t)gridDim.x * blockDim.x)

// keys[v] = degree(v) << 32 | v: ascending order ranks by (degree, id).
__global__ void k_degree_keys(const int64_t* __restrict__ off, uint32_t n, uint64_t* __restrict__ keys) {
    GRID_STRIDE(v, n) keys[v] = ((uint64_t)(off[v + 1] - off[v]) << 32) | v;
}

// new_of_old[old id] = rank.
__global__ void k_rank(const uint64_t* __restrict__ sorted, uint32_t n, uint32_t* __restrict__ new_of_old) {
    GRID_STRIDE(i, n) new_of_old[(uint32_t)sorted[i]] = (uint32_t)i;
}

// The edges of an index renamed by map (null: unchanged); with orient, an
// edge that does not point from a lower to a higher id becomes a self-loop,
// which the index builder drops.
__global__ void k_rename_edges(const uint32_t* __restrict__ key, const uint32_t* __restrict__ nbr, uint64_t m,
                               const uint32_t* __restrict__ map, int orient, uint32_t* __restrict__ os,
                               uint32_t* __restrict__ od) {
    GRID_STRIDE(e, m) {
        uint32_t u = key[e], v = nbr[e];
        if (map) {
            u = map[u];
            v = map[v];
        }
        if (orient && !(u < v)) v = u;
        os[e] = u;
        od[e] = v;
    }
}

constexpr int TW = 8;  // warps per block of the triangle-index kernel

// Triangle lists of the forward edges, 32 consecutive slots per warp grab.
// Each lane takes one edge (a, b); the shorter of out(a) and out(b)
// proposes, the longer is probed (its hash set, or binary search). The
// edges' candidates are laid out on one line by a warp scan and taken 32 at
// a time. PASS 0 writes the number of triangles of each edge to cnt; PASS 1
// writes them, in the proposer's ascending order, from toff[e].
template <int PASS>
__global__ void __launch_bounds__(TW * 32) k_tri_lists(GraphView G, uint64_t m, unsigned long long* __restrict__ next,
                                                      uint32_t* __restrict__ cnt, const int64_t* __restrict__ toff,
                                                      uint32_t* __restrict__ out) {
    __shared__ uint64_t s_cs[TW][33];
    __shared__ const uint32_t* s_prop[TW][32];
    __shared__ const uint32_t* s_tgt[TW][32];
    __shared__ uint32_t s_tlen[TW][32];
    __shared__ uint32_t s_tbits[TW][32];
    __shared__ uint32_t s_rc[TW][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t lt = gj_lanemask_lt();
    uint64_t* cs = s_cs[w];
    while (true) {
        unsigned long long e0 = 0;
        if (lane == 0) e0 = atomicAdd(next, 32ull);
        e0 = __shfl_sync(0xffffffffu, e0, 0);
        if (e0 >= m) break;
        const uint64_t e = e0 + lane;
        uint64_t len = 0;
        if (e < m) {
            const uint32_t a = __ldg(G.fk + e), b = __ldg(G.fn + e);
            const BindList La = gj_bind_list(G, GJ_BIND_FWD, a, 0), Lb = gj_bind_list(G, GJ_BIND_FWD, b, 0);
            const BindList& P = La.len <= Lb.len ? La : Lb;
            const BindList& T = La.len <= Lb.len ? Lb : La;
            len = P.len;
            s_prop[w][lane] = P.p;
            s_tgt[w][lane] = T.bits ? T.tab : T.p;
            s_tlen[w][lane] = T.len;
            s_tbits[w][lane] = T.bits;
        }
        s_rc[w][lane] = 0;
        uint64_t x = len;
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        cs[lane] = x - len;
        if (lane == 31) cs[32] = x;
        __syncwarp();
        const uint64_t total = cs[32];
        for (uint64_t base = 0; base < total; base += 32) {
            const uint64_t t = base + lane;
            const bool valid = t < total;
            uint32_t i = 32;  // the lane's edge within the grab (32: none)
            uint32_t c = 0;
            bool keep = false;
            if (valid) {
                uint32_t lo = 0, hi = 32;  // last i with cs[i] <= t
                while (hi - lo > 1) {
                    const uint32_t mid = (lo + hi) >> 1;
                    if (cs[mid] <= t) lo = mid; else hi = mid;
                }
                i = lo;
                c = __ldg(s_prop[w][i] + (t - cs[i]));
                keep = s_tbits[w][i] ? gj_tab_member(s_tgt[w][i], s_tbits[w][i], c)
                                     : gj_contains(s_tgt[w][i], s_tlen[w][i], c);
            }
            const uint32_t peers = __match_any_sync(0xffffffffu, i);
            const uint32_t km = __ballot_sync(0xffffffffu, keep);
            if (PASS == 1 && keep) out[toff[e0 + i] + s_rc[w][i] + __popc(peers & km & lt)] = c;
            __syncwarp();
            if (valid && (peers & lt) == 0) s_rc[w][i] += __popc(peers & km);  // the lowest lane of each edge
            __syncwarp();
        }
        if (PASS == 0 && e < m) cnt[e] = s_rc[w][lane];
        __syncwarp();
    }
}

// Slot count of each triangle list's hash set (0 for lists shorter than GJ_HASH_MIN_DEG).
__global__ void k_tri_tab_sizes(const int64_t* __restrict__ toff, uint64_t m, int64_t* __restrict__ size) {
    GRID_STRIDE(e, m) {
        const uint32_t len = (uint32_t)(toff[e + 1] - toff[e]);
        size[e] = len >= GJ_HASH_MIN_DEG ? (int64_t)(1ll << gj_tab_bits(len)) : 0;
    }
}

// Fills the hash sets of the long triangle lists, one warp per list (the
// same layout and probing as the index's sets: linear probing from the first
// slot of the key's home group of eight). A set of up to TAB_SMEM slots is
// built in the warp's shared memory and written out whole with 16-byte
// stores; larger sets are filled in place with global atomics.
constexpr int TTW = 4;               // warps per block of the insert kernel
constexpr uint32_t TAB_SMEM = 2048;  // slots of a warp's shared-memory set
__global__ void __launch_bounds__(TTW * 32) k_tri_tab_insert(const int64_t* __restrict__ toff,
                                                             const uint32_t* __restrict__ tn, uint64_t m,
                                                             const int64_t* __restrict__ tab_off,
                                                             uint32_t* __restrict__ tab) {
    __shared__ __align__(16) uint32_t s_tab[TTW][TAB_SMEM];
    const uint64_t warps = (uint64_t)gridDim.x * TTW;
    const int lane = threadIdx.x & 31;
    uint32_t* st = s_tab[threadIdx.x >> 5];
    for (uint64_t e = (uint64_t)blockIdx.x * TTW + (threadIdx.x >> 5); e < m; e += warps) {
        const int64_t a = toff[e];
        const uint32_t len = (uint32_t)(toff[e + 1] - a);
        if (len < GJ_HASH_MIN_DEG) continue;
        const uint32_t bits = gj_tab_bits(len), mask = (1u << bits) - 1u, size = 1u << bits;
        uint32_t* t = tab + tab_off[e];  // 128-byte aligned, size a multiple of 32 slots
        uint32_t* dst = size <= TAB_SMEM ? st : t;
        if (size <= TAB_SMEM) {
            for (uint32_t i = lane; i < size; i += 32) st[i] = GJ_EMPTY;
            __syncwarp();
        }
        for (uint32_t i = lane; i < len; i += 32) {
            const uint32_t x = tn[a + i];
            uint32_t h = gj_tab_start(x, bits);
            for (uint32_t probe = 0; probe <= mask; probe++) {
                if (atomicCAS(dst + h, GJ_EMPTY, x) == GJ_EMPTY) break;
                h = (h + 1u) & mask;
            }
        }
        if (size <= TAB_SMEM) {
            __syncwarp();
            for (uint32_t i = 4 * lane; i < size; i += 128)
                *reinterpret_cast<uint4*>(t + i) = *reinterpret_cast<const uint4*>(st + i);
            __syncwarp();
        }
    }
}

// Inserts every forward edge (key[e], nbr[e]) with its slot e into the edge
// map (linear probing; the map has at least twice as many entries as edges).
__global__ void k_edge_map(const uint32_t* __restrict__ key, const uint32_t* __restrict__ nbr, uint64_t m,
                           uint4* __restrict__ em, uint32_t bits) {
    const uint32_t mask = (uint32_t)((1ull << bits) - 1u);
    GRID_STRIDE(e, m) {
        const uint32_t a = key[e], b = nbr[e];
        const unsigned long long want = ((unsigned long long)b << 32) | a;  // {x = a, y = b} in memory order
        uint32_t h = gj_edge_home(a, b, bits);
        for (uint64_t probe = 0; probe <= mask; probe++) {
            unsigned long long* w = reinterpret_cast<unsigned long long*>(em + h);
            if (atomicCAS(w, ~0ull, want) == ~0ull) {
                em[h].z = (uint32_t)e;
                break;
            }
            h = (h + 1u) & mask;
        }
    }
}

}  // namespace

void gj_tri_release(gj_tri& t) {
    for (void* p : {(void*)t.off, (void*)t.nbr, (void*)t.tab_off, (void*)t.tab, (void*)t.emap})
        if (p) cudaFree(p);
    t = gj_tri{};
}

// The edge map of the forward index (2^ceil(log2(2 m)) entries, at least 2).
static int edge_map(gj_ctx* ctx, const gj_graph* g, gj_tri& t) {
    uint32_t bits = 1;
    while ((1ull << bits) < 2 * g->m) bits++;
    GJ_CUDA_TRY(ctx, gj_malloc(ctx, &t.emap, sizeof(uint4) << bits));
    GJ_CUDA_TRY(ctx, cudaMemsetAsync(t.emap, 0xff, sizeof(uint4) << bits, ctx->stream));
    if (g->m) {
        k_edge_map<<<grid_for(ctx, g->m), 256, 0, ctx->stream>>>(g->fwd.key, g->fwd.nbr, g->m, t.emap, bits);
        GJ_LAUNCHED(ctx);
    }
    GJ_CUDA_TRY(ctx, cudaGetLastError());
    t.ebits = bits;
    return GJ_OK;
}

// Hash sets of t's long lists (after its lists are written).
static int tri_tables(gj_ctx* ctx, uint64_t m, gj_tri& t) {
    cudaStream_t st = ctx->stream;
    GJ_CUDA_TRY(ctx, gj_malloc(ctx, &t.tab_off, sizeof(int64_t) * (m + 1)));
    int64_t* size = nullptr;
    GJ_CUDA_TRY(ctx, gj_malloc_async(ctx, &size, sizeof(int64_t) * (m ? m : 1), st));
    if (m) {
        k_tri_tab_sizes<<<grid_for(ctx, m), 256, 0, st>>>(t.off, m, size);
        GJ_LAUNCHED(ctx);
    }
    int rc = gj_scan_i64(ctx, size, t.tab_off, m);
    int64_t tsz = 0;
    if (rc == GJ_OK && (cudaMemcpyAsync(&tsz, t.tab_off + m, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                        cudaStreamSynchronize(st) != cudaSuccess))
        rc = GJ_E_CUDA;
    cudaFreeAsync(size, st);
    GJ_TRY(rc);
    GJ_CUDA_TRY(ctx, gj_malloc(ctx, &t.tab, sizeof(uint32_t) * (size_t)(tsz ? tsz : 1)));
    if (tsz > 0) {
        GJ_CUDA_TRY(ctx, cudaMemsetAsync(t.tab, 0xff, sizeof(uint32_t) * (size_t)tsz, st));
        k_tri_tab_insert<<<(unsigned)ctx->sm_count * 16, TTW * 32, 0, st>>>(t.off, t.nbr, m, t.tab_off, t.tab);
        GJ_LAUNCHED(ctx);
    }
    GJ_CUDA_TRY(ctx, cudaGetLastError());
    return GJ_OK;
}

int gj_tri_build(gj_ctx* ctx, gj_graph* g) {
    if (g->tri.off) return GJ_OK;
    cudaStream_t st = ctx->stream;
    const uint64_t m = g->m;
    gj_tri t;
    GJ_CUDA_TRY(ctx, gj_malloc(ctx, &t.off, sizeof(int64_t) * (m + 1)));
    uint32_t* cnt = nullptr;
    unsigned long long* next = nullptr;
    cudaError_t e = gj_malloc_async(ctx, &cnt, sizeof(uint32_t) * (m ? m : 1) + 256, st);
    if (e != cudaSuccess) {
        gj_tri_release(t);
        gj_set_error(ctx, GJ_E_NOMEM, std::string("triangle index: ") + cudaGetErrorString(e));
        return GJ_E_NOMEM;
    }
    next = (unsigned long long*)((char*)cnt + (((sizeof(uint32_t) * (m ? m : 1)) + 127) & ~(size_t)127));
    const GraphView G = g->view();
    const unsigned grid = (unsigned)ctx->sm_count * 8;
    int rc = GJ_OK;
    int64_t total = 0;
    auto run = [&](int pass) -> int {
        GJ_CUDA_TRY(ctx, cudaMemsetAsync(next, 0, 8, st));
        if (m) {
            if (pass == 0) k_tri_lists<0><<<grid, TW * 32, 0, st>>>(G, m, next, cnt, t.off, t.nbr);
            else k_tri_lists<1><<<grid, TW * 32, 0, st>>>(G, m, next, cnt, t.off, t.nbr);
            GJ_LAUNCHED(ctx);
        }
        GJ_CUDA_TRY(ctx, cudaGetLastError());
        return GJ_OK;
    };
    rc = run(0);
    if (rc == GJ_OK) rc = gj_scan_u32(ctx, cnt, t.off, m);
    if (rc == GJ_OK && cudaMemcpyAsync(&total, t.off + m, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess) rc = GJ_E_CUDA;
    if (rc == GJ_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = GJ_E_CUDA;
    if (rc == GJ_OK && gj_malloc(ctx, &t.nbr, sizeof(uint32_t) * (size_t)(total ? total : 1)) != cudaSuccess) {
        cudaGetLastError();
        gj_set_error(ctx, GJ_E_NOMEM, "triangle index: out of device memory");
        rc = GJ_E_NOMEM;
    }
    if (rc == GJ_OK) rc = run(1);
    cudaFreeAsync(cnt, st);
    if (rc == GJ_OK) rc = tri_tables(ctx, m, t);
    if (rc == GJ_OK) rc = edge_map(ctx, g, t);
    if (rc == GJ_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = GJ_E_CUDA;
    if (rc != GJ_OK) {
        gj_tri_release(t);
        return rc;
    }
    t.count = (uint64_t)total;
    g->tri = t;
    return GJ_OK;
}

int gj_graph_transform(gj_ctx* ctx, gj_graph* g, uint32_t flags) {
    const bool rename = flags & GJ_LOAD_DEGREE_ORDER, orient = flags & GJ_LOAD_ORIENT;
    if (!rename && !orient) return GJ_OK;
    cudaStream_t st = ctx->stream;
    const uint32_t n = g->n;
    const uint64_t m = g->m;
    uint32_t* map = nullptr;
    if (rename) {
        GJ_CUDA_TRY(ctx, gj_malloc(ctx, &map, sizeof(uint32_t) * n));
        uint64_t *keys = nullptr, *res = nullptr;
        cudaError_t e = gj_malloc_async(ctx, &keys, 16 * (size_t)n, st);
        if (e != cudaSuccess) {
            cudaFree(map);
            gj_set_error(ctx, GJ_E_NOMEM, "degree renaming: out of device memory");
            return GJ_E_NOMEM;
        }
        k_degree_keys<<<grid_for(ctx, n), 256, 0, st>>>(g->fwd.off, n, keys);
        GJ_LAUNCHED(ctx);
        int rc = gj_radix_sort_u64(ctx, keys, keys + n, n, 64, &res);
        if (rc == GJ_OK) {
            k_rank<<<grid_for(ctx, n), 256, 0, st>>>(res, n, map);
            GJ_LAUNCHED(ctx);
        }
        cudaFreeAsync(keys, st);
        if (rc != GJ_OK) {
            cudaFree(map);
            return rc;
        }
    }
    uint32_t* pairs = nullptr;
    cudaError_t e = gj_malloc_async(ctx, &pairs, 8 * (size_t)(m ? m : 1), st);
    if (e != cudaSuccess) {
        if (map) cudaFree(map);
        gj_set_error(ctx, GJ_E_NOMEM, "degree renaming: out of device memory");
        return GJ_E_NOMEM;
    }
    if (m) {
        k_rename_edges<<<grid_for(ctx, m), 256, 0, st>>>(g->fwd.key, g->fwd.nbr, m, map, orient ? 1 : 0, pairs,
                                                          pairs + m);
        GJ_LAUNCHED(ctx);
    }
    // rebuild the indices from the renamed edges (once the renaming has read the old ones)
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaFreeAsync(pairs, st);
        if (map) cudaFree(map);
        gj_set_error(ctx, GJ_E_CUDA, std::string("degree renaming: ") + cudaGetErrorString(e));
        return GJ_E_CUDA;
    }
    for (gj_csr* c : {&g->fwd, &g->rev, &g->spare_fwd, &g->spare_rev}) gj_csr_release(*c);
    gj_tri_release(g->tri);
    int rc = gj_csr_build(ctx, pairs, pairs + m, m, n, g);
    cudaFreeAsync(pairs, st);
    if (rc != GJ_OK) {
        if (map) cudaFree(map);
        return rc;
    }
    GJ_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    g->relabel = map;
    return GJ_OK;
}
