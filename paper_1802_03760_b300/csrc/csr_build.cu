// Index builder: turns an edge list into the forward index (out-neighbours
// of each vertex, sorted) and the reverse index (in-neighbours, sorted), the
// two indices every atom of every query shares (Section 4.1). An index gives
// an extension set's size in O(1) (offset difference), its contents in
// linear time (a contiguous sorted run) and membership by binary search,
// or by a hash set for lists of at least GJ_HASH_MIN_DEG entries (the
// three properties of Section 2.2).
//
// Steps per index: pack (key vertex, neighbour) into one 64-bit key with
// self-loops mapped to an all-ones sentinel, radix sort, keep the first of
// each run of equal keys, scatter neighbours and key vertices, set
// off[v] = first slot whose key vertex is >= v, then size and fill the
// hash sets of the long lists.
#include "gj_internal.cuh"

namespace {

constexpr uint64_t SENTINEL = ~0ull;

__global__ void k_pack(const uint32_t* __restrict__ hi, const uint32_t* __restrict__ lo, uint64_t m, uint32_t n,
                       int vb, uint64_t* __restrict__ keys, uint32_t* __restrict__ err) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
        uint32_t a = hi[i], b = lo[i];
        uint64_t k;
        if (a >= n || b >= n) {
            atomicOr(err, 1u);
            k = SENTINEL;
        } else if (a == b) {
            k = SENTINEL;  // self-loops are not edges of the relation
        } else {
            k = ((uint64_t)a << vb) | b;
        }
        keys[i] = k;
    }
}

__global__ void k_first_of_run(const uint64_t* __restrict__ keys, uint64_t m, uint32_t* __restrict__ flag) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
        uint64_t k = keys[i];
        flag[i] = (k != SENTINEL && (i == 0 || keys[i - 1] != k)) ? 1u : 0u;
    }
}

__global__ void k_scatter_unique(const uint64_t* __restrict__ keys, uint64_t m, const uint32_t* __restrict__ flag,
                                 const int64_t* __restrict__ pos, int vb, uint32_t* __restrict__ nbr,
                                 uint32_t* __restrict__ keyv) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t mask = (vb >= 64) ? ~0ull : ((1ull << vb) - 1);
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
        if (flag[i]) {
            uint64_t k = keys[i];
            int64_t p = pos[i];
            nbr[p] = (uint32_t)(k & mask);
            keyv[p] = (uint32_t)(k >> vb);
        }
    }
}

// off[v] = number of slots whose key vertex is < v, for v in [0, n].
__global__ void k_offsets(const uint32_t* __restrict__ keyv, uint64_t mu, uint32_t n, int64_t* __restrict__ off) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v <= n; v += stride) {
        uint64_t lo = 0, hi = mu;
        while (lo < hi) {
            uint64_t mid = (lo + hi) >> 1;
            if ((uint64_t)keyv[mid] < v) lo = mid + 1; else hi = mid;
        }
        off[v] = (int64_t)lo;
    }
}

// Slot count of each vertex's hash set (0 for lists shorter than GJ_HASH_MIN_DEG).
__global__ void k_tab_sizes(const int64_t* __restrict__ off, uint32_t n, int64_t* __restrict__ size) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const uint32_t len = (uint32_t)(off[v + 1] - off[v]);
        size[v] = len >= GJ_HASH_MIN_DEG ? (int64_t)(1ll << gj_tab_bits(len)) : 0;
    }
}

// Inserts every neighbour of a long list into its vertex's hash set by
// linear probing with atomicCAS. A set has at least twice as many slots as
// distinct keys, so every insertion finds an empty slot.
__global__ void k_tab_insert(const int64_t* __restrict__ off, const uint32_t* __restrict__ nbr,
                             const uint32_t* __restrict__ key, uint64_t m, const int64_t* __restrict__ tab_off,
                             uint32_t* __restrict__ tab) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
        const uint32_t v = key[e];
        const uint32_t len = (uint32_t)(off[v + 1] - off[v]);
        if (len < GJ_HASH_MIN_DEG) continue;
        const uint32_t bits = gj_tab_bits(len);
        const uint32_t mask = (1u << bits) - 1u;
        uint32_t* t = tab + tab_off[v];
        const uint32_t x = nbr[e];
        uint32_t h = gj_tab_start(x, bits);  // first slot of the home group
        for (uint32_t probe = 0; probe <= mask; probe++) {
            if (atomicCAS(t + h, GJ_EMPTY, x) == GJ_EMPTY) break;
            h = (h + 1u) & mask;
        }
    }
}

int vertex_bits(uint32_t n) {
    int b = 1;
    while (b < 32 && (1ull << b) < (uint64_t)n) b++;
    return b;
}

unsigned grid_for(gj_ctx* ctx, uint64_t work) {
    uint64_t want = (work + 255) / 256;
    uint64_t cap = (uint64_t)ctx->sm_count * 16;
    if (want > cap) want = cap;
    return (unsigned)(want ? want : 1);
}

// One index: keys from (hi, lo) pairs. tmp buffers are caller-provided.
int build_index(gj_ctx* ctx, const uint32_t* hi, const uint32_t* lo, uint64_t m, uint32_t n, gj_csr* out,
                uint64_t* mu_out, uint64_t* keys, uint64_t* keys2, uint32_t* flag, int64_t* pos, uint32_t* err) {
    cudaStream_t st = ctx->stream;
    int vb = vertex_bits(n);
    if (m > 0) { k_pack<<<grid_for(ctx, m), 256, 0, st>>>(hi, lo, m, n, vb, keys, err); GJ_LAUNCHED(ctx); }
    uint64_t* sorted = keys;
    GJ_TRY(gj_radix_sort_u64(ctx, keys, keys2, m, 2 * vb, &sorted));
    if (m > 0) { k_first_of_run<<<grid_for(ctx, m), 256, 0, st>>>(sorted, m, flag); GJ_LAUNCHED(ctx); }
    GJ_TRY(gj_scan_u32(ctx, flag, pos, m));
    int64_t mu = 0;
    GJ_CUDA_TRY(ctx, cudaMemcpyAsync(&mu, pos + m, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    GJ_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    GJ_CUDA_TRY(ctx, gj_malloc(ctx, &out->off, sizeof(int64_t) * ((size_t)n + 1)));
    GJ_CUDA_TRY(ctx, gj_malloc(ctx, &out->nbr, sizeof(uint32_t) * (size_t)(mu ? mu : 1)));
    GJ_CUDA_TRY(ctx, gj_malloc(ctx, &out->key, sizeof(uint32_t) * (size_t)(mu ? mu : 1)));
    out->cap_m = (uint64_t)(mu ? mu : 1);
    if (m > 0) {
        k_scatter_unique<<<grid_for(ctx, m), 256, 0, st>>>(sorted, m, flag, pos, vb, out->nbr, out->key);
        GJ_LAUNCHED(ctx);
    }
    GJ_TRY(gj_csr_finish(ctx, n, (uint64_t)mu, out));
    *mu_out = (uint64_t)mu;
    return GJ_OK;
}

}  // namespace

int gj_csr_finish(gj_ctx* ctx, uint32_t n, uint64_t mu, gj_csr* out) {
    cudaStream_t st = ctx->stream;
    if (!out->off) GJ_CUDA_TRY(ctx, gj_malloc(ctx, &out->off, sizeof(int64_t) * ((size_t)n + 1)));
    k_offsets<<<grid_for(ctx, (uint64_t)n + 1), 256, 0, st>>>(out->key, mu, n, out->off);
    GJ_LAUNCHED(ctx);
    GJ_CUDA_TRY(ctx, cudaGetLastError());
    // hash sets of the long lists
    int64_t* size = nullptr;
    GJ_CUDA_TRY(ctx, gj_malloc_async(ctx, &size, sizeof(int64_t) * ((size_t)n + 1), st));
    GJ_CUDA_TRY(ctx, gj_malloc(ctx, &out->tab_off, sizeof(int64_t) * ((size_t)n + 1)));
    k_tab_sizes<<<grid_for(ctx, n), 256, 0, st>>>(out->off, n, size);
    GJ_LAUNCHED(ctx);
    int rc = gj_scan_i64(ctx, size, out->tab_off, n);
    int64_t tsz = 0;
    if (rc == GJ_OK) {
        cudaMemcpyAsync(&tsz, out->tab_off + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
        cudaStreamSynchronize(st);
    }
    cudaFreeAsync(size, st);
    GJ_TRY(rc);
    GJ_CUDA_TRY(ctx, gj_malloc(ctx, &out->tab, sizeof(uint32_t) * (size_t)(tsz ? tsz : 1)));
    out->cap_tab = (uint64_t)(tsz ? tsz : 1);
    if (tsz > 0) {
        GJ_CUDA_TRY(ctx, cudaMemsetAsync(out->tab, 0xff, sizeof(uint32_t) * (size_t)tsz, st));
        k_tab_insert<<<grid_for(ctx, mu), 256, 0, st>>>(out->off, out->nbr, out->key, mu, out->tab_off, out->tab);
        GJ_LAUNCHED(ctx);
    }
    GJ_CUDA_TRY(ctx, cudaGetLastError());
    return GJ_OK;
}

int gj_csr_build(gj_ctx* ctx, const uint32_t* d_src, const uint32_t* d_dst, uint64_t m, uint32_t n, gj_graph* g) {
    cudaStream_t st = ctx->stream;
    uint64_t *keys = nullptr, *keys2 = nullptr;
    uint32_t* flag = nullptr;
    int64_t* pos = nullptr;
    uint32_t* err = nullptr;
    size_t mm = (size_t)(m ? m : 1);
    int rc = GJ_OK;
    auto fail = [&](cudaError_t e) {
        gj_set_error(ctx, GJ_E_CUDA, std::string("index build: ") + cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? GJ_E_NOMEM : GJ_E_CUDA;
    };
    cudaError_t e;
    if ((e = gj_malloc_async(ctx, &keys, mm * 8, st)) != cudaSuccess) return fail(e);
    if ((e = gj_malloc_async(ctx, &keys2, mm * 8, st)) != cudaSuccess) { cudaFreeAsync(keys, st); return fail(e); }
    if ((e = gj_malloc_async(ctx, &flag, mm * 4, st)) != cudaSuccess) { cudaFreeAsync(keys, st); cudaFreeAsync(keys2, st); return fail(e); }
    if ((e = gj_malloc_async(ctx, &pos, (mm + 1) * 8 + 64, st)) != cudaSuccess) {
        cudaFreeAsync(keys, st); cudaFreeAsync(keys2, st); cudaFreeAsync(flag, st); return fail(e);
    }
    err = (uint32_t*)(pos + mm + 1);
    cudaMemsetAsync(err, 0, sizeof(uint32_t), st);
    uint64_t mf = 0, mr = 0;
    rc = build_index(ctx, d_src, d_dst, m, n, &g->fwd, &mf, keys, keys2, flag, pos, err);
    if (rc == GJ_OK) rc = build_index(ctx, d_dst, d_src, m, n, &g->rev, &mr, keys, keys2, flag, pos, err);
    uint32_t herr = 0;
    if (rc == GJ_OK) {
        cudaMemcpyAsync(&herr, err, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) rc = fail(e);
    }
    cudaFreeAsync(keys, st);
    cudaFreeAsync(keys2, st);
    cudaFreeAsync(flag, st);
    cudaFreeAsync(pos, st);
    if (rc != GJ_OK) return rc;
    if (herr) {
        gj_set_error(ctx, GJ_E_RANGE, "vertex id >= num_vertices");
        return GJ_E_RANGE;
    }
    g->n = n;
    g->m = mf;
    (void)mr;  // the reverse index holds the same pairs transposed
    return GJ_OK;
}
