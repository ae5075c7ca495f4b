// Update batches (Section 3.3.1, Section 4.3): normalisation of a batch of
// signed edge updates against the committed graph, the per-direction
// insert/delete arrays that the new version of each index reads, and the
// commit that folds a batch into the indices.
//
// Normalisation follows R' = R + Delta R with updates applied in batch
// order: a stable sort groups the updates of each edge in batch order, the
// last one decides whether the edge is present afterwards, self-loops are
// dropped, and only edges whose presence changes remain, with sign +1
// (inserted) or -1 (deleted).
#include "gj_internal.cuh"

namespace {

constexpr uint64_t SENT = ~0ull;

unsigned grid_for(gj_ctx* ctx, uint64_t work) {
    uint64_t want = (work + 255) / 256;
    uint64_t cap = (uint64_t)ctx->sm_count * 16;
    if (want > cap) want = cap;
    return (unsigned)(want ? want : 1);
}

int vertex_bits(uint32_t n) {
    int b = 1;
    while (b < 32 && (1ull << b) < (uint64_t)n) b++;
    return b;
}

#define GRID_STRIDE(i, n) \
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += (uint64_t)gridDim.x * blockDim.x)

// err bit 1: vertex id out of range; bit 2: sign not +-1.
__global__ void k_dpack(const uint32_t* __restrict__ src, const uint32_t* __restrict__ dst,
                        const int8_t* __restrict__ sign, uint64_t b, uint32_t n, int vb, uint64_t* __restrict__ keys,
                        uint32_t* __restrict__ idx, uint32_t* __restrict__ err) {
    GRID_STRIDE(i, b) {
        const uint32_t u = src[i], v = dst[i];
        const int8_t s = sign[i];
        bool bad = false;
        if (u >= n || v >= n) {
            atomicOr(err, 1u);
            bad = true;
        }
        if (s != 1 && s != -1) {
            atomicOr(err, 2u);
            bad = true;
        }
        keys[i] = (bad || u == v) ? SENT : (((uint64_t)u << vb) | v);
        idx[i] = (uint32_t)i;
    }
}

// flag[p] = 1 if sorted update p is the last update of its edge and flips
// the edge's presence in the committed graph; lsign[p] = its sign.
__global__ void k_dlast(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ idx, uint64_t b,
                        const int8_t* __restrict__ sign, int vb, GraphView G, uint32_t* __restrict__ flag,
                        int8_t* __restrict__ lsign) {
    const uint64_t mask = (1ull << vb) - 1;
    GRID_STRIDE(p, b) {
        const uint64_t k = keys[p];
        uint32_t f = 0;
        int8_t s = 0;
        if (k != SENT && (p + 1 == b || keys[p + 1] != k)) {
            s = sign[idx[p]];
            const uint32_t u = (uint32_t)(k >> vb), v = (uint32_t)(k & mask);
            const bool present = gj_list_member(G.fo, G.fn, G.fto, G.ft, u, v);
            f = ((s > 0) != present) ? 1u : 0u;
        }
        flag[p] = f;
        lsign[p] = s;
    }
}

__global__ void k_dcompact(const uint64_t* __restrict__ keys, uint64_t b, const uint32_t* __restrict__ flag,
                           const int64_t* __restrict__ pos, const int8_t* __restrict__ lsign, int vb,
                           uint32_t* __restrict__ osrc, uint32_t* __restrict__ odst, int8_t* __restrict__ osign) {
    const uint64_t mask = (1ull << vb) - 1;
    GRID_STRIDE(p, b) {
        if (!flag[p]) continue;
        const int64_t o = pos[p];
        osrc[o] = (uint32_t)(keys[p] >> vb);
        odst[o] = (uint32_t)(keys[p] & mask);
        osign[o] = lsign[p];
    }
}

// flag[i] = 1 if element i has the wanted sign (signs read through idx when given).
__global__ void k_sign_flag(const int8_t* __restrict__ sign, const uint32_t* __restrict__ idx, uint64_t n, int want,
                            uint32_t* __restrict__ flag) {
    GRID_STRIDE(i, n) {
        const int8_t s = sign[idx ? idx[i] : i];
        flag[i] = (s == want) ? 1u : 0u;
    }
}

// Scatters flagged (owner, neighbour) pairs of keys (owner << vb | nbr) or of
// (own[], nbr[]) arrays into compact arrays.
__global__ void k_pair_compact(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ own,
                               const uint32_t* __restrict__ nbr, uint64_t n, int vb, const uint32_t* __restrict__ flag,
                               const int64_t* __restrict__ pos, uint32_t* __restrict__ okey,
                               uint32_t* __restrict__ onbr) {
    const uint64_t mask = (1ull << vb) - 1;
    GRID_STRIDE(i, n) {
        if (!flag[i]) continue;
        const int64_t o = pos[i];
        if (keys) {
            okey[o] = (uint32_t)(keys[i] >> vb);
            onbr[o] = (uint32_t)(keys[i] & mask);
        } else {
            okey[o] = own[i];
            onbr[o] = nbr[i];
        }
    }
}

__global__ void k_rev_keys(const uint32_t* __restrict__ src, const uint32_t* __restrict__ dst, uint64_t n, int vb,
                           uint64_t* __restrict__ keys, uint32_t* __restrict__ idx) {
    GRID_STRIDE(i, n) {
        keys[i] = ((uint64_t)dst[i] << vb) | src[i];
        idx[i] = (uint32_t)i;
    }
}

// Records, for every run of equal keys in a key-sorted array, the run's
// [lo, hi) in the vertex's hash-map entry (field 0: inserts, 1: deletes).
__global__ void k_range_map(const uint32_t* __restrict__ key, uint32_t n, int which, uint32_t* __restrict__ hkey,
                            uint4* __restrict__ hval, uint32_t bits) {
    const uint32_t mask = (1u << bits) - 1u;
    GRID_STRIDE(p, n) {
        const uint32_t v = key[p];
        if (p > 0 && key[p - 1] == v) continue;
        uint32_t hi = (uint32_t)p + 1;
        while (hi < n && key[hi] == v) hi++;
        uint32_t h = gj_tab_home(v, bits);
        for (uint32_t probe = 0; probe <= mask; probe++) {
            const uint32_t old = atomicCAS(hkey + h, GJ_EMPTY, v);
            if (old == GJ_EMPTY || old == v) break;
            h = (h + 1u) & mask;
        }
        if (which == 0) {
            hval[h].x = (uint32_t)p;
            hval[h].y = hi;
        } else {
            hval[h].z = (uint32_t)p;
            hval[h].w = hi;
        }
    }
}

// Number of entries below x in the sorted list a[0, len).
__device__ __forceinline__ uint64_t lower_count(const uint32_t* __restrict__ a, uint64_t len, uint32_t x) {
    uint64_t lo = 0, hi = len;
    while (lo < hi) {
        const uint64_t mid = (lo + hi) >> 1;
        if (a[mid] < x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// The list owners of the batch's inserts and deletes of one index
// direction, as 64-bit keys (to be sorted and deduplicated).
__global__ void k_touch_keys(const uint32_t* __restrict__ ik, uint32_t ni, const uint32_t* __restrict__ dk, uint32_t nd,
                             uint64_t* __restrict__ keys) {
    GRID_STRIDE(i, (uint64_t)ni + nd) keys[i] = i < ni ? ik[i] : dk[i - ni];
}

__global__ void k_run_flag(const uint64_t* __restrict__ keys, uint64_t n, uint32_t* __restrict__ flag) {
    GRID_STRIDE(i, n) flag[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1u : 0u;
}

__global__ void k_run_compact(const uint64_t* __restrict__ keys, uint64_t n, const uint32_t* __restrict__ flag,
                              const int64_t* __restrict__ pos, uint32_t* __restrict__ out) {
    GRID_STRIDE(i, n) if (flag[i]) out[pos[i]] = (uint32_t)keys[i];
}

// Per touched vertex (ascending): the change of its list length and of its
// hash set's slot count, its committed list length, its next list length and
// its next hash set's slot count.
__global__ void k_touch_info(const uint32_t* __restrict__ tv, uint32_t ntv, DeltaSide side,
                             const int64_t* __restrict__ off, int64_t* __restrict__ dlen,
                             int64_t* __restrict__ dtab, int64_t* __restrict__ olen, int64_t* __restrict__ nlen,
                             int64_t* __restrict__ ntab) {
    GRID_STRIDE(i, ntv) {
        const uint32_t v = tv[i];
        const uint4 r = gj_delta_ranges(side, v);
        const int64_t d = (int64_t)(r.y - r.x) - (int64_t)(r.w - r.z);
        const uint32_t ol = (uint32_t)(off[v + 1] - off[v]), nl = (uint32_t)((int64_t)ol + d);
        const int64_t ot = ol >= GJ_HASH_MIN_DEG ? (1ll << gj_tab_bits(ol)) : 0;
        const int64_t nt = nl >= GJ_HASH_MIN_DEG ? (1ll << gj_tab_bits(nl)) : 0;
        dlen[i] = d;
        dtab[i] = nt - ot;
        olen[i] = ol;
        nlen[i] = nl;
        ntab[i] = nt;
    }
}

// The touched vertex that owns flat item f, given the exclusive sums P of
// the items per touched vertex: the last i with P[i] <= f.
__device__ __forceinline__ uint32_t owner_of(const int64_t* __restrict__ P, uint32_t ntv, int64_t f) {
    uint32_t lo = 0, hi = ntv;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (P[mid] <= f) lo = mid; else hi = mid;
    }
    return lo;
}

// The next version's offsets: every list and hash set moves by the sum of
// the changes of the touched vertices before it (S, ST: exclusive sums).
__global__ void k_shift_offsets(const int64_t* __restrict__ off, const int64_t* __restrict__ toff, uint32_t n,
                                const uint32_t* __restrict__ tv, uint32_t ntv, const int64_t* __restrict__ S,
                                const int64_t* __restrict__ ST, int64_t* __restrict__ noff,
                                int64_t* __restrict__ ntoff) {
    GRID_STRIDE(v, (uint64_t)n + 1) {
        uint32_t lo = 0, hi = ntv;  // touched vertices below v
        while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if (tv[mid] < v) lo = mid + 1; else hi = mid;
        }
        noff[v] = off[v] + S[lo];
        ntoff[v] = toff[v] + ST[lo];
    }
}

// Block r moves the lists and hash sets of the untouched vertices between
// touched vertices r - 1 and r to their new place (a constant shift).
__global__ void k_shift_copy(const int64_t* __restrict__ off, const int64_t* __restrict__ toff,
                             const uint32_t* __restrict__ nbr, const uint32_t* __restrict__ key,
                             const uint32_t* __restrict__ tab, uint32_t n, const uint32_t* __restrict__ tv, uint32_t ntv,
                             const int64_t* __restrict__ S, const int64_t* __restrict__ ST, uint32_t* __restrict__ nnbr,
                             uint32_t* __restrict__ nkey, uint32_t* __restrict__ ntab) {
    for (uint64_t r = blockIdx.x; r <= ntv; r += gridDim.x) {
        const uint32_t lo_v = r == 0 ? 0u : tv[r - 1] + 1, hi_v = r == ntv ? n : tv[r];
        if (lo_v >= hi_v) continue;
        // eight independent loads per thread before its stores (bytes in flight)
        constexpr int U = 8;
        const int64_t a = off[lo_v], b = off[hi_v], sh = S[r];
        for (int64_t e0 = a + threadIdx.x; e0 < b; e0 += (int64_t)U * blockDim.x) {
            uint32_t x[U], y[U];
#pragma unroll
            for (int u = 0; u < U; u++) {
                const int64_t e = e0 + (int64_t)u * blockDim.x;
                if (e < b) {
                    x[u] = nbr[e];
                    y[u] = key[e];
                }
            }
#pragma unroll
            for (int u = 0; u < U; u++) {
                const int64_t e = e0 + (int64_t)u * blockDim.x;
                if (e < b) {
                    nnbr[e + sh] = x[u];
                    nkey[e + sh] = y[u];
                }
            }
        }
        const int64_t ta = toff[lo_v], tb = toff[hi_v], tsh = ST[r];
        for (int64_t e0 = ta + threadIdx.x; e0 < tb; e0 += (int64_t)U * blockDim.x) {
            uint32_t x[U];
#pragma unroll
            for (int u = 0; u < U; u++) {
                const int64_t e = e0 + (int64_t)u * blockDim.x;
                if (e < tb) x[u] = tab[e];
            }
#pragma unroll
            for (int u = 0; u < U; u++) {
                const int64_t e = e0 + (int64_t)u * blockDim.x;
                if (e < tb) ntab[e + tsh] = x[u];
            }
        }
    }
}

// The next lists of the touched vertices: the committed entries that the
// batch does not delete, and the batch's inserts, each written straight to
// its place (all lists sorted; deletes are in the committed list, inserts are
// not). Flat item f < OLP[ntv] is committed entry f - OLP[i] of touched vertex
// i; item OLP[ntv] + e is insert e of the direction.
__global__ void k_merge_touched(const int64_t* __restrict__ off, const uint32_t* __restrict__ nbr,
                                const uint32_t* __restrict__ tv, uint32_t ntv, DeltaSide side,
                                const int64_t* __restrict__ OLP, const int64_t* __restrict__ noff,
                                uint32_t* __restrict__ nnbr, uint32_t* __restrict__ nkey) {
    const int64_t nold = OLP[ntv];
    GRID_STRIDE(f, (uint64_t)nold + side.nins) {
        uint32_t v, x;
        int64_t p;
        if ((int64_t)f < nold) {
            const uint32_t i = owner_of(OLP, ntv, (int64_t)f);
            v = tv[i];
            const uint4 r = gj_delta_ranges(side, v);
            const int64_t t = (int64_t)f - OLP[i];
            x = nbr[off[v] + t];
            const uint32_t* del = side.del_nbr + r.z;
            if (gj_contains(del, r.w - r.z, x)) continue;
            // kept entries before x: t minus the deleted ones; plus the inserts below x
            p = noff[v] + t - (int64_t)lower_count(del, r.w - r.z, x) +
                (int64_t)lower_count(side.ins_nbr + r.x, r.y - r.x, x);
        } else {
            const uint32_t e = (uint32_t)((int64_t)f - nold);
            v = side.ins_key[e];
            x = side.ins_nbr[e];
            const uint4 r = gj_delta_ranges(side, v);
            const int64_t a = off[v], len = off[v + 1] - a;
            p = noff[v] + (int64_t)(e - r.x) + (int64_t)lower_count(nbr + a, (uint64_t)len, x) -
                (int64_t)lower_count(side.del_nbr + r.z, r.w - r.z, x);
        }
        nnbr[p] = x;
        nkey[p] = v;
    }
}

// Clears the next hash sets of the touched vertices (flat over their slots;
// NTP: exclusive sums of their slot counts).
__global__ void k_touched_clear(const uint32_t* __restrict__ tv, uint32_t ntv, const int64_t* __restrict__ NTP,
                                const int64_t* __restrict__ ntoff, uint32_t* __restrict__ ntab) {
    GRID_STRIDE(f, (uint64_t)NTP[ntv]) {
        const uint32_t i = owner_of(NTP, ntv, (int64_t)f);
        ntab[ntoff[tv[i]] + ((int64_t)f - NTP[i])] = GJ_EMPTY;
    }
}

// Fills them from the next lists (flat over the list entries; NLP: exclusive
// sums of the next list lengths), probing as gj_tab_member does: linearly
// from the first slot of the key's home group.
__global__ void k_touched_fill(const uint32_t* __restrict__ tv, uint32_t ntv, const int64_t* __restrict__ NLP,
                               const int64_t* __restrict__ noff, const uint32_t* __restrict__ nnbr,
                               const int64_t* __restrict__ ntoff, uint32_t* __restrict__ ntab) {
    GRID_STRIDE(f, (uint64_t)NLP[ntv]) {
        const uint32_t i = owner_of(NLP, ntv, (int64_t)f);
        const uint32_t v = tv[i];
        const uint32_t len = (uint32_t)(NLP[i + 1] - NLP[i]);
        if (len < GJ_HASH_MIN_DEG) continue;
        const uint32_t bits = gj_tab_bits(len), mask = (1u << bits) - 1u;
        uint32_t* t = ntab + ntoff[v];
        const uint32_t x = nnbr[noff[v] + ((int64_t)f - NLP[i])];
        uint32_t h = gj_tab_start(x, bits);
        for (uint32_t probe = 0; probe <= mask; probe++) {
            if (atomicCAS(t + h, GJ_EMPTY, x) == GJ_EMPTY) break;
            h = (h + 1u) & mask;
        }
    }
}

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

struct Arena {
    char* base;
    size_t used, cap;
    void* take(size_t bytes) {
        char* p = base + used;
        used += (bytes + 255) & ~(size_t)255;
        return used <= cap ? (void*)p : nullptr;
    }
};

int read_i64(gj_ctx* ctx, const int64_t* d, int64_t* h) {
    GJ_CUDA_TRY(ctx, cudaMemcpyAsync(h, d, 8, cudaMemcpyDeviceToHost, ctx->stream));
    GJ_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    return GJ_OK;
}

// Compacts the elements with flag set; returns their count.
int compact_pairs(gj_ctx* ctx, const uint64_t* keys, const uint32_t* own, const uint32_t* nbr, uint64_t n, int vb,
                  const uint32_t* flag, int64_t* pos, uint32_t* okey, uint32_t* onbr, uint32_t* count) {
    GJ_TRY(gj_scan_u32(ctx, flag, pos, n));
    int64_t c = 0;
    GJ_TRY(read_i64(ctx, pos + n, &c));
    if (n) {
        k_pair_compact<<<grid_for(ctx, n), 256, 0, ctx->stream>>>(keys, own, nbr, n, vb, flag, pos, okey, onbr);
        GJ_LAUNCHED(ctx);
    }
    *count = (uint32_t)c;
    return GJ_OK;
}

}  // namespace

void gj_delta_free(gj_ctx* ctx, DeltaBuf* d) {
    if (d->mem) cudaFreeAsync(d->mem, ctx->stream);
    d->mem = nullptr;
    d->batch = DeltaBatch{};
}

int gj_delta_prepare(gj_ctx* ctx, const gj_graph* g, const uint32_t* src, const uint32_t* dst, const int8_t* sign,
                     uint64_t b, DeltaBuf* out) {
    GJ_RANGE("delta: normalise batch");
    cudaStream_t st = ctx->stream;
    const uint64_t bb = b ? b : 1;
    // vertex -> range maps: at most nd distinct vertices per direction, 2x slots
    uint32_t mbits = 1;
    while ((1ull << mbits) < 2 * bb) mbits++;
    const size_t map_bytes = 2 * ((size_t)4 << mbits) + 2 * ((size_t)16 << mbits);
    const size_t bytes = 120 * bb + map_bytes + 72 * 256;
    const int k_src = ptr_kind(src, ctx->device), k_dst = ptr_kind(dst, ctx->device), k_sign = ptr_kind(sign, ctx->device);
    if (b && (k_src < 0 || k_dst < 0 || k_sign < 0)) {
        gj_set_error(ctx, GJ_E_INVALID, "update batch: an input array is in another device's memory");
        return GJ_E_INVALID;
    }
    GJ_CUDA_TRY(ctx, gj_malloc_async(ctx, &out->mem, bytes, st));
    Arena A{(char*)out->mem, 0, bytes};
    const uint32_t* d_src = src;
    const uint32_t* d_dst = dst;
    const int8_t* d_sign = sign;
    if (b && k_src == 0) {
        uint32_t* t = (uint32_t*)A.take(4 * bb);
        GJ_CUDA_TRY(ctx, cudaMemcpyAsync(t, src, 4 * b, cudaMemcpyHostToDevice, st));
        d_src = t;
    }
    if (b && k_dst == 0) {
        uint32_t* t = (uint32_t*)A.take(4 * bb);
        GJ_CUDA_TRY(ctx, cudaMemcpyAsync(t, dst, 4 * b, cudaMemcpyHostToDevice, st));
        d_dst = t;
    }
    if (b && k_sign == 0) {
        int8_t* t = (int8_t*)A.take(bb);
        GJ_CUDA_TRY(ctx, cudaMemcpyAsync(t, sign, b, cudaMemcpyHostToDevice, st));
        d_sign = t;
    }
    uint64_t* keys = (uint64_t*)A.take(8 * bb);
    uint64_t* keys_t = (uint64_t*)A.take(8 * bb);
    uint32_t* idx = (uint32_t*)A.take(4 * bb);
    uint32_t* idx_t = (uint32_t*)A.take(4 * bb);
    uint32_t* flag = (uint32_t*)A.take(4 * bb);
    int64_t* pos = (int64_t*)A.take(8 * (bb + 1));
    int8_t* lsign = (int8_t*)A.take(bb);
    uint32_t* chg_src = (uint32_t*)A.take(4 * bb);
    uint32_t* chg_dst = (uint32_t*)A.take(4 * bb);
    int8_t* chg_sign = (int8_t*)A.take(bb);
    uint32_t* f_ik = (uint32_t*)A.take(4 * bb);
    uint32_t* f_in = (uint32_t*)A.take(4 * bb);
    uint32_t* f_dk = (uint32_t*)A.take(4 * bb);
    uint32_t* f_dn = (uint32_t*)A.take(4 * bb);
    uint32_t* r_ik = (uint32_t*)A.take(4 * bb);
    uint32_t* r_in = (uint32_t*)A.take(4 * bb);
    uint32_t* r_dk = (uint32_t*)A.take(4 * bb);
    uint32_t* r_dn = (uint32_t*)A.take(4 * bb);
    uint32_t* f_hk = (uint32_t*)A.take((size_t)4 << mbits);
    uint4* f_hv = (uint4*)A.take((size_t)16 << mbits);
    uint32_t* r_hk = (uint32_t*)A.take((size_t)4 << mbits);
    uint4* r_hv = (uint4*)A.take((size_t)16 << mbits);
    uint32_t* err = (uint32_t*)A.take(256);
    if (!err) {
        gj_set_error(ctx, GJ_E_NOMEM, "update batch arena too small");
        return GJ_E_NOMEM;
    }
    GJ_CUDA_TRY(ctx, cudaMemsetAsync(err, 0, 4, st));
    const int vb = vertex_bits(g->n);
    const GraphView G = g->view();
    DeltaBatch& D = out->batch;
    D = DeltaBatch{};
    D.chg_src = chg_src;
    D.chg_dst = chg_dst;
    D.chg_sign = chg_sign;
    if (b == 0) return GJ_OK;

    k_dpack<<<grid_for(ctx, b), 256, 0, st>>>(d_src, d_dst, d_sign, b, g->n, vb, keys, idx, err);
    GJ_LAUNCHED(ctx);
    uint64_t* sk = keys;
    uint32_t* si = idx;
    GJ_TRY(gj_radix_sort_kv(ctx, keys, keys_t, idx, idx_t, b, 2 * vb, &sk, &si));
    k_dlast<<<grid_for(ctx, b), 256, 0, st>>>(sk, si, b, d_sign, vb, G, flag, lsign);
    GJ_LAUNCHED(ctx);
    GJ_TRY(gj_scan_u32(ctx, flag, pos, b));
    int64_t nd = 0;
    GJ_TRY(read_i64(ctx, pos + b, &nd));
    uint32_t herr = 0;
    GJ_CUDA_TRY(ctx, cudaMemcpy(&herr, err, 4, cudaMemcpyDeviceToHost));
    if (herr & 1u) {
        gj_set_error(ctx, GJ_E_RANGE, "update batch: vertex id >= num_vertices");
        return GJ_E_RANGE;
    }
    if (herr & 2u) {
        gj_set_error(ctx, GJ_E_INVALID, "update batch: sign must be +1 or -1");
        return GJ_E_INVALID;
    }
    k_dcompact<<<grid_for(ctx, b), 256, 0, st>>>(sk, b, flag, pos, lsign, vb, chg_src, chg_dst, chg_sign);
    GJ_LAUNCHED(ctx);
    D.n = (uint64_t)nd;
    if (nd == 0) return GJ_OK;
    // forward direction: the changes are already sorted by (src, dst)
    DeltaSide& F = D.view.fwd;
    k_sign_flag<<<grid_for(ctx, nd), 256, 0, st>>>(chg_sign, nullptr, nd, 1, flag);
    GJ_LAUNCHED(ctx);
    GJ_TRY(compact_pairs(ctx, nullptr, chg_src, chg_dst, nd, vb, flag, pos, f_ik, f_in, &F.nins));
    k_sign_flag<<<grid_for(ctx, nd), 256, 0, st>>>(chg_sign, nullptr, nd, -1, flag);
    GJ_LAUNCHED(ctx);
    GJ_TRY(compact_pairs(ctx, nullptr, chg_src, chg_dst, nd, vb, flag, pos, f_dk, f_dn, &F.ndel));
    F.ins_key = f_ik;
    F.ins_nbr = f_in;
    F.del_key = f_dk;
    F.del_nbr = f_dn;
    // reverse direction: sort the changes by (dst, src)
    DeltaSide& R = D.view.rev;
    k_rev_keys<<<grid_for(ctx, nd), 256, 0, st>>>(chg_src, chg_dst, nd, vb, keys, idx);
    GJ_LAUNCHED(ctx);
    GJ_TRY(gj_radix_sort_kv(ctx, keys, keys_t, idx, idx_t, nd, 2 * vb, &sk, &si));
    k_sign_flag<<<grid_for(ctx, nd), 256, 0, st>>>(chg_sign, si, nd, 1, flag);
    GJ_LAUNCHED(ctx);
    GJ_TRY(compact_pairs(ctx, sk, nullptr, nullptr, nd, vb, flag, pos, r_ik, r_in, &R.nins));
    k_sign_flag<<<grid_for(ctx, nd), 256, 0, st>>>(chg_sign, si, nd, -1, flag);
    GJ_LAUNCHED(ctx);
    GJ_TRY(compact_pairs(ctx, sk, nullptr, nullptr, nd, vb, flag, pos, r_dk, r_dn, &R.ndel));
    R.ins_key = r_ik;
    R.ins_nbr = r_in;
    R.del_key = r_dk;
    R.del_nbr = r_dn;
    // vertex -> (insert range, delete range) maps of both directions
    uint32_t hb = 1;
    while ((1ull << hb) < 2ull * (uint64_t)nd) hb++;
    GJ_CUDA_TRY(ctx, cudaMemsetAsync(f_hk, 0xff, (size_t)4 << hb, st));
    GJ_CUDA_TRY(ctx, cudaMemsetAsync(r_hk, 0xff, (size_t)4 << hb, st));
    GJ_CUDA_TRY(ctx, cudaMemsetAsync(f_hv, 0, (size_t)16 << hb, st));
    GJ_CUDA_TRY(ctx, cudaMemsetAsync(r_hv, 0, (size_t)16 << hb, st));
    struct Side { DeltaSide* S; uint32_t* hk; uint4* hv; };
    for (Side sd : {Side{&F, f_hk, f_hv}, Side{&R, r_hk, r_hv}}) {
        if (sd.S->nins) {
            k_range_map<<<grid_for(ctx, sd.S->nins), 256, 0, st>>>(sd.S->ins_key, sd.S->nins, 0, sd.hk, sd.hv, hb);
            GJ_LAUNCHED(ctx);
        }
        if (sd.S->ndel) {
            k_range_map<<<grid_for(ctx, sd.S->ndel), 256, 0, st>>>(sd.S->del_key, sd.S->ndel, 1, sd.hk, sd.hv, hb);
            GJ_LAUNCHED(ctx);
        }
        sd.S->hkey = sd.hk;
        sd.S->hval = sd.hv;
        sd.S->hbits = hb;
    }
    GJ_CUDA_TRY(ctx, cudaGetLastError());
    return GJ_OK;
}

void gj_csr_release(gj_csr& c) {
    for (void* p : {(void*)c.off, (void*)c.nbr, (void*)c.key, (void*)c.tab_off, (void*)c.tab})
        if (p) cudaFree(p);
    c = gj_csr{};
}

namespace {

// Arrays of c sized for n vertices, m slots and t hash-set slots, reusing
// those it has (a spare index) when they are large enough.
int ensure_csr(gj_ctx* ctx, gj_csr& c, uint32_t n, uint64_t m, uint64_t t) {
    if (!c.off) GJ_CUDA_TRY(ctx, gj_malloc(ctx, &c.off, sizeof(int64_t) * ((size_t)n + 1)));
    if (!c.tab_off) GJ_CUDA_TRY(ctx, gj_malloc(ctx, &c.tab_off, sizeof(int64_t) * ((size_t)n + 1)));
    if (c.cap_m < (m ? m : 1)) {
        if (c.nbr) cudaFree(c.nbr);
        if (c.key) cudaFree(c.key);
        c.nbr = c.key = nullptr;
        c.cap_m = 0;
        const uint64_t cap = m + m / 16 + 1024;  // room for the growth of later updates
        GJ_CUDA_TRY(ctx, gj_malloc(ctx, &c.nbr, sizeof(uint32_t) * cap));
        GJ_CUDA_TRY(ctx, gj_malloc(ctx, &c.key, sizeof(uint32_t) * cap));
        c.cap_m = cap;
    }
    if (c.cap_tab < (t ? t : 1)) {
        if (c.tab) cudaFree(c.tab);
        c.tab = nullptr;
        c.cap_tab = 0;
        const uint64_t cap = t + t / 16 + 1024;
        GJ_CUDA_TRY(ctx, gj_malloc(ctx, &c.tab, sizeof(uint32_t) * cap));
        c.cap_tab = cap;
    }
    return GJ_OK;
}

// The next version of one index, written into out (whose arrays are reused
// when large enough). Only the touched vertices (list owners of the batch's
// changes in this direction) are recomputed: their lists merged with the
// changes and their hash sets rebuilt; every other list and hash set is
// copied with the constant shift that the touched vertices before it add up
// to (the maintenance proportional to the change of Section 3.3.2, plus one
// coalesced copy of the untouched arrays).
int commit_side(gj_ctx* ctx, uint32_t n, const gj_csr& cur, uint64_t m, const DeltaSide& side, gj_csr& out,
                uint64_t* m_out) {
    cudaStream_t st = ctx->stream;
    const uint64_t nk = (uint64_t)side.nins + side.ndel;  // > 0
    // keys (and the sort's second buffer), flag, tv, then pos, dlen, S, dtab,
    // ST, olen, OLP, nlen, NLP, ntab, NTP; every piece starts on a 256-byte boundary
    const size_t bytes = 16 * nk + 4 * nk + 4 * nk + 11 * 8 * (nk + 1) + 14 * 256;
    char* mem = nullptr;
    GJ_CUDA_TRY(ctx, gj_malloc_async(ctx, &mem, bytes, st));
    Arena A{mem, 0, bytes};
    uint64_t* keys = (uint64_t*)A.take(16 * nk);
    uint32_t* flag = (uint32_t*)A.take(4 * nk);
    int64_t* pos = (int64_t*)A.take(8 * (nk + 1));
    uint32_t* tv = (uint32_t*)A.take(4 * nk);
    int64_t* dlen = (int64_t*)A.take(8 * (nk + 1));
    int64_t* S = (int64_t*)A.take(8 * (nk + 1));
    int64_t* dtab = (int64_t*)A.take(8 * (nk + 1));
    int64_t* ST = (int64_t*)A.take(8 * (nk + 1));
    int64_t* olen = (int64_t*)A.take(8 * (nk + 1));
    int64_t* OLP = (int64_t*)A.take(8 * (nk + 1));
    int64_t* nlen = (int64_t*)A.take(8 * (nk + 1));
    int64_t* NLP = (int64_t*)A.take(8 * (nk + 1));
    int64_t* ntb = (int64_t*)A.take(8 * (nk + 1));
    int64_t* NTP = (int64_t*)A.take(8 * (nk + 1));
    if (!NTP) {  // the pieces above must fit the allocation
        cudaFreeAsync(mem, st);
        gj_set_error(ctx, GJ_E_NOMEM, "update commit: arena too small");
        return GJ_E_NOMEM;
    }
    int rc = GJ_OK;
    int64_t h[3] = {0, 0, 0};  // distinct touched vertices, growth of the lists, of the hash sets
    uint32_t ntv = 0;
    auto step = [&]() -> int {
        k_touch_keys<<<grid_for(ctx, nk), 256, 0, st>>>(side.ins_key, side.nins, side.del_key, side.ndel, keys);
        GJ_LAUNCHED(ctx);
        uint64_t* sorted = keys;
        GJ_TRY(gj_radix_sort_u64(ctx, keys, keys + nk, nk, vertex_bits(n), &sorted));
        k_run_flag<<<grid_for(ctx, nk), 256, 0, st>>>(sorted, nk, flag);
        GJ_LAUNCHED(ctx);
        GJ_TRY(gj_scan_u32(ctx, flag, pos, nk));
        k_run_compact<<<grid_for(ctx, nk), 256, 0, st>>>(sorted, nk, flag, pos, tv);
        GJ_LAUNCHED(ctx);
        GJ_TRY(read_i64(ctx, pos + nk, &h[0]));
        ntv = (uint32_t)h[0];
        k_touch_info<<<grid_for(ctx, ntv), 256, 0, st>>>(tv, ntv, side, cur.off, dlen, dtab, olen, nlen, ntb);
        GJ_LAUNCHED(ctx);
        GJ_TRY(gj_scan_i64(ctx, dlen, S, ntv));
        GJ_TRY(gj_scan_i64(ctx, dtab, ST, ntv));
        GJ_TRY(gj_scan_i64(ctx, olen, OLP, ntv));
        GJ_TRY(gj_scan_i64(ctx, nlen, NLP, ntv));
        GJ_TRY(gj_scan_i64(ctx, ntb, NTP, ntv));
        int64_t hf[3] = {0, 0, 0};  // old entries, next entries, next hash-set slots of the touched vertices
        GJ_CUDA_TRY(ctx, cudaMemcpyAsync(&hf[0], OLP + ntv, 8, cudaMemcpyDeviceToHost, st));
        GJ_CUDA_TRY(ctx, cudaMemcpyAsync(&hf[1], NLP + ntv, 8, cudaMemcpyDeviceToHost, st));
        GJ_CUDA_TRY(ctx, cudaMemcpyAsync(&hf[2], NTP + ntv, 8, cudaMemcpyDeviceToHost, st));
        int64_t t_old = 0;
        GJ_CUDA_TRY(ctx, cudaMemcpyAsync(&h[1], S + ntv, 8, cudaMemcpyDeviceToHost, st));
        GJ_CUDA_TRY(ctx, cudaMemcpyAsync(&h[2], ST + ntv, 8, cudaMemcpyDeviceToHost, st));
        GJ_CUDA_TRY(ctx, cudaMemcpyAsync(&t_old, cur.tab_off + n, 8, cudaMemcpyDeviceToHost, st));
        GJ_CUDA_TRY(ctx, cudaStreamSynchronize(st));
        const uint64_t m2 = (uint64_t)((int64_t)m + h[1]), t2 = (uint64_t)(t_old + h[2]);
        GJ_TRY(ensure_csr(ctx, out, n, m2, t2));
        k_shift_offsets<<<grid_for(ctx, (uint64_t)n + 1), 256, 0, st>>>(cur.off, cur.tab_off, n, tv, ntv, S, ST, out.off,
                                                                         out.tab_off);
        GJ_LAUNCHED(ctx);
        const unsigned regions = (unsigned)(ntv + 1 < (uint64_t)ctx->sm_count * 16 ? ntv + 1 : ctx->sm_count * 16);
        k_shift_copy<<<regions, 256, 0, st>>>(cur.off, cur.tab_off, cur.nbr, cur.key, cur.tab, n, tv, ntv, S, ST,
                                              out.nbr, out.key, out.tab);
        GJ_LAUNCHED(ctx);
        k_merge_touched<<<grid_for(ctx, (uint64_t)hf[0] + side.nins), 256, 0, st>>>(cur.off, cur.nbr, tv, ntv, side,
                                                                                     OLP, out.off, out.nbr, out.key);
        GJ_LAUNCHED(ctx);
        if (hf[2] > 0) {
            k_touched_clear<<<grid_for(ctx, (uint64_t)hf[2]), 256, 0, st>>>(tv, ntv, NTP, out.tab_off, out.tab);
            GJ_LAUNCHED(ctx);
            k_touched_fill<<<grid_for(ctx, (uint64_t)hf[1]), 256, 0, st>>>(tv, ntv, NLP, out.off, out.nbr, out.tab_off,
                                                                            out.tab);
            GJ_LAUNCHED(ctx);
        }
        GJ_CUDA_TRY(ctx, cudaGetLastError());
        *m_out = m2;
        return GJ_OK;
    };
    rc = step();
    cudaFreeAsync(mem, st);
    return rc;
}

}  // namespace

int gj_delta_commit(gj_ctx* ctx, gj_graph* g, const DeltaBatch& d, gj_csr* old_fwd, gj_csr* old_rev) {
    GJ_RANGE("delta: commit (%llu changes)", (unsigned long long)d.n);
    cudaStream_t st = ctx->stream;
    if (d.n == 0) {
        g->version++;
        return GJ_OK;
    }
    // the next version goes into the previous version's arrays when there are some
    gj_csr nf = g->spare_fwd, nr = g->spare_rev;
    g->spare_fwd = gj_csr{};
    g->spare_rev = gj_csr{};
    uint64_t mf = 0, mr = 0;
    int rc = commit_side(ctx, g->n, g->fwd, g->m, d.view.fwd, nf, &mf);
    if (rc == GJ_OK) rc = commit_side(ctx, g->n, g->rev, g->m, d.view.rev, nr, &mr);
    if (rc == GJ_OK && cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        gj_set_error(ctx, GJ_E_CUDA, "update commit: the index kernels failed");
        rc = GJ_E_CUDA;
    }
    if (rc != GJ_OK) {  // the committed graph is unchanged
        gj_csr_release(nf);
        gj_csr_release(nr);
        return rc;
    }
    if (old_fwd && old_rev) {  // readers still in flight keep the previous arrays
        *old_fwd = g->fwd;
        *old_rev = g->rev;
    } else {
        g->spare_fwd = g->fwd;
        g->spare_rev = g->rev;
    }
    g->fwd = nf;
    g->rev = nr;
    g->m = mf;
    g->version++;
    gj_tri_release(g->tri);  // the triangle index described the previous version
    return GJ_OK;
}
