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

// flag[e] = 1 if index slot e (owner key[e], neighbour nbr[e]) survives the
// batch's deletions in that direction.
__global__ void k_keep_slots(const uint32_t* __restrict__ key, const uint32_t* __restrict__ nbr, uint64_t m,
                             DeltaSide side, uint32_t* __restrict__ flag) {
    GRID_STRIDE(e, m) {
        const uint32_t u = key[e], v = nbr[e];
        const uint4 r = gj_delta_ranges(side, u);
        flag[e] = gj_contains(side.del_nbr + r.z, r.w - r.z, v) ? 0u : 1u;
    }
}

// Merges two (owner, neighbour)-sorted slot lists without common pairs: each
// element's output position is its own index plus the number of elements of
// the other list that sort before it.
__global__ void k_merge_slots(const uint32_t* __restrict__ ak, const uint32_t* __restrict__ an, uint64_t na,
                              const uint32_t* __restrict__ bk, const uint32_t* __restrict__ bn, uint64_t nb,
                              uint32_t* __restrict__ ok, uint32_t* __restrict__ on) {
    GRID_STRIDE(i, na + nb) {
        const bool in_a = i < na;
        const uint64_t j = in_a ? i : i - na;
        const uint32_t k = in_a ? ak[j] : bk[j];
        const uint32_t x = in_a ? an[j] : bn[j];
        const uint64_t key = ((uint64_t)k << 32) | x;
        const uint32_t* ok_ = in_a ? bk : ak;
        const uint32_t* on_ = in_a ? bn : an;
        uint64_t lo = 0, hi = in_a ? nb : na;
        while (lo < hi) {
            const uint64_t mid = (lo + hi) >> 1;
            const uint64_t mk = ((uint64_t)ok_[mid] << 32) | on_[mid];
            if (mk < key) lo = mid + 1; else hi = mid;
        }
        ok[j + lo] = k;
        on[j + lo] = x;
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
    GJ_CUDA_TRY(ctx, cudaMallocAsync(&out->mem, bytes, st));
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

// The next version of one index: the committed slots minus the batch's
// deletions, merged with its (sorted) inserts, then offsets and hash sets.
int commit_side(gj_ctx* ctx, uint32_t n, const gj_csr& cur, uint64_t m, const DeltaSide& side, gj_csr* out,
                uint64_t* m_out) {
    cudaStream_t st = ctx->stream;
    const uint64_t mm = m ? m : 1;
    const uint64_t m2 = m - side.ndel + side.nins;
    char* mem = nullptr;
    const size_t bytes = 4 * mm + 8 * (mm + 1) + 8 * mm + 4 * 256;
    GJ_CUDA_TRY(ctx, cudaMallocAsync(&mem, bytes, st));
    Arena A{mem, 0, bytes};
    uint32_t* flag = (uint32_t*)A.take(4 * mm);
    int64_t* pos = (int64_t*)A.take(8 * (mm + 1));
    uint32_t* kk = (uint32_t*)A.take(4 * mm);
    uint32_t* kn = (uint32_t*)A.take(4 * mm);
    uint32_t kept = 0;
    int rc = GJ_OK;
    if (m) {
        k_keep_slots<<<grid_for(ctx, m), 256, 0, st>>>(cur.key, cur.nbr, m, side, flag);
        GJ_LAUNCHED(ctx);
        rc = compact_pairs(ctx, nullptr, cur.key, cur.nbr, m, 0, flag, pos, kk, kn, &kept);
    }
    if (rc == GJ_OK && cudaMalloc(&out->key, 4 * (size_t)(m2 ? m2 : 1)) != cudaSuccess) rc = GJ_E_NOMEM;
    if (rc == GJ_OK && cudaMalloc(&out->nbr, 4 * (size_t)(m2 ? m2 : 1)) != cudaSuccess) rc = GJ_E_NOMEM;
    if (rc == GJ_OK && (uint64_t)kept + side.nins > 0) {
        k_merge_slots<<<grid_for(ctx, kept + side.nins), 256, 0, st>>>(kk, kn, kept, side.ins_key, side.ins_nbr,
                                                                      side.nins, out->key, out->nbr);
        GJ_LAUNCHED(ctx);
    }
    cudaFreeAsync(mem, st);
    if (rc == GJ_OK) rc = gj_csr_finish(ctx, n, m2, out);
    *m_out = m2;
    return rc;
}

}  // namespace

int gj_delta_commit(gj_ctx* ctx, gj_graph* g, const DeltaBatch& d, gj_csr* old_fwd, gj_csr* old_rev) {
    cudaStream_t st = ctx->stream;
    if (d.n == 0) {
        g->version++;
        return GJ_OK;
    }
    gj_csr nf, nr;
    uint64_t mf = 0, mr = 0;
    int rc = commit_side(ctx, g->n, g->fwd, g->m, d.view.fwd, &nf, &mf);
    if (rc == GJ_OK) rc = commit_side(ctx, g->n, g->rev, g->m, d.view.rev, &nr, &mr);
    if (rc != GJ_OK) {
        gj_csr_release(nf);
        gj_csr_release(nr);
        return rc;
    }
    GJ_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    if (old_fwd && old_rev) {
        *old_fwd = g->fwd;
        *old_rev = g->rev;
    } else {
        gj_csr_release(g->fwd);
        gj_csr_release(g->rev);
    }
    g->fwd = nf;
    g->rev = nr;
    g->m = mf;
    g->version++;
    gj_tri_release(g->tri);  // the triangle index described the previous version
    return GJ_OK;
}
