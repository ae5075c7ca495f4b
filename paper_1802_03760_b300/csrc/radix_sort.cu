// Least-significant-digit radix sort of 64-bit keys, 8-bit digits. Each
// pass: per-tile digit histograms, a digit-major exclusive scan of them,
// then a stable scatter in which every warp ranks its keys with
// __match_any_sync. Used by the index builder on packed (vertex, neighbour)
// keys.
#include "gj_internal.cuh"

namespace {

constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ITEMS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;
constexpr int RS_BINS = 256;

// hist[d * ntiles + tile] = number of keys of the tile with digit d.
__global__ void __launch_bounds__(RS_THREADS) k_rs_hist(const uint64_t* __restrict__ keys, uint64_t n, int shift,
                                                       uint32_t* __restrict__ hist, uint32_t ntiles) {
    __shared__ uint32_t h[RS_BINS];
    h[threadIdx.x] = 0;
    __syncthreads();
    uint64_t base = (uint64_t)blockIdx.x * RS_TILE;
#pragma unroll 4
    for (int j = 0; j < RS_ITEMS; j++) {
        uint64_t i = base + (uint64_t)j * RS_THREADS + threadIdx.x;
        if (i < n) atomicAdd(&h[(uint32_t)(keys[i] >> shift) & 0xffu], 1u);
    }
    __syncthreads();
    hist[(uint64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

template <bool VALUES>
__global__ void __launch_bounds__(RS_THREADS) k_rs_scatter(const uint64_t* __restrict__ keys, uint64_t n, int shift,
                                                          const int64_t* __restrict__ digit_off, uint32_t ntiles,
                                                          uint64_t* __restrict__ out, const uint32_t* __restrict__ vin,
                                                          uint32_t* __restrict__ vout) {
    __shared__ uint32_t wcount[RS_WARPS][RS_BINS];
    __shared__ int64_t boff[RS_BINS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int d = lane; d < RS_BINS; d += 32) wcount[warp][d] = 0;
    __syncwarp();
    // keys of this warp, in input order (warp, item, lane)
    const uint64_t wbase = (uint64_t)blockIdx.x * RS_TILE + (uint64_t)warp * 32 * RS_ITEMS;
    uint64_t k[RS_ITEMS];
    uint32_t rank[RS_ITEMS];
    uint32_t val[VALUES ? RS_ITEMS : 1];
    const uint32_t lt = gj_lanemask_lt();
#pragma unroll
    for (int j = 0; j < RS_ITEMS; j++) {
        uint64_t i = wbase + (uint64_t)j * 32 + lane;
        bool valid = i < n;
        k[j] = valid ? keys[i] : 0;
        if (VALUES) val[j] = valid ? vin[i] : 0;
        uint32_t d = valid ? ((uint32_t)(k[j] >> shift) & 0xffu) : RS_BINS;  // invalid lanes form their own group
        uint32_t peers = __match_any_sync(0xffffffffu, d);
        uint32_t before = (d < RS_BINS) ? wcount[warp][d] : 0;
        __syncwarp();
        if (d < RS_BINS && (peers & lt) == 0) wcount[warp][d] = before + __popc(peers);
        __syncwarp();
        rank[j] = before + __popc(peers & lt);
    }
    __syncthreads();
    // per digit: exclusive prefix over warps, and this tile's global offset
    {
        int d = threadIdx.x;
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < RS_WARPS; w++) {
            uint32_t c = wcount[w][d];
            wcount[w][d] = run;
            run += c;
        }
        boff[d] = digit_off[(uint64_t)d * ntiles + blockIdx.x];
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < RS_ITEMS; j++) {
        uint64_t i = wbase + (uint64_t)j * 32 + lane;
        if (i < n) {
            uint32_t d = (uint32_t)(k[j] >> shift) & 0xffu;
            const int64_t pos = boff[d] + wcount[warp][d] + rank[j];
            out[pos] = k[j];
            if (VALUES) vout[pos] = val[j];
        }
    }
}

}  // namespace

namespace {

int radix_sort_impl(gj_ctx* ctx, uint64_t* keys, uint64_t* tmp, uint32_t* vals, uint32_t* vtmp, uint64_t n, int bits,
                    uint64_t** result, uint32_t** vresult) {
    *result = keys;
    if (vresult) *vresult = vals;
    if (n <= 1 || bits <= 0) return GJ_OK;
    uint32_t ntiles = gj_div_up(n, RS_TILE);
    uint64_t nh = (uint64_t)RS_BINS * ntiles;
    uint32_t* hist = nullptr;
    GJ_TRY(gj_scratch(ctx, 2, nh * sizeof(uint32_t) + (nh + 1) * sizeof(int64_t) + 256, (void**)&hist));
    int64_t* off = (int64_t*)(((uintptr_t)(hist + nh) + 255) & ~(uintptr_t)255);
    uint64_t* src = keys;
    uint64_t* dst = tmp;
    uint32_t* vsrc = vals;
    uint32_t* vdst = vtmp;
    for (int shift = 0; shift < bits; shift += 8) {
        k_rs_hist<<<ntiles, RS_THREADS, 0, ctx->stream>>>(src, n, shift, hist, ntiles);
        GJ_LAUNCHED(ctx);
        GJ_TRY(gj_scan_u32(ctx, hist, off, nh));
        if (vals)
            k_rs_scatter<true><<<ntiles, RS_THREADS, 0, ctx->stream>>>(src, n, shift, off, ntiles, dst, vsrc, vdst);
        else
            k_rs_scatter<false><<<ntiles, RS_THREADS, 0, ctx->stream>>>(src, n, shift, off, ntiles, dst, nullptr,
                                                                        nullptr);
        GJ_LAUNCHED(ctx);
        GJ_CUDA_TRY(ctx, cudaGetLastError());
        uint64_t* t = src;
        src = dst;
        dst = t;
        uint32_t* vt = vsrc;
        vsrc = vdst;
        vdst = vt;
    }
    *result = src;
    if (vresult) *vresult = vsrc;
    return GJ_OK;
}

}  // namespace

int gj_radix_sort_u64(gj_ctx* ctx, uint64_t* keys, uint64_t* tmp, uint64_t n, int bits, uint64_t** result) {
    return radix_sort_impl(ctx, keys, tmp, nullptr, nullptr, n, bits, result, nullptr);
}

int gj_radix_sort_kv(gj_ctx* ctx, uint64_t* keys, uint64_t* ktmp, uint32_t* vals, uint32_t* vtmp, uint64_t n, int bits,
                     uint64_t** kresult, uint32_t** vresult) {
    return radix_sort_impl(ctx, keys, ktmp, vals, vtmp, n, bits, kresult, vresult);
}
