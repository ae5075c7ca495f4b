// Device-wide exclusive prefix sums (reduce, scan the block totals, scan
// each tile with its block offset). Used for candidate offsets of the
// prefix buffers, compaction offsets and radix-sort digit offsets.
#include "gj_internal.cuh"

namespace {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

template <typename T>
__global__ void __launch_bounds__(SCAN_THREADS) k_tile_sums(const T* __restrict__ in, uint64_t n,
                                                           int64_t* __restrict__ sums) {
    __shared__ int64_t warp_sums[SCAN_THREADS / 32];
    uint64_t base = (uint64_t)blockIdx.x * SCAN_TILE;
    int64_t s = 0;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; j++) {
        uint64_t i = base + (uint64_t)j * SCAN_THREADS + threadIdx.x;
        if (i < n) s += (int64_t)in[i];
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) warp_sums[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t t = 0;
        for (int w = 0; w < SCAN_THREADS / 32; w++) t += warp_sums[w];
        sums[blockIdx.x] = t;
    }
}

// Exclusive scan of one tile, offset by tile_off[blockIdx.x] (or 0).
template <typename T>
__global__ void __launch_bounds__(SCAN_THREADS) k_tile_scan(const T* __restrict__ in, uint64_t n,
                                                           const int64_t* __restrict__ tile_off,
                                                           int64_t* __restrict__ out) {
    __shared__ int64_t warp_tot[SCAN_THREADS / 32];
    uint64_t base = (uint64_t)blockIdx.x * SCAN_TILE + (uint64_t)threadIdx.x * SCAN_ITEMS;
    int64_t v[SCAN_ITEMS];
    int64_t s = 0;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; j++) {
        uint64_t i = base + j;
        v[j] = (i < n) ? (int64_t)in[i] : 0;
        s += v[j];
    }
    // exclusive scan of thread sums across the block
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t incl = s;
    for (int o = 1; o < 32; o <<= 1) {
        int64_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    int64_t wpre = 0;
    for (int w = 0; w < warp; w++) wpre += warp_tot[w];
    int64_t run = (tile_off ? tile_off[blockIdx.x] : 0) + wpre + incl - s;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; j++) {
        uint64_t i = base + j;
        if (i < n) out[i] = run;
        run += v[j];
    }
    // the last thread of the last tile ends with the grand total: out[n]
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == SCAN_THREADS - 1) out[n] = run;
}

uint64_t scan_work(uint64_t n) {
    uint64_t nt = (n + SCAN_TILE - 1) / SCAN_TILE;
    return nt <= 1 ? 1 : 2 * nt + 1 + scan_work(nt);
}

// work holds scan_work(n) int64 values.
template <typename T>
void scan_rec(cudaStream_t st, const T* in, int64_t* out, uint64_t n, int64_t* work) {
    uint64_t nt = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (nt <= 1) {
        k_tile_scan<T><<<1, SCAN_THREADS, 0, st>>>(in, n, nullptr, out);
        return;
    }
    int64_t* sums = work;
    int64_t* offs = work + nt;  // nt + 1 values
    k_tile_sums<T><<<(unsigned)nt, SCAN_THREADS, 0, st>>>(in, n, sums);
    scan_rec<int64_t>(st, sums, offs, nt, work + 2 * nt + 1);
    k_tile_scan<T><<<(unsigned)nt, SCAN_THREADS, 0, st>>>(in, n, offs, out);
}

template <typename T>
int scan_impl(gj_ctx* ctx, const T* in, int64_t* out, uint64_t n) {
    if (n == 0) {
        GJ_CUDA_TRY(ctx, cudaMemsetAsync(out, 0, sizeof(int64_t), ctx->stream));
        return GJ_OK;
    }
    int64_t* work = nullptr;
    GJ_TRY(gj_scratch(ctx, 3, sizeof(int64_t) * scan_work(n), (void**)&work));
    scan_rec<T>(ctx->stream, in, out, n, work);
    for (uint64_t m = n;; m = (m + SCAN_TILE - 1) / SCAN_TILE) {  // 1 launch per single-tile level, else 2
        if (m <= (uint64_t)SCAN_TILE) { GJ_LAUNCHED(ctx); break; }
        GJ_LAUNCHED(ctx);
        GJ_LAUNCHED(ctx);
    }
    GJ_CUDA_TRY(ctx, cudaGetLastError());
    return GJ_OK;
}

}  // namespace

int gj_scan_u32(gj_ctx* ctx, const uint32_t* in, int64_t* out, uint64_t n) {
    return scan_impl<uint32_t>(ctx, in, out, n);
}

int gj_scan_i64(gj_ctx* ctx, const int64_t* in, int64_t* out, uint64_t n) {
    return scan_impl<int64_t>(ctx, in, out, n);
}
