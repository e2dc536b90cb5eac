// Tile-plan builder (see tiles.cuh).  One block per tile: the tile's columns are
// marked in a shared-memory bitmap over a window of column indices, a prefix sum
// of the bitmap's popcounts ranks every marked column, and the ranks give both
// the ascending distinct-column list and each pair's local index.  Windows are
// taken in turn from the tile's smallest to its largest column, so any spread of
// columns (periodic wrap, unordered particles) is handled.
#include <climits>
#include "tiles.cuh"

namespace {

constexpr int kPlanThreads = 256;
constexpr int kPlanWords = 4096;             // bitmap words per window: 131072 columns
constexpr int kWordsPerThread = kPlanWords / kPlanThreads;

__global__ void __launch_bounds__(kPlanThreads) k_tile_plan(const int64_t* __restrict__ row_ptr,
                                                            const int32_t* __restrict__ col, int64_t n,
                                                            int32_t* __restrict__ hdr, int32_t* __restrict__ tile_m,
                                                            int32_t* __restrict__ tile_e, int32_t* __restrict__ uidx,
                                                            uint16_t* __restrict__ lcol) {
    __shared__ uint32_t bm[kPlanWords];
    __shared__ int32_t wpre[kPlanWords];
    __shared__ int32_t wsum[kPlanThreads / 32];
    __shared__ int32_t range[3];
    const int tid = threadIdx.x, T = kPlanThreads, NW = kPlanThreads / 32;
    const int64_t tile = blockIdx.x;
    const int64_t i0 = tile * kTileRows;
    const int64_t i1 = i0 + kTileRows < n ? i0 + kTileRows : n;
    const int64_t P0 = row_ptr[i0], P1 = row_ptr[i1];
    if (tid == 0) { range[0] = INT_MAX; range[1] = -1; range[2] = 0; }
    __syncthreads();
    // longest row of the tile
    if (tid < kTileRows && i0 + tid < i1) {
        int64_t len = row_ptr[i0 + tid + 1] - row_ptr[i0 + tid];
        atomicMax(&range[2], (int)(len < INT_MAX ? len : INT_MAX));
    }
    int lo = INT_MAX, hi = -1;
    for (int64_t p = P0 + tid; p < P1; p += T) {
        int j = col[p];
        lo = min(lo, j);
        hi = max(hi, j);
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if ((tid & 31) == 0) {
        atomicMin(&range[0], lo);
        atomicMax(&range[1], hi);
    }
    __syncthreads();
    const int64_t jmin = range[0], jmax = range[1];
    const int64_t span = 32LL * kPlanWords;
    int base = 0;
    for (int64_t w0 = jmin; w0 <= jmax; w0 += span) {
        for (int w = tid; w < kPlanWords; w += T) bm[w] = 0u;
        __syncthreads();
        for (int64_t p = P0 + tid; p < P1; p += T) {
            int64_t d = (int64_t)col[p] - w0;
            if (d >= 0 && d < span) atomicOr(&bm[d >> 5], 1u << (d & 31));
        }
        __syncthreads();
        // exclusive prefix of the word popcounts; thread t owns a run of words
        int own = 0;
        for (int k = 0; k < kWordsPerThread; ++k) own += __popc(bm[tid * kWordsPerThread + k]);
        int incl = own;
        for (int o = 1; o < 32; o <<= 1) {
            int v = __shfl_up_sync(0xffffffffu, incl, o);
            if ((tid & 31) >= o) incl += v;
        }
        if ((tid & 31) == 31) wsum[tid >> 5] = incl;
        __syncthreads();
        int before = 0, total = 0;
        for (int w = 0; w < NW; ++w) {
            if (w < (tid >> 5)) before += wsum[w];
            total += wsum[w];
        }
        int run = before + incl - own;
        for (int k = 0; k < kWordsPerThread; ++k) {
            int w = tid * kWordsPerThread + k;
            wpre[w] = run;
            run += __popc(bm[w]);
        }
        __syncthreads();
        // the distinct columns in ascending order
        for (int w = tid; w < kPlanWords; w += T) {
            uint32_t bits = bm[w];
            int r = base + wpre[w];
            while (bits) {
                int bit = __ffs(bits) - 1;
                uidx[P0 + r] = (int32_t)(w0 + 32LL * w + bit);
                ++r;
                bits &= bits - 1u;
            }
        }
        // each pair's local index
        for (int64_t p = P0 + tid; p < P1; p += T) {
            int64_t d = (int64_t)col[p] - w0;
            if (d >= 0 && d < span) {
                int w = (int)(d >> 5), bit = (int)(d & 31);
                int slot = base + wpre[w] + __popc(bm[w] & ((1u << bit) - 1u));
                lcol[p] = (uint16_t)(slot < 65535 ? slot : 65535);
            }
        }
        base += total;
        __syncthreads();
    }
    if (tid == 0) {
        tile_m[tile] = base;
        tile_e[tile] = kTileRows * range[2];
        int64_t np = P1 - P0;
        atomicMax(&hdr[0], base);
        atomicMax(&hdr[1], (int)(np < INT_MAX ? np : INT_MAX));
        atomicMax(&hdr[2], range[2]);
    }
}

__global__ void k_max_row(const int64_t* __restrict__ row_ptr, int64_t n, unsigned long long* __restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long len = i < n ? (unsigned long long)(row_ptr[i + 1] - row_ptr[i]) : 0ull;
    for (int o = 16; o > 0; o >>= 1) len = max(len, __shfl_xor_sync(0xffffffffu, len, o));
    if ((threadIdx.x & 31) == 0 && len) atomicMax(out, len);
}

}  // namespace

int sph_row_stats(sph_ctx* ctx, const int64_t* row_ptr, int64_t n, cudaStream_t s, int64_t* nnz, int64_t* maxrow) {
    int st = SPH_OK;
    unsigned long long* d = (unsigned long long*)sph_scratch(ctx, S_MISC2, 64, &st);
    if (st) return st;
    SPH_CUDA(ctx, cudaMemsetAsync(d, 0, 8, s));
    if (n > 0) k_max_row<<<grid_for(n, 256), 256, 0, s>>>(row_ptr, n, d);
    SPH_LAUNCH_CHECK(ctx);
    int64_t* h = (int64_t*)ctx->pinned;
    SPH_CUDA(ctx, cudaMemcpyAsync(h, row_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    SPH_CUDA(ctx, cudaMemcpyAsync(h + 1, d, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    SPH_CUDA(ctx, cudaStreamSynchronize(s));
    *nnz = h[0];
    *maxrow = h[1];
    return SPH_OK;
}

int sph_build_tile_plan(sph_ctx* ctx, const int64_t* row_ptr, const int32_t* col, int64_t n, int64_t nnz,
                        void* buf, cudaStream_t s, int32_t* maxm, int32_t* maxp, int32_t* maxw) {
    if (((uintptr_t)buf & 31u) || n < 1) return SPH_ERR_ARG;
    TilePlan t = tile_plan_view(buf, n, nnz);
    SPH_CUDA(ctx, cudaMemsetAsync(t.hdr, 0, 64, s));
    k_tile_plan<<<(unsigned)t.ntiles, kPlanThreads, 0, s>>>(row_ptr, col, n, t.hdr, t.tile_m, t.tile_e, t.uidx,
                                                            t.lcol);
    SPH_LAUNCH_CHECK(ctx);
    int st = sph_exclusive_scan_i64(ctx, t.tile_e, t.tile_so, t.ntiles, s);
    if (st) return st;
    int32_t* h = (int32_t*)ctx->pinned;
    SPH_CUDA(ctx, cudaMemcpyAsync(h, t.hdr, 3 * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    SPH_CUDA(ctx, cudaStreamSynchronize(s));
    *maxm = h[0];
    *maxp = h[1];
    *maxw = h[2];
    return SPH_OK;
}
