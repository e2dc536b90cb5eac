// Tile plans for the fixed-list pair passes (TL, Sec. 3.2).
//
// The rows are cut into tiles of kTileRows consecutive particles.  In Morton
// order (sph_cell_order) a tile is a compact group of cells whose rows share most
// of their neighbours.  The plan lists, per tile, the distinct columns of its rows
// (ascending), so that a pass can stage those neighbours' data in shared memory
// once per tile, and lays the tile's pairs out in a sliced order (pair k of row r
// at k * kTileRows + r) so that the threads of a warp, one row each, read
// consecutive 16-byte entries.  Lists and reference positions are fixed in the
// total-Lagrangian method, so a plan is built once, when the float32 state is
// packed, and the per-pair entries can carry precomputed geometry.
#pragma once
#include "common.cuh"

constexpr int kTileRows = 128;

// Plan buffer layout (a 32-byte aligned buffer; 16-byte aligned sections, the
// entry section 32-byte aligned):
//   int32  hdr[16]          [0] most distinct columns of a tile, [1] most pairs of a
//                           tile, [2] longest row
//   int32  tile_m[ntiles]   distinct columns of tile b
//   int32  tile_e[ntiles]   sliced entries of tile b: kTileRows * (longest row of b)
//   int64  tile_so[ntiles+1] first sliced entry of tile b (exclusive scan of tile_e)
//   int32  uidx[nnz]        tile b's distinct columns at uidx[row_ptr[b*kTileRows] + k],
//                           k < tile_m[b]
//   uint16 lcol[nnz]        position of col[p] among its tile's distinct columns
//   geo[ntiles * kTileRows * maxrow]  sliced per-pair entries of `ebytes` bytes (a
//                           multiple of 16), filled by the method that uses the plan;
//                           padding entries are zero
struct TilePlan {
    int32_t* hdr;
    int32_t* tile_m;
    int32_t* tile_e;
    int64_t* tile_so;
    int32_t* uidx;
    uint16_t* lcol;
    float4* geo;
    int64_t ntiles;
};

static inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

static inline size_t align32(size_t x) { return (x + 31) & ~(size_t)31; }

// Offset of the entry section: 32-byte aligned (entries are read with 256-bit
// loads; the plan buffer itself must be 32-byte aligned).
static inline size_t tile_plan_geo_offset(int64_t n, int64_t nnz) {
    int64_t ntiles = (n + kTileRows - 1) / kTileRows;
    return align32(64 + 2 * align16((size_t)ntiles * 4) + align16((size_t)(ntiles + 1) * 8) +
                   align16((size_t)nnz * 4) + align16((size_t)nnz * 2));
}

static inline size_t tile_plan_bytes(int64_t n, int64_t nnz, int64_t maxrow, int ebytes = 16) {
    int64_t ntiles = (n + kTileRows - 1) / kTileRows;
    return tile_plan_geo_offset(n, nnz) + (size_t)ntiles * kTileRows * (size_t)maxrow * (size_t)ebytes;
}

static inline TilePlan tile_plan_view(void* buf, int64_t n, int64_t nnz) {
    TilePlan t;
    unsigned char* b = (unsigned char*)buf;
    t.ntiles = (n + kTileRows - 1) / kTileRows;
    t.hdr = (int32_t*)b;
    b += 64;
    t.tile_m = (int32_t*)b;
    b += align16((size_t)t.ntiles * 4);
    t.tile_e = (int32_t*)b;
    b += align16((size_t)t.ntiles * 4);
    t.tile_so = (int64_t*)b;
    b += align16((size_t)(t.ntiles + 1) * 8);
    t.uidx = (int32_t*)b;
    b += align16((size_t)nnz * 4);
    t.lcol = (uint16_t*)b;
    t.geo = (float4*)((unsigned char*)buf + tile_plan_geo_offset(n, nnz));
    return t;
}

// Reads nnz = row_ptr[n] and the longest row (synchronises the stream).
int sph_row_stats(sph_ctx* ctx, const int64_t* row_ptr, int64_t n, cudaStream_t s, int64_t* nnz,
                  int64_t* maxrow);

// Builds the index part of the plan of (row_ptr, col) into buf (at least
// tile_plan_bytes(n, nnz, maxrow) bytes, 32-byte aligned): hdr, tile_m, tile_e,
// tile_so, uidx and lcol.  Returns the three header maxima on the host
// (synchronises the stream).
int sph_build_tile_plan(sph_ctx* ctx, const int64_t* row_ptr, const int32_t* col, int64_t n, int64_t nnz,
                        void* buf, cudaStream_t s, int32_t* maxm, int32_t* maxp, int32_t* maxw);

// Shared-memory records of the distinct columns staged per tile: `planes` arrays
// of mcap float4, mcap = the plan's maximum, within 96 KB and within `cap` when
// cap > 0 (sph_set_stage_cap).  Tiles with more distinct columns than mcap read
// their neighbours from global memory instead.
static inline int stage_mcap(int32_t maxm, int planes, int cap) {
    const size_t limit = 96 * 1024;
    int64_t room = (int64_t)(limit / (16 * (size_t)planes));
    int64_t m = maxm < 1 ? 1 : maxm;
    if (m > room) m = room;
    if (cap > 0 && m > cap) m = cap;
    return (int)m;
}

// Row order of the sliced entries: a row's pairs are laid out by their offset
// r_i - r_j quantised to h/2 (z, y, x major to minor), then by list position, so
// that at a given position the threads of a warp, neighbouring rows, tend to read
// neighbours at the same offset.  rfun(k, r) gives the float64 offset of the row's
// k-th pair.  Returns false (list order kept) for rows longer than kSortCap.
constexpr int kSortCap = 128;

template <int DIM, typename RF>
__device__ __forceinline__ bool offset_order(int len, double two_over_h, RF rfun, uint32_t* order) {
    if (len > kSortCap) return false;
    for (int k = 0; k < len; ++k) {
        double r[3];
        rfun(k, r);
        uint32_t key = 0;
#pragma unroll
        for (int a = DIM - 1; a >= 0; --a) {
            double q = rint(r[a] * two_over_h);
            int c = (int)fmin(fmax(q, -8.0), 7.0) + 8;
            key = key * 16u + (uint32_t)c;
        }
        uint32_t v = (key << 20) | (uint32_t)k;
        int at = k;
        while (at > 0 && order[at - 1] > v) {
            order[at] = order[at - 1];
            --at;
        }
        order[at] = v;
    }
    return true;
}
