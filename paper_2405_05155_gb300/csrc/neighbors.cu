// a1 cell binning / ordering and a2 CSR neighbour lists (compact support, Eq. 5).
//
// Design: a counting sort of the particles by linear cell id (cells of edge
// >= kappa h) gives, per cell, a contiguous run of particle indices in
// ascending order.  Each particle then visits the distinct neighbouring cells
// (1-3 per axis, ascending ids) and tests the candidates.  The test must equal
// the float64 definition bit for bit, but GB300's float64 rate is low, so
// candidates are first screened in float32 against thresholds rc^2 -/+ delta,
// where delta bounds the float32 error of the squared distance (position
// rounding, subtraction, minimum image and the sum of squares); only the few
// candidates inside the band are decided in float64 with unfused multiply and
// add.  When the particles are themselves stored in cell order (the layout the
// pair loops use) the visit order already yields ascending j; otherwise a row is
// sorted in place.
#include <math.h>
#include "neighbors.cuh"

using namespace nb;

namespace {

__global__ void k_cell_ids(const double* __restrict__ pos, int64_t n, CellGrid g,
                           int32_t* __restrict__ cid, int32_t* __restrict__ count,
                           int* __restrict__ flags, unsigned* __restrict__ absmax) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float m = 0.0f;
    if (i < n) {
        int c[3] = {0, 0, 0};
        bool bad = false;
        for (int k = 0; k < g.dim; ++k) {
            double x = pos[k * n + i];
            if (!isfinite(x)) bad = true;
            if ((g.periodic >> k) & 1u) {
                if (!(x >= g.lo[k] && x <= g.lo[k] + g.len[k])) bad = true;
            }
            c[k] = cell_coord(x, k, g);
            m = fmaxf(m, __double2float_ru(fabs(x)));
        }
        if (bad) { atomicExch(&flags[FLAG_BAD_INPUT], 1); c[0] = c[1] = c[2] = 0; m = 0.0f; }
        int id = (c[2] * g.n[1] + c[1]) * g.n[0] + c[0];
        cid[i] = id;
        atomicAdd(&count[id], 1);
    }
    // non-negative floats order like their bit patterns; one atomic per warp
    unsigned wm = __reduce_max_sync(0xffffffffu, __float_as_uint(m));
    if ((threadIdx.x & 31) == 0 && wm) atomicMax(absmax, wm);
}

// Morton (Z-order) key of a cell: bit l of the coordinate on axis a goes to the
// next free key position, level by level from the least significant bit, axes in
// order x, y, z; an axis drops out once its bits (ceil(log2 n_a)) are used up, so
// the keys of the grid lie in [0, 2^(sum of bits)), at most 2^dim times the cells.
struct MortonBits {
    int bits[3];
    int total;
};

MortonBits morton_bits(const CellGrid& g) {
    MortonBits mb;
    mb.total = 0;
    for (int a = 0; a < 3; ++a) {
        int b = 0;
        if (a < g.dim)
            while ((1LL << b) < (long long)g.n[a]) ++b;
        mb.bits[a] = b;
        mb.total += b;
    }
    return mb;
}

__device__ __forceinline__ int32_t morton_key(const int* c, const MortonBits& mb, int dim) {
    uint32_t key = 0;
    int at = 0;
    for (int l = 0; l < 21; ++l)
        for (int a = 0; a < dim; ++a)
            if (l < mb.bits[a]) key |= (uint32_t)((c[a] >> l) & 1) << at++;
    return (int32_t)key;
}

__global__ void k_morton_ids(const double* __restrict__ pos, int64_t n, CellGrid g, MortonBits mb,
                             int32_t* __restrict__ key, int32_t* __restrict__ count, int* __restrict__ flags) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int c[3] = {0, 0, 0};
    bool bad = false;
    for (int k = 0; k < g.dim; ++k) {
        double x = pos[k * n + i];
        if (!isfinite(x)) bad = true;
        if ((g.periodic >> k) & 1u) {
            if (!(x >= g.lo[k] && x <= g.lo[k] + g.len[k])) bad = true;
        }
        c[k] = cell_coord(x, k, g);
    }
    if (bad) { atomicExch(&flags[FLAG_BAD_INPUT], 1); c[0] = c[1] = c[2] = 0; }
    int32_t id = morton_key(c, mb, g.dim);
    key[i] = id;
    atomicAdd(&count[id], 1);
}

__global__ void k_scatter(const int32_t* __restrict__ cid, int64_t n, const int32_t* __restrict__ start,
                          int32_t* __restrict__ fill, int32_t* __restrict__ sorted) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int c = cid[i];
    int slot = atomicAdd(&fill[c], 1);
    sorted[start[c] + slot] = (int32_t)i;
}

// Restore index order inside each cell (the scatter order is arbitrary).
__global__ void k_sort_cells(const int32_t* __restrict__ start, int64_t ncell, int32_t* __restrict__ sorted) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    int b = start[c], e = start[c + 1];
    for (int a = b + 1; a < e; ++a) {
        int v = sorted[a];
        int k = a - 1;
        while (k >= b && sorted[k] > v) { sorted[k + 1] = sorted[k]; --k; }
        sorted[k + 1] = v;
    }
}

__global__ void k_pack_sorted(const double* __restrict__ pos, int64_t n, int dim,
                              const int32_t* __restrict__ sorted, float4* __restrict__ p32) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    int j = sorted[k];
    float4 p;
    p.x = (float)pos[j];
    p.y = (float)pos[n + j];
    p.z = dim == 3 ? (float)pos[2 * n + j] : 0.0f;
    p.w = __int_as_float(j);
    p32[k] = p;
}

template <int DIM, bool FILL>
__global__ void k_neighbors(const double* __restrict__ pos, int64_t n, CellGrid g, double rc2, double lmax,
                            const unsigned* __restrict__ absmax, const int32_t* __restrict__ start,
                            const float4* __restrict__ p32, int32_t* __restrict__ row_len,
                            const int64_t* __restrict__ row_ptr, int32_t* __restrict__ col,
                            int64_t cap, int* __restrict__ flags) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (FILL && row_ptr[n] > cap) {
        if (i == 0) atomicExch(&flags[FLAG_CAPACITY], 1);
        return;
    }
    Band band = make_band(absmax, lmax, rc2, DIM);
    double xi[3] = {0.0, 0.0, 0.0};
    float xf[3] = {0.0f, 0.0f, 0.0f};
    int ci[3] = {0, 0, 0};
    for (int k = 0; k < DIM; ++k) {
        xi[k] = pos[k * n + i];
        xf[k] = (float)xi[k];
        ci[k] = cell_coord(xi[k], k, g);
    }
    float Lf[3], Hf[3];
    for (int k = 0; k < 3; ++k) { Lf[k] = (float)g.len[k]; Hf[k] = (float)g.half[k]; }
    int lx[3], ly[3], lz[3] = {0, 0, 0};
    int mx = axis_cells(ci[0], 0, g, lx);
    int my = axis_cells(ci[1], 1, g, ly);
    int mz = DIM == 3 ? axis_cells(ci[2], 2, g, lz) : 1;
    int cnt = 0;
    int64_t base_out = FILL ? row_ptr[i] : 0;
    int last = -1;
    bool ordered = true;
    for (int az = 0; az < mz; ++az) {
        for (int ay = 0; ay < my; ++ay) {
            int rowbase = (lz[az] * g.n[1] + ly[ay]) * g.n[0];
            for (int ax = 0; ax < mx; ++ax) {
                int c = rowbase + lx[ax];
                int b = start[c], e = start[c + 1];
                for (int k = b; k < e; ++k) {
                    float4 p = p32[k];
                    int j = __float_as_int(p.w);
                    if (j == (int)i) continue;
                    float pj[3] = {p.x, p.y, p.z};
                    float d2 = 0.0f;
#pragma unroll
                    for (int a = 0; a < DIM; ++a) {
                        float dx = xf[a] - pj[a];
                        if ((g.periodic >> a) & 1u) {
                            if (dx > Hf[a]) dx -= Lf[a];
                            else if (dx < -Hf[a]) dx += Lf[a];
                        }
                        d2 = fmaf(dx, dx, d2);
                    }
                    bool in;
                    if (d2 < band.lo) in = true;
                    else if (d2 > band.hi) in = false;
                    else in = exact_within(pos, n, DIM, xi, j, g, rc2);
                    if (in) {
                        if (FILL) {
                            col[base_out + cnt] = j;
                            if (j < last) ordered = false;
                            last = j;
                        }
                        ++cnt;
                    }
                }
            }
        }
    }
    if (!FILL) {
        row_len[i] = cnt;
    } else if (!ordered) {
        int32_t* row = col + base_out;
        for (int a = 1; a < cnt; ++a) {
            int v = row[a];
            int k = a - 1;
            while (k >= 0 && row[k] > v) { row[k + 1] = row[k]; --k; }
            row[k + 1] = v;
        }
    }
}

__global__ void k_widen_order(const int32_t* __restrict__ sorted, int64_t n, int64_t* __restrict__ order) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) order[k] = sorted[k];
}

double periodic_lmax(const CellGrid& g) {
    double m = 0.0;
    for (int k = 0; k < g.dim; ++k)
        if ((g.periodic >> k) & 1u) m = fmax(m, g.len[k]);
    return m;
}

}  // namespace

int sph_build_cells(sph_ctx* ctx, const sph_domain* dom, const double* pos, cudaStream_t s, CellList* cl) {
    int st = sph_check_domain(dom);
    if (st) return st;
    cl->grid = sph_make_grid(dom);
    const CellGrid& g = cl->grid;
    if (g.total > (1LL << 28)) return SPH_ERR_ARG;
    int64_t n = dom->n;
    cl->cell_id = (int32_t*)sph_scratch(ctx, S_CELL_ID, (size_t)n * 4, &st);
    int32_t* count = (int32_t*)sph_scratch(ctx, S_CELL_COUNT, (size_t)(g.total + 1) * 4, &st);
    cl->cell_start = (int32_t*)sph_scratch(ctx, S_CELL_START, (size_t)(g.total + 1) * 4, &st);
    int32_t* fill = (int32_t*)sph_scratch(ctx, S_CELL_FILL, (size_t)(g.total + 1) * 4, &st);
    cl->sorted = (int32_t*)sph_scratch(ctx, S_SORTED, (size_t)n * 4, &st);
    cl->p32 = (float4*)sph_scratch(ctx, S_P32SORTED, (size_t)n * 16, &st);
    unsigned* absmax = (unsigned*)sph_scratch(ctx, S_ABSMAX, 64, &st);
    if (st) return st;
    cl->band = (float*)absmax;
    SPH_CUDA(ctx, cudaMemsetAsync(count, 0, (size_t)(g.total + 1) * 4, s));
    SPH_CUDA(ctx, cudaMemsetAsync(fill, 0, (size_t)(g.total + 1) * 4, s));
    SPH_CUDA(ctx, cudaMemsetAsync(absmax, 0, 64, s));
    if (n > 0)
        k_cell_ids<<<grid_for(n, 256), 256, 0, s>>>(pos, n, g, cl->cell_id, count, ctx->flags, absmax);
    st = sph_exclusive_scan_i32(ctx, count, cl->cell_start, g.total, s);
    if (st) return st;
    if (n > 0) {
        k_scatter<<<grid_for(n, 256), 256, 0, s>>>(cl->cell_id, n, cl->cell_start, fill, cl->sorted);
        k_sort_cells<<<grid_for(g.total, 128), 128, 0, s>>>(cl->cell_start, g.total, cl->sorted);
        k_pack_sorted<<<grid_for(n, 256), 256, 0, s>>>(pos, n, g.dim, cl->sorted, cl->p32);
    }
    SPH_LAUNCH_CHECK(ctx);
    return SPH_OK;
}

int sph_count_neighbors(sph_ctx* ctx, const CellList& cl, const double* pos, int64_t n, double rc2,
                        int32_t* row_len, cudaStream_t s) {
    if (n == 0) return SPH_OK;
    const unsigned* absmax = (const unsigned*)cl.band;
    double lmax = periodic_lmax(cl.grid);
    if (cl.grid.dim == 2)
        k_neighbors<2, false><<<grid_for(n, 128), 128, 0, s>>>(pos, n, cl.grid, rc2, lmax, absmax, cl.cell_start,
                                                              cl.p32, row_len, nullptr, nullptr, 0, ctx->flags);
    else
        k_neighbors<3, false><<<grid_for(n, 128), 128, 0, s>>>(pos, n, cl.grid, rc2, lmax, absmax, cl.cell_start,
                                                              cl.p32, row_len, nullptr, nullptr, 0, ctx->flags);
    SPH_LAUNCH_CHECK(ctx);
    return SPH_OK;
}

int sph_fill_neighbors(sph_ctx* ctx, const CellList& cl, const double* pos, int64_t n, double rc2,
                       const int64_t* row_ptr, int32_t* col, int64_t cap, cudaStream_t s) {
    if (n == 0) return SPH_OK;
    const unsigned* absmax = (const unsigned*)cl.band;
    double lmax = periodic_lmax(cl.grid);
    if (cl.grid.dim == 2)
        k_neighbors<2, true><<<grid_for(n, 128), 128, 0, s>>>(pos, n, cl.grid, rc2, lmax, absmax, cl.cell_start,
                                                             cl.p32, nullptr, row_ptr, col, cap, ctx->flags);
    else
        k_neighbors<3, true><<<grid_for(n, 128), 128, 0, s>>>(pos, n, cl.grid, rc2, lmax, absmax, cl.cell_start,
                                                             cl.p32, nullptr, row_ptr, col, cap, ctx->flags);
    SPH_LAUNCH_CHECK(ctx);
    return SPH_OK;
}

// Reads back and clears the device flags; returns SPH_ERR_ARG on bad input.
static int take_flags(sph_ctx* ctx, cudaStream_t s, int* host_flags) {
    SPH_CUDA(ctx, cudaMemcpyAsync(host_flags, ctx->flags, FLAG_COUNT * sizeof(int), cudaMemcpyDeviceToHost, s));
    SPH_CUDA(ctx, cudaMemsetAsync(ctx->flags, 0, FLAG_COUNT * sizeof(int), s));
    SPH_CUDA(ctx, cudaStreamSynchronize(s));
    return SPH_OK;
}

extern "C" int sph_cell_order(sph_ctx* ctx, const sph_domain* dom, const double* pos, int64_t* order,
                              void* stream) {
    if (!ctx || !dom) return SPH_ERR_ARG;
    int st = sph_check_domain(dom);
    if (st) return st;
    if (dom->n > 0 && (!pos || !order)) return SPH_ERR_ARG;
    cudaStream_t s = as_stream(stream);
    // counting sort of the particles by the Morton key of their cell, stable by index
    CellGrid g = sph_make_grid(dom);
    MortonBits mb = morton_bits(g);
    if (mb.total > 29) return SPH_ERR_ARG;
    int64_t n = dom->n, nkeys = 1LL << mb.total;
    int32_t* key = (int32_t*)sph_scratch(ctx, S_CELL_ID, (size_t)n * 4, &st);
    int32_t* count = (int32_t*)sph_scratch(ctx, S_CELL_COUNT, (size_t)(nkeys + 1) * 4, &st);
    int32_t* start = (int32_t*)sph_scratch(ctx, S_CELL_START, (size_t)(nkeys + 1) * 4, &st);
    int32_t* fill = (int32_t*)sph_scratch(ctx, S_CELL_FILL, (size_t)(nkeys + 1) * 4, &st);
    int32_t* sorted = (int32_t*)sph_scratch(ctx, S_SORTED, (size_t)n * 4, &st);
    if (st) return st;
    SPH_CUDA(ctx, cudaMemsetAsync(count, 0, (size_t)(nkeys + 1) * 4, s));
    SPH_CUDA(ctx, cudaMemsetAsync(fill, 0, (size_t)(nkeys + 1) * 4, s));
    if (n > 0) k_morton_ids<<<grid_for(n, 256), 256, 0, s>>>(pos, n, g, mb, key, count, ctx->flags);
    st = sph_exclusive_scan_i32(ctx, count, start, nkeys, s);
    if (st) return st;
    if (n > 0) {
        k_scatter<<<grid_for(n, 256), 256, 0, s>>>(key, n, start, fill, sorted);
        k_sort_cells<<<grid_for(nkeys, 128), 128, 0, s>>>(start, nkeys, sorted);
        k_widen_order<<<grid_for(n, 256), 256, 0, s>>>(sorted, n, order);
    }
    SPH_LAUNCH_CHECK(ctx);
    int* hf = (int*)ctx->pinned;
    st = take_flags(ctx, s, hf);
    if (st) return st;
    if (hf[FLAG_BAD_INPUT]) return SPH_ERR_ARG;
    return SPH_OK;
}

extern "C" int sph_build_neighbors(sph_ctx* ctx, const sph_domain* dom, const double* pos, int64_t* row_ptr,
                                   int32_t* col, int64_t cap, int64_t* nnz_host, void* stream) {
    if (!ctx || !dom || !row_ptr || !nnz_host || cap < 0) return SPH_ERR_ARG;
    int st = sph_check_domain(dom);
    if (st) return st;
    int64_t n = dom->n;
    if (n > 0 && !pos) return SPH_ERR_ARG;
    if (cap > 0 && !col) return SPH_ERR_ARG;
    cudaStream_t s = as_stream(stream);
    CellList cl;
    st = sph_build_cells(ctx, dom, pos, s, &cl);
    if (st) return st;
    int32_t* row_len = (int32_t*)sph_scratch(ctx, S_ROW_LEN, (size_t)(n + 1) * 4, &st);
    if (st) return st;
    st = sph_count_neighbors(ctx, cl, pos, n, cl.grid.rc2, row_len, s);
    if (st) return st;
    st = sph_exclusive_scan_i64(ctx, row_len, row_ptr, n, s);
    if (st) return st;
    int64_t* hp = (int64_t*)ctx->pinned;
    SPH_CUDA(ctx, cudaMemcpyAsync(hp + 8, row_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    int* hf = (int*)ctx->pinned;
    st = take_flags(ctx, s, hf);
    if (st) return st;
    if (hf[FLAG_BAD_INPUT]) return SPH_ERR_ARG;
    int64_t nnz = hp[8];
    *nnz_host = nnz;
    if (nnz > cap) return SPH_ERR_CAPACITY;
    st = sph_fill_neighbors(ctx, cl, pos, n, cl.grid.rc2, row_ptr, col, cap, s);
    if (st) return st;
    return SPH_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free variant of sph_build_neighbors.
//
// Some callers cannot allocate device memory: a plug-in inside an application
// that owns the whole device-memory budget (it reserves its pool at start-up
// and treats any other cudaMalloc as a failure), or a latency-critical loop in
// which cudaMalloc / cudaFree would synchronise the device.  For them this
// entry point keeps all of its scratch (cell ids and counts, the sorted
// particle copy, row lengths, scan partials, flags) in one file-scope static
// device array of fixed size, SPH_STATIC_SCRATCH_BYTES, which every GPU that
// loads the library holds until the process exits.  The caller still provides
// pos, row_ptr and col.  All calls share the array: the parts that must start
// at zero are cleared on every call, and calls that overlap on the GPU (two
// streams, two host threads) race on it.
namespace {

constexpr int64_t kStaticMaxParticles = SPH_STATIC_MAX_PARTICLES;
constexpr int64_t kStaticMaxCells = SPH_STATIC_MAX_CELLS;
constexpr int64_t kStaticScanBlocks = (kStaticMaxParticles > kStaticMaxCells ? kStaticMaxParticles : kStaticMaxCells) / 2048 + 2;

constexpr size_t round256(size_t b) { return (b + 255) / 256 * 256; }
constexpr size_t kOffCellId = 0;
constexpr size_t kOffSorted = kOffCellId + round256(4 * kStaticMaxParticles);
constexpr size_t kOffP32 = kOffSorted + round256(4 * kStaticMaxParticles);
constexpr size_t kOffRowLen = kOffP32 + round256(16 * kStaticMaxParticles);
constexpr size_t kOffCount = kOffRowLen + round256(4 * (kStaticMaxParticles + 1));
constexpr size_t kOffStart = kOffCount + round256(4 * (kStaticMaxCells + 1));
constexpr size_t kOffFill = kOffStart + round256(4 * (kStaticMaxCells + 1));
constexpr size_t kOffScan64 = kOffFill + round256(4 * (kStaticMaxCells + 1));
constexpr size_t kOffScan32 = kOffScan64 + round256(8 * (kStaticScanBlocks + 1));
constexpr size_t kOffAbsmax = kOffScan32 + round256(4 * (kStaticScanBlocks + 1));
constexpr size_t kOffFlags = kOffAbsmax + 256;
constexpr size_t kStaticBytes = kOffFlags + 256;
static_assert(kStaticBytes <= SPH_STATIC_SCRATCH_BYTES, "static scratch layout exceeds the documented size");

}  // namespace

static __device__ __align__(256) unsigned char g_neighbor_static_scratch[SPH_STATIC_SCRATCH_BYTES];

namespace {

// Device address of the static array on the current device.  Looked up on every call
// (a host-side table lookup, no device work): an address cached across calls would go
// stale if the device's primary context were reset and the module loaded elsewhere.
// Host code cannot use the symbol itself as a device pointer.
int static_scratch_address(unsigned char** out) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_neighbor_static_scratch) != cudaSuccess || !p) return SPH_ERR_CUDA;
    *out = (unsigned char*)p;
    return SPH_OK;
}

}  // namespace

extern "C" int sph_build_neighbors_static(const sph_domain* dom, const double* pos, int64_t* row_ptr,
                                          int32_t* col, int64_t cap, int64_t* nnz_host, void* stream) {
    if (!dom || !row_ptr || !nnz_host || cap < 0) return SPH_ERR_ARG;
    int st = sph_check_domain(dom);
    if (st) return st;
    int64_t n = dom->n;
    if (n > 0 && !pos) return SPH_ERR_ARG;
    if (cap > 0 && !col) return SPH_ERR_ARG;
    CellGrid g = sph_make_grid(dom);
    if (n > kStaticMaxParticles || g.total > kStaticMaxCells) return SPH_ERR_LIMIT;
    unsigned char* base = nullptr;
    st = static_scratch_address(&base);
    if (st) return st;
    cudaStream_t s = as_stream(stream);
    int32_t* cid = (int32_t*)(base + kOffCellId);
    int32_t* sorted = (int32_t*)(base + kOffSorted);
    float4* p32 = (float4*)(base + kOffP32);
    int32_t* row_len = (int32_t*)(base + kOffRowLen);
    int32_t* count = (int32_t*)(base + kOffCount);
    int32_t* start = (int32_t*)(base + kOffStart);
    int32_t* fill = (int32_t*)(base + kOffFill);
    int64_t* scan64 = (int64_t*)(base + kOffScan64);
    int32_t* scan32 = (int32_t*)(base + kOffScan32);
    unsigned* absmax = (unsigned*)(base + kOffAbsmax);
    int* flags = (int*)(base + kOffFlags);
    // what must start at zero on every call
    if (cudaMemsetAsync(count, 0, (size_t)(g.total + 1) * 4, s) != cudaSuccess) return SPH_ERR_CUDA;
    if (cudaMemsetAsync(fill, 0, (size_t)(g.total + 1) * 4, s) != cudaSuccess) return SPH_ERR_CUDA;
    if (cudaMemsetAsync(absmax, 0, 256, s) != cudaSuccess) return SPH_ERR_CUDA;
    if (cudaMemsetAsync(flags, 0, 256, s) != cudaSuccess) return SPH_ERR_CUDA;
    if (n > 0) k_cell_ids<<<grid_for(n, 256), 256, 0, s>>>(pos, n, g, cid, count, flags, absmax);
    st = sph_exclusive_scan_i32_buf(count, start, g.total, scan32, s);
    if (st) return st;
    double lmax = periodic_lmax(g);
    if (n > 0) {
        k_scatter<<<grid_for(n, 256), 256, 0, s>>>(cid, n, start, fill, sorted);
        k_sort_cells<<<grid_for(g.total, 128), 128, 0, s>>>(start, g.total, sorted);
        k_pack_sorted<<<grid_for(n, 256), 256, 0, s>>>(pos, n, g.dim, sorted, p32);
        if (g.dim == 2)
            k_neighbors<2, false><<<grid_for(n, 128), 128, 0, s>>>(pos, n, g, g.rc2, lmax, absmax, start, p32, row_len,
                                                                  nullptr, nullptr, 0, flags);
        else
            k_neighbors<3, false><<<grid_for(n, 128), 128, 0, s>>>(pos, n, g, g.rc2, lmax, absmax, start, p32, row_len,
                                                                  nullptr, nullptr, 0, flags);
    }
    if (cudaPeekAtLastError() != cudaSuccess) return SPH_ERR_CUDA;
    st = sph_exclusive_scan_i64_buf(row_len, row_ptr, n, scan64, s);
    if (st) return st;
    int64_t nnz = 0;
    int bad = 0;
    if (cudaMemcpyAsync(&nnz, row_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess) return SPH_ERR_CUDA;
    if (cudaMemcpyAsync(&bad, flags + FLAG_BAD_INPUT, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return SPH_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return SPH_ERR_CUDA;
    if (bad) return SPH_ERR_ARG;
    *nnz_host = nnz;
    if (nnz > cap) return SPH_ERR_CAPACITY;
    if (n > 0) {
        if (g.dim == 2)
            k_neighbors<2, true><<<grid_for(n, 128), 128, 0, s>>>(pos, n, g, g.rc2, lmax, absmax, start, p32, nullptr,
                                                                 row_ptr, col, cap, flags);
        else
            k_neighbors<3, true><<<grid_for(n, 128), 128, 0, s>>>(pos, n, g, g.rc2, lmax, absmax, start, p32, nullptr,
                                                                 row_ptr, col, cap, flags);
    }
    return cudaPeekAtLastError() == cudaSuccess ? SPH_OK : SPH_ERR_CUDA;
}
