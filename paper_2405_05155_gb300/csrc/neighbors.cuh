// Internal interface of the cell-list / neighbour-list builder (a1, a2).
#pragma once
#include "common.cuh"

// ---- device helpers shared by the neighbour builder and the cell-sweep passes
namespace nb {

__device__ __forceinline__ int cell_coord(double x, int k, const CellGrid& g) {
    double c = floor((x - g.lo[k]) / g.size[k]);
    int n = g.n[k];
    if (!isfinite(c)) return 0;           // non-finite input (flagged by the caller)
    if ((g.periodic >> k) & 1u) {
        // positions are validated to lie in [lo, lo+len]: c in [0, n]
        long long ci = (long long)c;
        ci %= n;
        if (ci < 0) ci += n;
        return (int)ci;
    }
    if (!(c >= 0.0)) return 0;            // also maps NaN (flagged elsewhere) to 0
    if (c > (double)(n - 1)) return n - 1;
    return (int)c;
}

// Distinct neighbouring cell coordinates along one axis, ascending.
__device__ __forceinline__ int axis_cells(int c, int k, const CellGrid& g, int out[3]) {
    int n = g.n[k];
    int a, b = c, d;
    if ((g.periodic >> k) & 1u) {
        a = c - 1 < 0 ? n - 1 : c - 1;
        d = c + 1 >= n ? 0 : c + 1;
        // sort three values
        int v0 = a, v1 = b, v2 = d, t;
        if (v0 > v1) { t = v0; v0 = v1; v1 = t; }
        if (v1 > v2) { t = v1; v1 = v2; v2 = t; }
        if (v0 > v1) { t = v0; v0 = v1; v1 = t; }
        int m = 0;
        out[m++] = v0;
        if (v1 != v0) out[m++] = v1;
        if (v2 != v1) out[m++] = v2;
        return m;
    }
    a = c - 1 < 0 ? 0 : c - 1;
    d = c + 1 > n - 1 ? n - 1 : c + 1;
    int m = 0;
    out[m++] = a;
    if (b != a) out[m++] = b;
    if (d != b) out[m++] = d;
    return m;
}

struct Band { float lo, hi; };

__device__ __forceinline__ Band make_band(const unsigned* absmax, double lmax, double rc2, int dim) {
    const double u32 = 5.9604644775390625e-08;   // 2^-24
    double P = (double)__uint_as_float(*absmax);
    double eps = 4.0 * u32 * (P + lmax);
    double rc = sqrt(rc2);
    double delta = 4.0 * sqrt((double)dim) * rc * eps + 6.0 * eps * eps + 8.0 * u32 * rc2 + 1e-15 * rc2;
    Band b;
    b.lo = __double2float_rd(rc2 - delta);
    b.hi = __double2float_ru(rc2 + delta);
    return b;
}

// Float64 neighbour predicate of the definition: minimum image, unfused sum of squares.
__device__ __forceinline__ bool exact_within(const double* __restrict__ pos, int64_t n, int dim,
                                             const double xi[3], int j, const CellGrid& g, double rc2) {
    double d2 = 0.0;
    for (int k = 0; k < dim; ++k) {
        double dx = __dsub_rn(xi[k], pos[k * n + j]);
        if ((g.periodic >> k) & 1u) {
            if (dx > g.half[k]) dx = __dsub_rn(dx, g.len[k]);
            else if (dx < -g.half[k]) dx = __dadd_rn(dx, g.len[k]);
        }
        double sq = __dmul_rn(dx, dx);
        d2 = k == 0 ? sq : __dadd_rn(d2, sq);
    }
    return d2 <= rc2;
}

}  // namespace nb

struct CellList {
    CellGrid grid;
    int32_t* cell_id = nullptr;    // [n] linear cell id per particle
    int32_t* cell_start = nullptr; // [total+1] first sorted slot of each cell
    int32_t* sorted = nullptr;     // [n] particle index in (cell, index) order
    float4* p32 = nullptr;         // [n] float32 positions in sorted order, .w = index bits
    float* band = nullptr;         // [2] float32 screening thresholds (lo, hi)
};

// Bin the particles into cells (counting sort, stable by index) and prepare the
// float32 screening copy.  Flags FLAG_BAD_INPUT in ctx->flags on non-finite or
// out-of-box (periodic axis) positions; does not synchronise.
int sph_build_cells(sph_ctx* ctx, const sph_domain* dom, const double* pos, cudaStream_t s,
                    CellList* cl);

// Per-particle neighbour counts (row_len[n]) for cut-off^2 = rc2 (<= grid.rc2).
int sph_count_neighbors(sph_ctx* ctx, const CellList& cl, const double* pos, int64_t n,
                        double rc2, int32_t* row_len, cudaStream_t s);

// Fill CSR rows (ascending j) given row_ptr; requires row_ptr[n] <= cap, checked
// on the device: if exceeded, FLAG_CAPACITY is set and nothing is written.
int sph_fill_neighbors(sph_ctx* ctx, const CellList& cl, const double* pos, int64_t n,
                       double rc2, const int64_t* row_ptr, int32_t* col, int64_t cap,
                       cudaStream_t s);
