// Internal interface of the cell-list / neighbour-list builder (a1, a2).
#pragma once
#include "common.cuh"

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
