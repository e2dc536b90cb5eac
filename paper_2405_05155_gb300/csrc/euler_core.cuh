// Per-pair physics and packed-record helpers of the Eulerian WCSPH passes, shared by the
// single-case kernels (eulerian.cu) and the batched persistent kernel (batched.cu).
#pragma once
#include "async.cuh"
#include "common.cuh"
#include "tiles.cuh"

namespace euler {

enum { WANT_MOM = 1, WANT_MASS = 2, WANT_BOTH = 3 };
enum { OUT_RATES = 0, OUT_MOM = 1, OUT_MASS = 2, OUT_FUSED = 3 };

template <typename R>
struct EulerK {
    R coef;        // Wendland gs coefficient -5 alpha_d h^-(d+2)
    R inv_h;
    R rho0, c0, inv_c0, c0sq, eta, mu2, eps_h2, dt;
    R half[3];
    R Lh[3], Ll[3];   // box length split hi + lo (float32 path; Ll = 0 in float64)
    R S[3], Sl[3];    // float32 path: cell size (hi + lo) of the cell-relative positions
    int ncell[3];
    uint32_t periodic;
};

template <int DIM> struct NSym { static constexpr int v = DIM == 2 ? 3 : 6; };

template <int DIM, typename R>
__device__ __forceinline__ void sym_matvec(const R* Bs, const R* x, R* y) {
    if (DIM == 2) {
        y[0] = Bs[0] * x[0] + Bs[1] * x[1];
        y[1] = Bs[1] * x[0] + Bs[2] * x[1];
    } else {
        y[0] = Bs[0] * x[0] + Bs[1] * x[1] + Bs[2] * x[2];
        y[1] = Bs[1] * x[0] + Bs[3] * x[1] + Bs[4] * x[2];
        y[2] = Bs[2] * x[0] + Bs[4] * x[1] + Bs[5] * x[2];
    }
}

template <typename R> __device__ __forceinline__ R rsqrt_(R x);
template <> __device__ __forceinline__ double rsqrt_<double>(double x) { return 1.0 / sqrt(x); }
template <> __device__ __forceinline__ float rsqrt_<float>(float x) { return rsqrtf(x); }

// One directed pair (i, j): contributions to d rho_i/dt and d(rho v)_i/dt.
template <int DIM, int MODE, typename R>
__device__ __forceinline__ void euler_pair(const R* r, R d2, const R* Bi, const R* Bj, const R* vi, const R* vj,
                                           R drho_i, R drho_j, R Vj, const EulerK<R>& K, R& mass, R* mom) {
    constexpr int NS = NSym<DIM>::v;
    R q = sqrt(d2) * K.inv_h;
    R gs = wendland_gs<R>(q, K.coef);
    R gw[DIM], Bb[NS], g[DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a) gw[a] = gs * r[a];
#pragma unroll
    for (int s = 0; s < NS; ++s) Bb[s] = R(0.5) * (Bi[s] + Bj[s]);
    sym_matvec<DIM, R>(Bb, gw, g);                    // Eq. 27
    R rinv = rsqrt_<R>(d2);
    R nrm[DIM];
    R ul = R(0), ur = R(0);
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        nrm[a] = -r[a] * rinv;                        // from i towards j
        ul += vi[a] * nrm[a];
        ur += vj[a] * nrm[a];
    }
    R pi = K.c0sq * drho_i, pj = K.c0sq * drho_j;    // p = c0^2 (rho - rho0)
    R rho_bar = K.rho0 + R(0.5) * (drho_i + drho_j);
    R du = ul - ur;
    R beta = fmin(K.eta * fmax(du * K.inv_c0, R(0)), R(1));   // Eq. 26 limiter
    R ubar = R(0.5) * (ul + ur);
    R ustar = ubar + R(0.5) * beta * beta * (pi - pj) / (rho_bar * K.c0);   // Eq. 25
    R pstar = R(0.5) * (pi + pj) + R(0.5) * beta * rho_bar * K.c0 * du;
    R vs[DIM];
    R vg = R(0);
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        vs[a] = R(0.5) * (vi[a] + vj[a]) + (ustar - ubar) * nrm[a];
        vg += vs[a] * g[a];
    }
    if (MODE & WANT_MASS) mass = R(-2) * Vj * rho_bar * vg;
    if (MODE & WANT_MOM) {
        R visc = K.mu2 * Vj * (gs * d2) / (d2 + K.eps_h2);
#pragma unroll
        for (int a = 0; a < DIM; ++a)
            mom[a] = R(-2) * Vj * (rho_bar * vs[a] * vg + pstar * g[a]) + visc * (vi[a] - vj[a]);
    }
}

// ---------------------------------------------------------------- float32 path
// Records of 16 floats (two 32-byte lines, two 256-bit loads per neighbour):
//   3D: (ox, oy, oz, cell, V, B00, B01, B02) (B11, B12, B22, 0, vx, vy, vz, drho)
//   2D: (ox, oy, cell, V, B00, B01, B11, 0) (0, 0, 0, 0, vx, vy, 0, drho)
// positions cell-relative (see rel_pair); the dynamic part (v, drho) is the
// float4 at offset 12, the only part a pass writes (into the other buffer).
constexpr int kRecWords = 16;

template <int DIM>
__device__ __forceinline__ void unpack_rec(const F8& a, const F8& b, float* o, uint32_t& cell, float& V, float* Bs,
                                           float* v, float& drho) {
    if constexpr (DIM == 3) {
        o[0] = a.v[0]; o[1] = a.v[1]; o[2] = a.v[2];
        cell = __float_as_uint(a.v[3]);
        V = a.v[4];
        Bs[0] = a.v[5]; Bs[1] = a.v[6]; Bs[2] = a.v[7];
        Bs[3] = b.v[0]; Bs[4] = b.v[1]; Bs[5] = b.v[2];
        v[0] = b.v[4]; v[1] = b.v[5]; v[2] = b.v[6];
    } else {
        o[0] = a.v[0]; o[1] = a.v[1];
        cell = __float_as_uint(a.v[2]);
        V = a.v[3];
        Bs[0] = a.v[4]; Bs[1] = a.v[5]; Bs[2] = a.v[6];
        v[0] = b.v[4]; v[1] = b.v[5];
    }
    drho = b.v[7];
}

template <int DIM>
__device__ __forceinline__ void store_dyn(float* rec, int64_t i, const float* v, float drho) {
    float vz = 0.0f;
    if constexpr (DIM == 3) vz = v[2];
    *reinterpret_cast<float4*>(rec + kRecWords * i + 12) = make_float4(v[0], v[1], vz, drho);
}

// Pair loop of one particle over its CSR row (LANES lanes per row, compensated
// sums, next neighbour's record loaded before the current pair is evaluated).
template <int DIM, int MODE, int LANES, bool PER>
__device__ __forceinline__ void euler_row32(const float* __restrict__ R, const int32_t* __restrict__ col,
                                            int64_t b, int64_t e, int lane, const float* oi, uint32_t bi,
                                            const float* Bi, const float* vi, float dri, const EulerK<float>& K,
                                            float& rm, float* rp) {
    constexpr int NS = NSym<DIM>::v;
    Kahan<float> am;
    Kahan<float> ap[DIM];
    am.init();
#pragma unroll
    for (int a = 0; a < DIM; ++a) ap[a].init();
    int64_t p = b + lane;
    int j = p < e ? __ldg(&col[p]) : -1;
    F8 ja, jb;
    if (j >= 0) { ja = ldg8(R + kRecWords * (int64_t)j); jb = ldg8(R + kRecWords * (int64_t)j + 8); }
    while (j >= 0) {
        int64_t pn = p + LANES;
        int jn = pn < e ? __ldg(&col[pn]) : -1;
        F8 na = ja, nb2 = jb;
        if (jn >= 0) { na = ldg8(R + kRecWords * (int64_t)jn); nb2 = ldg8(R + kRecWords * (int64_t)jn + 8); }
        float oj[DIM], Vj, Bj[NS], vj[DIM], drj;
        uint32_t bj;
        unpack_rec<DIM>(ja, jb, oj, bj, Vj, Bj, vj, drj);
        float r[DIM], d2;
        rel_pair<DIM, PER>(oi, bi, oj, bj, K.ncell, K.S, K.Sl, K.periodic, r, d2);
        float m = 0.0f, mo[DIM];
        euler_pair<DIM, MODE, float>(r, d2, Bi, Bj, vi, vj, dri, drj, Vj, K, m, mo);
        if (MODE & WANT_MASS) am.add(m);
        if (MODE & WANT_MOM) {
#pragma unroll
            for (int a = 0; a < DIM; ++a) ap[a].add(mo[a]);
        }
        p = pn;
        j = jn;
        ja = na;
        jb = nb2;
    }
    rm = group_sum<LANES>(am.value());
#pragma unroll
    for (int a = 0; a < DIM; ++a) rp[a] = group_sum<LANES>(ap[a].value());
}

// Epilogue of the two-pass step / fused step: new (v, drho) of particle i.
template <int DIM, int OUT>
__device__ __forceinline__ void euler_update32(const float* vi, float dri, float rm, const float* rp,
                                               const EulerK<float>& K, float* vn, float& drn) {
    float rho_i = K.rho0 + dri;
    if (OUT == OUT_MOM) {
#pragma unroll
        for (int a = 0; a < DIM; ++a) vn[a] = vi[a] + K.dt * rp[a] / rho_i;
        drn = dri;
    } else if (OUT == OUT_MASS) {
        float ddr = K.dt * rm;
        drn = dri + ddr;
        float ratio = 1.0f - ddr / (K.rho0 + drn);     // rho^n / rho^{n+1}
#pragma unroll
        for (int a = 0; a < DIM; ++a) vn[a] = vi[a] * ratio;
    } else {
        float ddr = K.dt * rm;
        drn = dri + ddr;
        float rho1 = K.rho0 + drn;
        float ratio = 1.0f - ddr / rho1;
#pragma unroll
        for (int a = 0; a < DIM; ++a) vn[a] = vi[a] * ratio + K.dt * rp[a] / rho1;
    }
}

// ------------------------------------------------- planned passes (tile plans)
// Entry ring of a planned pass (see euler_tile_g), after the stage: either kEntryChunks
// chunks of one step of the tile's sliced entries (kTileRows entries of 32 bytes, 4 KB),
// then a full and an empty mbarrier per chunk; or, per thread, kEntryChunks 32-byte slots
// (the same 16 KB).
constexpr int kEntryChunks = 4;
constexpr uint32_t kChunkBytes = kTileRows * 32;
constexpr size_t kEntryRingBytes = (size_t)kEntryChunks * kChunkBytes + 2 * kEntryChunks * 8;
// The chunk ring's launches of at least this many waves of blocks (SPH_RING_AUTO).
constexpr int kChunkRingWaves = 2;
// Polls of a bounded mbarrier wait before a block gives up (FLAG_TIMEOUT).
constexpr uint32_t kEuWaitPolls = 1u << 22;

struct GeoArgsE {
    const int32_t* tile_m;
    const int64_t* tile_so;
    const int32_t* uidx;
    const float* geo;   // 8 floats per entry
    int mcap;
    uint32_t test_polls;   // > 0 (sph_set_wait_test): no copy is issued, the waits run out after this many polls
    int chunk_ring;        // 1: the TMA chunk ring, 0: the per-thread cp.async ring (SPH_RING_*; the
                           // launch picks the kernel instantiation by it)
};

// One pair of a planned pass from its entry and the neighbour's (v_j, drho_j).
// Every operation is written out (fused multiply-adds explicit, products and sums
// rounded on their own), so the result does not depend on where it is inlined.
template <int DIM, int MODE>
__device__ __forceinline__ void euler_pair_geo(const F8& e, float4 dj, const float* vi, float dri,
                                               const EulerK<float>& K, Kahan<float>& am, Kahan<float>* ap) {
    const float G[3] = {e.v[0], e.v[1], e.v[2]};
    const float nrm[3] = {e.v[4], e.v[5], e.v[6]};
    const float vj[3] = {dj.x, dj.y, dj.z};
    const float drj = dj.w;
    float ul = __fmul_rn(vi[0], nrm[0]), ur = __fmul_rn(vj[0], nrm[0]);
#pragma unroll
    for (int a = 1; a < DIM; ++a) {
        ul = fmaf(vi[a], nrm[a], ul);
        ur = fmaf(vj[a], nrm[a], ur);
    }
    const float pi = __fmul_rn(K.c0sq, dri), pj = __fmul_rn(K.c0sq, drj);
    const float rho_bar = fmaf(0.5f, __fadd_rn(dri, drj), K.rho0);
    const float du = __fsub_rn(ul, ur);
    const float beta = fminf(__fmul_rn(K.eta, fmaxf(__fmul_rn(du, K.inv_c0), 0.0f)), 1.0f);
    const float ubar = __fmul_rn(0.5f, __fadd_rn(ul, ur));
    const float rc = __fmul_rn(rho_bar, K.c0);
    const float hb = __fmul_rn(0.5f, beta);
    const float ustar = fmaf(__fmul_rn(hb, beta), __fdiv_rn(__fsub_rn(pi, pj), rc), ubar);   // Eq. 25
    const float pstar = fmaf(__fmul_rn(hb, rc), du, __fmul_rn(0.5f, __fadd_rn(pi, pj)));
    const float dus = __fsub_rn(ustar, ubar);
    float vs[DIM];
    float vG = 0.0f;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        vs[a] = fmaf(dus, nrm[a], __fmul_rn(0.5f, __fadd_rn(vi[a], vj[a])));
        vG = a == 0 ? __fmul_rn(vs[0], G[0]) : fmaf(vs[a], G[a], vG);
    }
    if (MODE & WANT_MASS) am.add(__fmul_rn(rho_bar, vG));
    if (MODE & WANT_MOM) {
#pragma unroll
        for (int a = 0; a < DIM; ++a)
            ap[a].add(fmaf(e.v[3], __fsub_rn(vi[a], vj[a]), fmaf(pstar, G[a], __fmul_rn(__fmul_rn(rho_bar, vs[a]), vG))));
    }
}

// One tile of kTileRows rows of a planned pass (see sph_eulerian_plan): rows
// row_base + t*kTileRows + [0, kTileRows) of the record arrays, which belong to a
// case of n rows starting at row_base; row_ptr is indexed by global row and rp0 =
// row_ptr[row_base], so that row_ptr[row] - rp0 indexes the case's plan arrays,
// whose neighbour indices are case-local.  The tile's neighbour (v_j, drho_j) are
// staged in sp (A.mcap float4); a tile with more distinct neighbours reads them
// from Rin.  The block must be kTileRows threads.
template <int DIM, int MODE, int OUT, bool CHUNK>
__device__ __forceinline__ void euler_tile_g(const float* __restrict__ Rin, float* __restrict__ Rout,
                                             const int64_t* __restrict__ row_ptr, int64_t row_base, int64_t rp0,
                                             int64_t n, int64_t tile, const EulerK<float>& K, const GeoArgsE& A,
                                             float4* sp, double* __restrict__ rate_mass,
                                             double* __restrict__ rate_mom, int* __restrict__ flags) {
    const int64_t i0 = tile * kTileRows;
    const int64_t i = i0 + threadIdx.x;
    const bool active = i < n;
    const int64_t ii = row_base + (active ? i : i0);
    const int64_t P0 = row_ptr[row_base + i0] - rp0;
    const int len = active ? (int)(row_ptr[ii + 1] - row_ptr[ii]) : 0;
    const int m = A.tile_m[tile];
    const int64_t so = A.tile_so[tile];
    const int width = CHUNK ? (int)((A.tile_so[tile + 1] - so) / kTileRows) : 0;
    // Chunk ring (CHUNK): the tile's entries arrive by TMA bulk copies, step k of the
    // sliced layout (entry k of all kTileRows rows) being one contiguous 4 KB chunk.  Thread 0
    // keeps kEntryChunks chunks in flight in a ring after the stage, each completing on its
    // full mbarrier, and refills a slot once all the block's threads have read it (its empty
    // mbarrier, kTileRows arrivals).  The first chunks are requested before the neighbours
    // are staged.  Every wait is bounded; a block whose wait runs out sets FLAG_TIMEOUT, waits
    // (bounded) for the copies it issued and leaves.  A.test_polls > 0: nothing is copied
    // and the waits run out.  Thread ring (otherwise): each thread streams its own entries
    // through kEntryChunks 32-byte slots, kEntryChunks - 1 entries ahead with cp.async, and
    // refills a slot once it has evaluated the pair that read it: no thread waits for
    // another, the shorter chain when one wave of blocks is the whole pass.
    float4* ring = sp + A.mcap;
    uint64_t* full = reinterpret_cast<uint64_t*>(ring + (size_t)kEntryChunks * 2 * kTileRows);
    uint64_t* empty = full + kEntryChunks;
    const float* g0 = A.geo + 8 * so;
    const bool test_wait = A.test_polls > 0;
    const uint32_t polls = test_wait ? A.test_polls : kEuWaitPolls;
    int issued = 0;                                      // chunks thread 0 has requested
    if (CHUNK && threadIdx.x == 0) {
        for (int c = 0; c < kEntryChunks; ++c) {
            mbar_init(&full[c], 1);
            mbar_init(&empty[c], kTileRows);
        }
        mbar_fence_init();
        if (!test_wait) {
            for (; issued < kEntryChunks && issued < width; ++issued) {
                mbar_arrive_expect_tx(&full[issued], kChunkBytes);
                tma_load_1d(ring + (size_t)issued * 2 * kTileRows, g0 + (int64_t)8 * issued * kTileRows, kChunkBytes,
                            &full[issued]);
            }
        }
    }
    const float4 own = __ldg(reinterpret_cast<const float4*>(Rin + kRecWords * ii) + 3);
    const bool staged = m <= A.mcap;
    if (staged) {
        for (int s = threadIdx.x; s < m; s += blockDim.x) {
            // a plan out of date with the lists reads wrong but in-bounds records
            int64_t j = row_base + min(max((int64_t)A.uidx[P0 + s], (int64_t)0), n - 1);
            sp[s] = __ldg(reinterpret_cast<const float4*>(Rin + kRecWords * j) + 3);
        }
    }
    __syncthreads();
    const float vi[3] = {own.x, own.y, own.z};
    const float dri = own.w;
    Kahan<float> am;
    Kahan<float> ap[DIM];
    am.init();
#pragma unroll
    for (int a = 0; a < DIM; ++a) ap[a].init();
    const int smax = max(m - 1, 0);
    auto pair = [&](const float4* d) {
        const float4 lo = d[0], hi = d[1];
        F8 e;
        e.v[0] = lo.x; e.v[1] = lo.y; e.v[2] = lo.z; e.v[3] = lo.w;
        e.v[4] = hi.x; e.v[5] = hi.y; e.v[6] = hi.z; e.v[7] = hi.w;
        const int s = min(max(__float_as_int(e.v[7]), 0), smax);
        if (staged) {
            euler_pair_geo<DIM, MODE>(e, sp[s], vi, dri, K, am, ap);
        } else {
            const int64_t j = row_base + min(max((int64_t)A.uidx[P0 + s], (int64_t)0), n - 1);
            euler_pair_geo<DIM, MODE>(e, __ldg(reinterpret_cast<const float4*>(Rin + kRecWords * j) + 3), vi, dri,
                                      K, am, ap);
        }
    };
    bool late = false;
    if constexpr (!CHUNK) {
        float4* own_ring = ring + 2 * threadIdx.x;
        const float* g = g0 + 8 * (int64_t)threadIdx.x;
        auto issue = [&](int k) {
            float4* d = own_ring + (k % kEntryChunks) * (2 * kTileRows);
            const float* src = g + (int64_t)8 * k * kTileRows;
            cp_async16(d, src);
            cp_async16(d + 1, src + 4);
        };
#pragma unroll
        for (int k = 0; k < kEntryChunks - 1; ++k) {
            if (k < len) issue(k);
            cp_async_commit();
        }
        for (int k = 0; k < len; ++k) {
            if (k + kEntryChunks - 1 < len) issue(k + kEntryChunks - 1);
            cp_async_commit();
            cp_async_wait_group<kEntryChunks - 1>();
            pair(own_ring + (k % kEntryChunks) * (2 * kTileRows));
        }
    }
    for (int k = 0; k < width; ++k) {
        const int slot = k % kEntryChunks;
        const uint32_t par = (uint32_t)(k / kEntryChunks) & 1u;
        if (!mbar_wait_bounded(&full[slot], par, polls)) {
            late = true;
            break;
        }
        if (k < len) pair(ring + (size_t)slot * 2 * kTileRows + 2 * threadIdx.x);
        mbar_arrive(&empty[slot]);
        if (threadIdx.x == 0 && k + kEntryChunks < width) {
            if (!mbar_wait_bounded(&empty[slot], par, polls)) {
                late = true;
                break;
            }
            mbar_arrive_expect_tx(&full[slot], kChunkBytes);
            tma_load_1d(ring + (size_t)slot * 2 * kTileRows, g0 + (int64_t)8 * (k + kEntryChunks) * kTileRows,
                        kChunkBytes, &full[slot]);
            ++issued;
        }
    }
    if (CHUNK && __syncthreads_or(late)) {             // block-uniform from here
        if (threadIdx.x == 0) {
            atomicExch(&flags[FLAG_TIMEOUT], 1);
            // the copies issued and perhaps in flight: the last one of each slot
            for (int c = max(issued - kEntryChunks, 0); c < issued; ++c)
                mbar_wait_bounded(&full[c % kEntryChunks], (uint32_t)(c / kEntryChunks) & 1u, kEuWaitPolls);
        }
        return;
    }
    if (!active) return;
    float rm = am.value(), rp[DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a) rp[a] = ap[a].value();
    if (OUT == OUT_RATES) {
        if (MODE & WANT_MASS) rate_mass[i] = (double)rm;
        if (MODE & WANT_MOM)
            for (int a = 0; a < DIM; ++a) rate_mom[a * n + i] = (double)rp[a];
        return;
    }
    float vn[DIM], drn;
    euler_update32<DIM, OUT>(vi, dri, rm, rp, K, vn, drn);
    store_dyn<DIM>(Rout, ii, vn, drn);
}

}  // namespace euler
