// a5/a6: Riemann-based Eulerian weakly-compressible SPH (Sec. 3.1; Eqs. 18, 25-27).
//
// Two pair-pass kernels share one per-pair device function:
//  * k_euler64: float64 structure-of-arrays state, one thread per particle;
//  * k_euler32: float32 records of 16 floats (two 32-byte lines: cell-relative
//    position, volume, B, velocity, density; two 256-bit loads per neighbour),
//    LANES consecutive lanes per particle striding over the CSR row, compensated
//    (Kahan) sums, group shuffle reduce.
// A pass computes the mass and/or momentum rates of a particle and applies the
// pointwise part of the update in its epilogue (EOS p = c0^2 drho, velocity
// from momentum), so a step is one (fused) or two (momentum, continuity) launches.
#include "common.cuh"
#include "euler_core.cuh"
#include "tiles.cuh"

namespace {

using namespace euler;

// ---------------------------------------------------------------- float64 path
template <int DIM, int MODE, int OUT>
__global__ void k_euler64(const double* __restrict__ pos, const double* __restrict__ vol,
                          const double* __restrict__ B, const int64_t* __restrict__ row_ptr,
                          const int32_t* __restrict__ col, int64_t n, EulerK<double> K,
                          const double* __restrict__ drho, const double* __restrict__ v,
                          double* __restrict__ drho_out, double* __restrict__ v_out,
                          double* __restrict__ rate_mass, double* __restrict__ rate_mom) {
    constexpr int NS = NSym<DIM>::v;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double xi[DIM], vi[DIM], Bi[NS];
#pragma unroll
    for (int a = 0; a < DIM; ++a) { xi[a] = pos[a * n + i]; vi[a] = v[a * n + i]; }
#pragma unroll
    for (int s = 0; s < NS; ++s) Bi[s] = B[s * n + i];
    double dri = drho[i];
    double am = 0.0, ap[DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a) ap[a] = 0.0;
    for (int64_t p = row_ptr[i], e = row_ptr[i + 1]; p < e; ++p) {
        int j = col[p];
        double r[DIM], vj[DIM], Bj[NS], d2 = 0.0;
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            double dx = xi[a] - pos[a * n + j];
            if ((K.periodic >> a) & 1u) {
                if (dx > K.half[a]) dx -= K.Lh[a];
                else if (dx < -K.half[a]) dx += K.Lh[a];
            }
            r[a] = dx;
            d2 += dx * dx;
            vj[a] = v[a * n + j];
        }
#pragma unroll
        for (int s = 0; s < NS; ++s) Bj[s] = B[s * n + j];
        double m = 0.0, mo[DIM];
        euler_pair<DIM, MODE, double>(r, d2, Bi, Bj, vi, vj, dri, drho[j], vol[j], K, m, mo);
        if (MODE & WANT_MASS) am += m;
        if (MODE & WANT_MOM) {
#pragma unroll
            for (int a = 0; a < DIM; ++a) ap[a] += mo[a];
        }
    }
    double rho_i = K.rho0 + dri;
    if (OUT == OUT_RATES) {
        if (MODE & WANT_MASS) rate_mass[i] = am;
        if (MODE & WANT_MOM)
            for (int a = 0; a < DIM; ++a) rate_mom[a * n + i] = ap[a];
    } else if (OUT == OUT_MOM) {          // v' = (rho^n v^n + dt R_mom) / rho^n ; keep drho^n
        drho_out[i] = dri;
        for (int a = 0; a < DIM; ++a) v_out[a * n + i] = (rho_i * vi[a] + K.dt * ap[a]) / rho_i;
    } else if (OUT == OUT_MASS) {         // rho^{n+1}; v^{n+1} = v' rho^n / rho^{n+1}
        double dr1 = dri + K.dt * am;
        double rho1 = K.rho0 + dr1;
        drho_out[i] = dr1;
        for (int a = 0; a < DIM; ++a) v_out[a * n + i] = (rho_i * vi[a]) / rho1;
    } else {                              // fused forward Euler
        double dr1 = dri + K.dt * am;
        double rho1 = K.rho0 + dr1;
        drho_out[i] = dr1;
        for (int a = 0; a < DIM; ++a) v_out[a * n + i] = (rho_i * vi[a] + K.dt * ap[a]) / rho1;
    }
}

// ---------------------------------------------------------------- float32 path
template <int DIM, int MODE, int OUT, int LANES, bool PER>
__global__ void __launch_bounds__(256) k_euler32(const float* __restrict__ Rin, float* __restrict__ Rout,
                                                 const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                                 int64_t n, EulerK<float> K, double* __restrict__ rate_mass,
                                                 double* __restrict__ rate_mom) {
    constexpr int NS = NSym<DIM>::v;
    int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t i = gt / LANES;
    int lane = (int)(gt % LANES);
    bool active = i < n;
    int64_t ii = active ? i : 0;
    F8 ma = ldg8(Rin + kRecWords * ii), mb = ldg8(Rin + kRecWords * ii + 8);
    float oi[DIM], Vi, Bi[NS], vi[DIM], dri;
    uint32_t bi;
    unpack_rec<DIM>(ma, mb, oi, bi, Vi, Bi, vi, dri);
    int64_t b = active ? row_ptr[ii] : 0, e = active ? row_ptr[ii + 1] : 0;
    float rm, rp[DIM];
    euler_row32<DIM, MODE, LANES, PER>(Rin, col, b, e, lane, oi, bi, Bi, vi, dri, K, rm, rp);
    if (!active || lane != 0) return;
    if (OUT == OUT_RATES) {
        if (MODE & WANT_MASS) rate_mass[i] = (double)rm;
        if (MODE & WANT_MOM)
            for (int a = 0; a < DIM; ++a) rate_mom[a * n + i] = (double)rp[a];
        return;
    }
    float vn[DIM], drn;
    euler_update32<DIM, OUT>(vi, dri, rm, rp, K, vn, drn);
    store_dyn<DIM>(Rout, i, vn, drn);
}

// ---------------------------------------------------- float32 passes on a tile plan
// Eulerian particles do not move, so every pair's geometry is fixed: k_eu_geo
// computes it once in float64 (tiles.cuh layout, 32-byte entries, rows ordered by
// offset) as
//   (G, Vis, n, slot),  G = -2 V_j (B_i + B_j)/2 grad W_ij   (Eqs. 18, 27),
//   Vis = 2 mu V_j (r_ij . grad W_ij) / (r^2 + 0.01 h^2),  n = -r_ij / r,
// each rounded once to float32.  A planned pass then needs only the neighbour's
// (v_j, drho_j), which a block stages per tile in shared memory, and evaluates the
// acoustic Riemann flux (Eqs. 25-26) pair by pair.
template <int DIM>
__global__ void __launch_bounds__(kTileRows) k_eu_geo(const double* __restrict__ pos, const double* __restrict__ vol,
                                                      const double* __restrict__ B,
                                                      const int64_t* __restrict__ row_ptr,
                                                      const int32_t* __restrict__ col,
                                                      const uint16_t* __restrict__ lcol,
                                                      const int32_t* __restrict__ tile_e,
                                                      const int64_t* __restrict__ tile_so, int64_t n,
                                                      EulerK<double> K, float* __restrict__ geo) {
    constexpr int NS = NSym<DIM>::v;
    const int64_t tile = blockIdx.x;
    const int64_t i = tile * kTileRows + threadIdx.x;
    const bool active = i < n;
    const int64_t b = active ? row_ptr[i] : 0;
    const int len = active ? (int)(row_ptr[i + 1] - b) : 0;
    const int width = tile_e[tile] / kTileRows;
    float* out = geo + 8 * (tile_so[tile] + threadIdx.x);
    double xi[DIM], Bi[NS];
#pragma unroll
    for (int a = 0; a < DIM; ++a) xi[a] = active ? pos[a * n + i] : 0.0;
#pragma unroll
    for (int s = 0; s < NS; ++s) Bi[s] = active ? B[s * n + i] : 0.0;
    auto rij = [&](int j, double* r, double& d2) {
        d2 = 0.0;
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            double dx = xi[a] - pos[a * n + j];
            if ((K.periodic >> a) & 1u) {
                if (dx > K.half[a]) dx -= K.Lh[a];
                else if (dx < -K.half[a]) dx += K.Lh[a];
            }
            r[a] = dx;
            d2 += dx * dx;
        }
    };
    uint32_t order[kSortCap];
    const bool sorted = offset_order<DIM>(
        len, 2.0 * K.inv_h,
        [&](int k, double* rr) {
            double r[DIM], d2;
            rij(col[b + k], r, d2);
            for (int a = 0; a < DIM; ++a) rr[a] = r[a];
        },
        order);
    for (int k = 0; k < width; ++k) {
        float e[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        if (k < len) {
            int64_t p = b + (sorted ? (int)(order[k] & 0xFFFFFu) : k);
            int j = col[p];
            double r[DIM], d2, Bb[NS], gw[DIM], g[DIM];
            rij(j, r, d2);
            double gs = wendland_gs<double>(sqrt(d2) * K.inv_h, K.coef);
            double Vj = vol[j];
#pragma unroll
            for (int a = 0; a < DIM; ++a) gw[a] = gs * r[a];
#pragma unroll
            for (int s = 0; s < NS; ++s) Bb[s] = 0.5 * (Bi[s] + B[s * n + j]);
            sym_matvec<DIM, double>(Bb, gw, g);
            double rinv = 1.0 / sqrt(d2);
            for (int a = 0; a < DIM; ++a) {
                e[a] = (float)(-2.0 * Vj * g[a]);
                e[4 + a] = (float)(-r[a] * rinv);
            }
            e[3] = (float)(K.mu2 * Vj * (gs * d2) / (d2 + K.eps_h2));
            e[7] = __int_as_float((int)lcol[p]);
        }
        float4* o = reinterpret_cast<float4*>(out + (int64_t)8 * k * kTileRows);
        o[0] = make_float4(e[0], e[1], e[2], e[3]);
        o[1] = make_float4(e[4], e[5], e[6], e[7]);
    }
}

template <int DIM, int MODE, int OUT, bool CHUNK>
__global__ void __launch_bounds__(kTileRows, 6) k_euler32g(const float* __restrict__ Rin, float* __restrict__ Rout,
                                                           const int64_t* __restrict__ row_ptr, int64_t n,
                                                           EulerK<float> K, GeoArgsE A,
                                                           double* __restrict__ rate_mass,
                                                           double* __restrict__ rate_mom, int* __restrict__ flags) {
    extern __shared__ __align__(16) unsigned char eu_smem[];
    // launched as a programmatic dependent of the previous pass: its blocks are scheduled
    // while that pass finishes and read nothing before it has completed
    grid_dependency_wait();
    grid_launch_dependents();
    // the momentum pass of the two-pass step walks the tiles in reverse, the continuity
    // pass forwards: each starts on the pair entries the previous one read last (in L2)
    const int64_t tile = MODE == WANT_MOM ? gridDim.x - 1 - blockIdx.x : blockIdx.x;
    euler_tile_g<DIM, MODE, OUT, CHUNK>(Rin, Rout, row_ptr, 0, 0, n, tile, K, A,
                                        reinterpret_cast<float4*>(eu_smem), rate_mass, rate_mom, flags);
}

// ---------------------------------------------------------------- pack / unpack
template <int DIM>
__global__ void k_pack_rec(const double* __restrict__ pos, const double* __restrict__ vol,
                           const double* __restrict__ B, const double* __restrict__ drho,
                           const double* __restrict__ v, int64_t n, RelGrid g, float* __restrict__ R0,
                           float* __restrict__ R1) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double x[3] = {0, 0, 0};
    for (int a = 0; a < DIM; ++a) x[a] = pos[a * n + i];
    float o[3] = {0, 0, 0};
    uint32_t bits = rel_encode<DIM>(x, g, o);
    float rec[kRecWords];
    for (int k = 0; k < kRecWords; ++k) rec[k] = 0.0f;
    if (DIM == 3) {
        rec[0] = o[0]; rec[1] = o[1]; rec[2] = o[2]; rec[3] = __uint_as_float(bits);
        rec[4] = (float)vol[i];
        for (int s = 0; s < 6; ++s) rec[5 + s] = (float)B[s * n + i];
    } else {
        rec[0] = o[0]; rec[1] = o[1]; rec[2] = __uint_as_float(bits); rec[3] = (float)vol[i];
        for (int s = 0; s < 3; ++s) rec[4 + s] = (float)B[s * n + i];
    }
    for (int a = 0; a < DIM; ++a) rec[12 + a] = (float)v[a * n + i];
    rec[15] = (float)drho[i];
    float4* d0 = reinterpret_cast<float4*>(R0 + kRecWords * i);
    float4* d1 = reinterpret_cast<float4*>(R1 + kRecWords * i);
    for (int k = 0; k < 4; ++k) {
        float4 w = make_float4(rec[4 * k], rec[4 * k + 1], rec[4 * k + 2], rec[4 * k + 3]);
        d0[k] = w;
        d1[k] = w;
    }
}

template <int DIM>
__global__ void k_unpack_rec(const float* __restrict__ R, int64_t n, double* __restrict__ drho,
                             double* __restrict__ v) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float4 d = *reinterpret_cast<const float4*>(R + kRecWords * i + 12);
    float vv[3] = {d.x, d.y, d.z};
    drho[i] = d.w;
    for (int a = 0; a < DIM; ++a) v[a * n + i] = vv[a];
}

template <typename R>
EulerK<R> make_consts(const sph_eulerian_params* p) {
    EulerK<R> K;
    const sph_domain& d = p->dom;
    double h = d.h;
    double hd2 = d.dim == 2 ? h * h * h * h : h * h * h * h * h;
    K.coef = (R)(-5.0 * wendland_alpha(d.dim) / hd2);
    K.inv_h = (R)(1.0 / h);
    K.rho0 = (R)p->rho0;
    K.c0 = (R)p->c0;
    K.inv_c0 = (R)(1.0 / p->c0);
    K.c0sq = (R)(p->c0 * p->c0);
    K.eta = (R)p->eta;
    K.mu2 = (R)(2.0 * p->mu);
    K.eps_h2 = (R)(0.01 * h * h);
    K.dt = (R)p->dt;
    K.periodic = d.periodic_mask;
    RelGrid g = make_rel_grid(d);
    for (int a = 0; a < 3; ++a) {
        K.half[a] = (R)(0.5 * d.len[a]);
        K.Lh[a] = (R)d.len[a];
        K.Ll[a] = (R)(d.len[a] - (double)K.Lh[a]);
        K.S[a] = (R)g.S[a];
        K.Sl[a] = (R)(g.S[a] - (double)K.S[a]);
        K.ncell[a] = g.n[a];
    }
    return K;
}

int check_params(const sph_eulerian_params* p, const sph_eulerian_state* st) {
    if (!p || !st) return SPH_ERR_ARG;
    int s = sph_check_domain(&p->dom);
    if (s) return s;
    if (p->precision != SPH_FP64 && p->precision != SPH_FP32_KAHAN) return SPH_ERR_ARG;
    if (p->integrator != SPH_TWO_PASS && p->integrator != SPH_FUSED) return SPH_ERR_ARG;
    if (!(p->c0 > 0.0) || !(p->rho0 > 0.0) || !(p->mu >= 0.0) || !(p->eta >= 0.0)) return SPH_ERR_ARG;
    if (p->dom.n > 0 && (!st->row_ptr || !st->col)) return SPH_ERR_ARG;
    if (p->precision == SPH_FP32_KAHAN) {
        // the cell-relative minimum image needs len >= 2 kappa h + 2 S on periodic axes
        if (!rel_grid_periodic_ok(make_rel_grid(p->dom), p->dom.dim, p->dom.kappa * p->dom.h)) return SPH_ERR_ARG;
        if (((uintptr_t)st->rec & 31u) || ((uintptr_t)st->rec_tmp & 31u)) return SPH_ERR_ARG;
    }
    return SPH_OK;
}

// Launch one float64 pass.
template <int DIM>
void launch64(int mode, int out, const sph_eulerian_params* p, const sph_eulerian_state* st, const EulerK<double>& K,
              const double* drho, const double* v, double* drho_out, double* v_out, double* rm, double* rp,
              cudaStream_t s) {
    int64_t n = p->dom.n;
    dim3 g(grid_for(n, 128)), b(128);
#define L64(M, O) k_euler64<DIM, M, O><<<g, b, 0, s>>>(st->pos, st->vol, st->B, st->row_ptr, st->col, n, K, drho, v, drho_out, v_out, rm, rp)
    if (out == OUT_RATES) L64(WANT_BOTH, OUT_RATES);
    else if (out == OUT_MOM) L64(WANT_MOM, OUT_MOM);
    else if (out == OUT_MASS) L64(WANT_MASS, OUT_MASS);
    else L64(WANT_BOTH, OUT_FUSED);
#undef L64
}

template <int DIM, int LANES, bool PER>
void launch32(int out, const sph_eulerian_params* p, const sph_eulerian_state* st, const EulerK<float>& K,
              const float* rin, float* rout, double* rm, double* rp, cudaStream_t s) {
    int64_t n = p->dom.n;
    const int block = 256;
    dim3 g(grid_for(n * LANES, block)), b(block);
#define L32(M, O) k_euler32<DIM, M, O, LANES, PER><<<g, b, 0, s>>>(rin, rout, st->row_ptr, st->col, n, K, rm, rp)
    if (out == OUT_RATES) L32(WANT_BOTH, OUT_RATES);
    else if (out == OUT_MOM) L32(WANT_MOM, OUT_MOM);
    else if (out == OUT_MASS) L32(WANT_MASS, OUT_MASS);
    else L32(WANT_BOTH, OUT_FUSED);
#undef L32
}

template <int DIM, bool PER>
void dispatch32p(int lanes, int out, const sph_eulerian_params* p, const sph_eulerian_state* st,
                 const EulerK<float>& K, const float* rin, float* rout, double* rm, double* rp, cudaStream_t s) {
    switch (lanes) {
        case 1: launch32<DIM, 1, PER>(out, p, st, K, rin, rout, rm, rp, s); break;
        case 2: launch32<DIM, 2, PER>(out, p, st, K, rin, rout, rm, rp, s); break;
        case 8: launch32<DIM, 8, PER>(out, p, st, K, rin, rout, rm, rp, s); break;
        default: launch32<DIM, 4, PER>(out, p, st, K, rin, rout, rm, rp, s); break;
    }
}

// The state's tile plan as launch arguments (tile_m == nullptr: none built).
struct EuPlan {
    GeoArgsE A;
    size_t bytes;
    bool on;
};

EuPlan eu_plan(const sph_ctx* ctx, const sph_eulerian_state* st, int64_t n) {
    EuPlan t;
    t.on = st->plan && st->plan_nnz > 0 && st->plan_maxm > 0;
    t.A = GeoArgsE{nullptr, nullptr, nullptr, nullptr, 0};
    t.bytes = 0;
    if (!t.on) return t;
    TilePlan tp = tile_plan_view(st->plan, n, st->plan_nnz);
    int mc = stage_mcap(st->plan_maxm, 1, ctx->stage_cap);
    t.A = GeoArgsE{tp.tile_m, tp.tile_so, tp.uidx, reinterpret_cast<const float*>(tp.geo), mc, ctx->wait_test_polls};
    const int64_t waves = kChunkRingWaves * (int64_t)6 * (ctx->num_sms > 0 ? ctx->num_sms : 1);
    t.A.chunk_ring = ctx->entry_ring == SPH_RING_CHUNK || (ctx->entry_ring == SPH_RING_AUTO && tp.ntiles >= waves);
    t.bytes = (size_t)mc * 16 + kEntryRingBytes;
    return t;
}

template <int DIM>
void launch32g(int out, int64_t n, const sph_eulerian_state* st, const EulerK<float>& K, const EuPlan& ep,
               const float* rin, float* rout, double* rm, double* rp, int* flags, cudaStream_t s) {
    dim3 g((unsigned)((n + kTileRows - 1) / kTileRows)), b(kTileRows);
#define LG(M, O)                                                                    \
    {                                                                               \
        auto* f = ep.A.chunk_ring ? k_euler32g<DIM, M, O, true> : k_euler32g<DIM, M, O, false>; \
        sph_allow_dynamic_smem((const void*)f);                                     \
        (void)launch_dependent(true, f, g, b, ep.bytes, s, rin, rout, (const int64_t*)st->row_ptr, n, K, ep.A, rm, rp, flags); \
    }
    if (out == OUT_RATES) LG(WANT_BOTH, OUT_RATES)
    else if (out == OUT_MOM) LG(WANT_MOM, OUT_MOM)
    else if (out == OUT_MASS) LG(WANT_MASS, OUT_MASS)
    else LG(WANT_BOTH, OUT_FUSED)
#undef LG
}

void dispatch32(sph_ctx* ctx, int lanes, int out, const sph_eulerian_params* p, const sph_eulerian_state* st,
                const EulerK<float>& K, const float* rin, float* rout, double* rm, double* rp, cudaStream_t s) {
    EuPlan ep = eu_plan(ctx, st, p->dom.n);
    if (ep.on) {
        if (ep.A.chunk_ring) ctx->waits_pending = true;     // the chunk ring's bounded waits
        if (p->dom.dim == 2) launch32g<2>(out, p->dom.n, st, K, ep, rin, rout, rm, rp, ctx->flags, s);
        else launch32g<3>(out, p->dom.n, st, K, ep, rin, rout, rm, rp, ctx->flags, s);
        return;
    }
    bool per = p->dom.periodic_mask != 0;
    if (p->dom.dim == 2) {
        if (per) dispatch32p<2, true>(lanes, out, p, st, K, rin, rout, rm, rp, s);
        else dispatch32p<2, false>(lanes, out, p, st, K, rin, rout, rm, rp, s);
    } else {
        if (per) dispatch32p<3, true>(lanes, out, p, st, K, rin, rout, rm, rp, s);
        else dispatch32p<3, false>(lanes, out, p, st, K, rin, rout, rm, rp, s);
    }
}

}  // namespace

extern "C" int sph_eulerian_pack(sph_ctx* ctx, const sph_eulerian_params* p, const sph_eulerian_state* st,
                                 void* stream) {
    if (!ctx) return SPH_ERR_ARG;
    int r = check_params(p, st);
    if (r) return r;
    int64_t n = p->dom.n;
    if (n == 0) return SPH_OK;
    if (!st->pos || !st->vol || !st->B || !st->drho || !st->v || !st->rec || !st->rec_tmp) return SPH_ERR_ARG;
    cudaStream_t s = as_stream(stream);
    RelGrid g = make_rel_grid(p->dom);
    if (p->dom.dim == 2)
        k_pack_rec<2><<<grid_for(n, 256), 256, 0, s>>>(st->pos, st->vol, st->B, st->drho, st->v, n, g, st->rec,
                                                       st->rec_tmp);
    else
        k_pack_rec<3><<<grid_for(n, 256), 256, 0, s>>>(st->pos, st->vol, st->B, st->drho, st->v, n, g, st->rec,
                                                       st->rec_tmp);
    SPH_LAUNCH_CHECK(ctx);
    return SPH_OK;
}

// Tile plan of the state's lists and fixed geometry (see sph.h).
extern "C" int sph_eulerian_plan_bytes(sph_ctx* ctx, const sph_eulerian_params* p, const sph_eulerian_state* st,
                                       int64_t* bytes_host, void* stream) {
    if (!ctx || !bytes_host) return SPH_ERR_ARG;
    int r = check_params(p, st);
    if (r) return r;
    int64_t n = p->dom.n, nnz = 0, maxrow = 0;
    if (n > 0) {
        r = sph_row_stats(ctx, st->row_ptr, n, as_stream(stream), &nnz, &maxrow);
        if (r) return r;
    }
    *bytes_host = (int64_t)tile_plan_bytes(n, nnz, maxrow, 32);
    return SPH_OK;
}

extern "C" int sph_eulerian_plan(sph_ctx* ctx, const sph_eulerian_params* p, sph_eulerian_state* st, void* stream) {
    if (!ctx) return SPH_ERR_ARG;
    int r = check_params(p, st);
    if (r) return r;
    if (!st->plan || !st->pos || !st->vol || !st->B) return SPH_ERR_ARG;
    int64_t n = p->dom.n;
    cudaStream_t s = as_stream(stream);
    st->plan_nnz = 0;
    st->plan_maxm = st->plan_maxrow = 0;
    if (n == 0) return SPH_OK;
    int64_t nnz = 0, maxrow = 0;
    r = sph_row_stats(ctx, st->row_ptr, n, s, &nnz, &maxrow);
    if (r) return r;
    if (st->plan_bytes < (int64_t)tile_plan_bytes(n, nnz, maxrow, 32)) return SPH_ERR_CAPACITY;
    if (nnz == 0) return SPH_OK;
    int32_t mm = 0, mp = 0, mw = 0;
    r = sph_build_tile_plan(ctx, st->row_ptr, st->col, n, nnz, st->plan, s, &mm, &mp, &mw);
    if (r) return r;
    TilePlan tp = tile_plan_view(st->plan, n, nnz);
    EulerK<double> K = make_consts<double>(p);
    unsigned nt = (unsigned)tp.ntiles;
    float* geo = reinterpret_cast<float*>(tp.geo);
    if (p->dom.dim == 2)
        k_eu_geo<2><<<nt, kTileRows, 0, s>>>(st->pos, st->vol, st->B, st->row_ptr, st->col, tp.lcol, tp.tile_e,
                                             tp.tile_so, n, K, geo);
    else
        k_eu_geo<3><<<nt, kTileRows, 0, s>>>(st->pos, st->vol, st->B, st->row_ptr, st->col, tp.lcol, tp.tile_e,
                                             tp.tile_so, n, K, geo);
    SPH_LAUNCH_CHECK(ctx);
    SPH_CUDA(ctx, cudaStreamSynchronize(s));
    st->plan_nnz = nnz;
    st->plan_maxm = mm;
    st->plan_maxrow = mw;
    return SPH_OK;
}

extern "C" int sph_eulerian_unpack(sph_ctx* ctx, const sph_eulerian_params* p, const sph_eulerian_state* st,
                                   void* stream) {
    if (!ctx) return SPH_ERR_ARG;
    int r = check_params(p, st);
    if (r) return r;
    int64_t n = p->dom.n;
    if (n == 0) return SPH_OK;
    if (!st->drho || !st->v || !st->rec) return SPH_ERR_ARG;
    cudaStream_t s = as_stream(stream);
    if (p->dom.dim == 2) k_unpack_rec<2><<<grid_for(n, 256), 256, 0, s>>>(st->rec, n, st->drho, st->v);
    else k_unpack_rec<3><<<grid_for(n, 256), 256, 0, s>>>(st->rec, n, st->drho, st->v);
    SPH_LAUNCH_CHECK(ctx);
    // a bounded wait that expired in a planned pass since the last read of the flag
    if (!ctx->waits_pending) return SPH_OK;
    ctx->waits_pending = false;
    return sph_take_timeout(ctx, s);
}

// Weakly-compressible EOS of Sec. 3.1.1, p = c0^2 (rho - rho0), solved for the stored
// density offset: drho = p / c0^2.
__global__ void k_eos_drho(const double* __restrict__ pr, int64_t n, double c2, double* __restrict__ drho) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) drho[i] = pr[i] / c2;
}

extern "C" int sph_eulerian_density_from_pressure(sph_ctx* ctx, const sph_eulerian_params* p, const double* pr,
                                                  double* drho, void* stream) {
    if (!ctx || !p) return SPH_ERR_ARG;
    int64_t n = p->dom.n;
    if (n < 0 || !(p->c0 > 0.0) || !isfinite(p->c0)) return SPH_ERR_ARG;
    if (n == 0) return SPH_OK;
    if (!pr || !drho) return SPH_ERR_ARG;
    cudaStream_t s = as_stream(stream);
    k_eos_drho<<<grid_for(n, 256), 256, 0, s>>>(pr, n, p->c0 * p->c0, drho);
    SPH_LAUNCH_CHECK(ctx);
    return SPH_OK;
}

extern "C" int sph_eulerian_rates(sph_ctx* ctx, const sph_eulerian_params* p, const sph_eulerian_state* st,
                                  double* drho_dt, double* dmom_dt, void* stream) {
    if (!ctx) return SPH_ERR_ARG;
    int r = check_params(p, st);
    if (r) return r;
    int64_t n = p->dom.n;
    if (n == 0) return SPH_OK;
    if (!drho_dt || !dmom_dt) return SPH_ERR_ARG;
    cudaStream_t s = as_stream(stream);
    if (p->precision == SPH_FP64) {
        if (!st->pos || !st->vol || !st->B || !st->drho || !st->v) return SPH_ERR_ARG;
        EulerK<double> K = make_consts<double>(p);
        if (p->dom.dim == 2) launch64<2>(0, OUT_RATES, p, st, K, st->drho, st->v, nullptr, nullptr, drho_dt, dmom_dt, s);
        else launch64<3>(0, OUT_RATES, p, st, K, st->drho, st->v, nullptr, nullptr, drho_dt, dmom_dt, s);
    } else {
        if (!st->rec) return SPH_ERR_ARG;
        EulerK<float> K = make_consts<float>(p);
        dispatch32(ctx, ctx->lanes[SPH_PASS_EULERIAN], OUT_RATES, p, st, K, st->rec, nullptr, drho_dt, dmom_dt, s);
    }
    SPH_LAUNCH_CHECK(ctx);
    return SPH_OK;
}

extern "C" int sph_eulerian_step(sph_ctx* ctx, const sph_eulerian_params* p, const sph_eulerian_state* st,
                                 int nsteps, void* stream) {
    if (!ctx || nsteps < 0) return SPH_ERR_ARG;
    int r = check_params(p, st);
    if (r) return r;
    int64_t n = p->dom.n;
    if (n == 0 || nsteps == 0) return SPH_OK;
    cudaStream_t s = as_stream(stream);
    int dim = p->dom.dim;
    if (p->precision == SPH_FP64) {
        if (!st->pos || !st->vol || !st->B || !st->drho || !st->v || !st->drho_tmp || !st->v_tmp) return SPH_ERR_ARG;
        EulerK<double> K = make_consts<double>(p);
        double *d0 = st->drho, *v0 = st->v, *d1 = st->drho_tmp, *v1 = st->v_tmp;
        for (int k = 0; k < nsteps; ++k) {
            if (p->integrator == SPH_TWO_PASS) {
                int t = sph_timer_begin(ctx, SPH_TIMER_EU_MOMENTUM, s);
                if (dim == 2) launch64<2>(0, OUT_MOM, p, st, K, d0, v0, d1, v1, nullptr, nullptr, s);
                else launch64<3>(0, OUT_MOM, p, st, K, d0, v0, d1, v1, nullptr, nullptr, s);
                sph_timer_end(ctx, t, s);
                t = sph_timer_begin(ctx, SPH_TIMER_EU_MASS, s);
                if (dim == 2) launch64<2>(0, OUT_MASS, p, st, K, d1, v1, d0, v0, nullptr, nullptr, s);
                else launch64<3>(0, OUT_MASS, p, st, K, d1, v1, d0, v0, nullptr, nullptr, s);
                sph_timer_end(ctx, t, s);
            } else {
                int t = sph_timer_begin(ctx, SPH_TIMER_EU_FUSED, s);
                if (dim == 2) launch64<2>(0, OUT_FUSED, p, st, K, d0, v0, d1, v1, nullptr, nullptr, s);
                else launch64<3>(0, OUT_FUSED, p, st, K, d0, v0, d1, v1, nullptr, nullptr, s);
                sph_timer_end(ctx, t, s);
                double* tt = d0; d0 = d1; d1 = tt;
                tt = v0; v0 = v1; v1 = tt;
            }
        }
        SPH_LAUNCH_CHECK(ctx);
        if (d0 != st->drho) {
            SPH_CUDA(ctx, cudaMemcpyAsync(st->drho, d0, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
            SPH_CUDA(ctx, cudaMemcpyAsync(st->v, v0, dim * n * sizeof(double), cudaMemcpyDeviceToDevice, s));
        }
        return SPH_OK;
    }
    if (!st->rec || !st->rec_tmp) return SPH_ERR_ARG;
    EulerK<float> K = make_consts<float>(p);
    float* r0 = st->rec;
    float* r1 = st->rec_tmp;
    int lanes = ctx->lanes[SPH_PASS_EULERIAN];
    for (int k = 0; k < nsteps; ++k) {
        if (p->integrator == SPH_TWO_PASS) {
            int t = sph_timer_begin(ctx, SPH_TIMER_EU_MOMENTUM, s);
            dispatch32(ctx, lanes, OUT_MOM, p, st, K, r0, r1, nullptr, nullptr, s);
            sph_timer_end(ctx, t, s);
            t = sph_timer_begin(ctx, SPH_TIMER_EU_MASS, s);
            dispatch32(ctx, lanes, OUT_MASS, p, st, K, r1, r0, nullptr, nullptr, s);
            sph_timer_end(ctx, t, s);
        } else {
            int t = sph_timer_begin(ctx, SPH_TIMER_EU_FUSED, s);
            dispatch32(ctx, lanes, OUT_FUSED, p, st, K, r0, r1, nullptr, nullptr, s);
            sph_timer_end(ctx, t, s);
            float* tt = r0; r0 = r1; r1 = tt;
        }
    }
    SPH_LAUNCH_CHECK(ctx);
    if (r0 != st->rec)
        SPH_CUDA(ctx, cudaMemcpyAsync(st->rec, r0, (size_t)n * kRecWords * 4, cudaMemcpyDeviceToDevice, s));
    return SPH_OK;
}

// Autotuner of the float32 pair passes (lanes per particle in {1, 2, 4, 8}); the
// dynamic state is saved before and restored after every trial.
extern "C" int sph_autotune_eulerian(sph_ctx* ctx, const sph_eulerian_params* p, const sph_eulerian_state* st,
                                     int trial_steps, int* lanes_host, double* ms_host, void* stream) {
    if (!ctx || trial_steps < 1) return SPH_ERR_ARG;
    int r = check_params(p, st);
    if (r) return r;
    if (p->precision != SPH_FP32_KAHAN || !st->rec || !st->rec_tmp) return SPH_ERR_ARG;
    int64_t n = p->dom.n;
    if (n == 0) return SPH_OK;
    cudaStream_t s = as_stream(stream);
    size_t bq = (size_t)n * kRecWords * 4;
    void* save = sph_scratch(ctx, S_MISC3, bq, &r);
    if (r) return r;
    SPH_CUDA(ctx, cudaMemcpyAsync(save, st->rec, bq, cudaMemcpyDeviceToDevice, s));
    cudaEvent_t e0, e1;
    SPH_CUDA(ctx, cudaEventCreate(&e0));
    SPH_CUDA(ctx, cudaEventCreate(&e1));
    const int lanes_set[4] = {1, 2, 4, 8};
    int keep = ctx->lanes[SPH_PASS_EULERIAN];
    const int timing = ctx->timing;
    ctx->timing = 0;
    double best = 1e300;
    int bl = keep;
    for (int li = 0; li < 4; ++li) {
        ctx->lanes[SPH_PASS_EULERIAN] = lanes_set[li];
        r = sph_eulerian_step(ctx, p, st, 1, stream);
        if (r) break;
        SPH_CUDA(ctx, cudaEventRecord(e0, s));
        r = sph_eulerian_step(ctx, p, st, trial_steps, stream);
        if (r) break;
        SPH_CUDA(ctx, cudaEventRecord(e1, s));
        SPH_CUDA(ctx, cudaEventSynchronize(e1));
        float ms = 0.0f;
        SPH_CUDA(ctx, cudaEventElapsedTime(&ms, e0, e1));
        if (ms < best) { best = ms; bl = lanes_set[li]; }
        SPH_CUDA(ctx, cudaMemcpyAsync(st->rec, save, bq, cudaMemcpyDeviceToDevice, s));
        SPH_CUDA(ctx, cudaMemcpyAsync(st->rec_tmp, save, bq, cudaMemcpyDeviceToDevice, s));
    }
    ctx->timing = timing;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (r) { ctx->lanes[SPH_PASS_EULERIAN] = keep; return r; }
    ctx->lanes[SPH_PASS_EULERIAN] = bl;
    if (lanes_host) *lanes_host = bl;
    if (ms_host) *ms_host = best / trial_steps;
    SPH_CUDA(ctx, cudaStreamSynchronize(s));
    return SPH_OK;
}
