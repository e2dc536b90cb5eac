// a5/a6: Riemann-based Eulerian weakly-compressible SPH (Sec. 3.1; Eqs. 18, 25-27).
//
// Two pair-pass kernels share one per-pair device function:
//  * k_euler64: float64 structure-of-arrays state, one thread per particle;
//  * k_euler32: float32 packed records (positions split hi+lo so that r_ij keeps
//    ~1e-7 relative accuracy in any box), LANES consecutive lanes per particle
//    striding over the CSR row, compensated (Kahan) sums, group shuffle reduce.
// A pass computes the mass and/or momentum rates of a particle and applies the
// pointwise part of the update in its epilogue (EOS p = c0^2 drho, velocity
// from momentum), so a step is one (fused) or two (momentum, continuity) launches.
#include "common.cuh"
#include "euler_core.cuh"

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

template <int DIM, int MODE, int OUT, int LANES>
__global__ void __launch_bounds__(256) k_euler32(const float4* __restrict__ geo, const int64_t* __restrict__ row_ptr,
                                                 const int32_t* __restrict__ col, int64_t n, EulerK<float> K,
                                                 const float4* __restrict__ q, float4* __restrict__ q_out,
                                                 double* __restrict__ rate_mass, double* __restrict__ rate_mom) {
    constexpr int NS = NSym<DIM>::v;
    int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t i = gt / LANES;
    int lane = (int)(gt % LANES);
    bool active = i < n;
    int64_t ii = active ? i : 0;
    float xhi[DIM], xli[DIM], Vi, Bi[NS], vi[DIM], dri;
    load_geo32<DIM>(reinterpret_cast<const float4*>(geo), ii, xhi, xli, Vi, Bi);
    load_q32<DIM>(q, ii, vi, dri);
    Kahan<float> am;
    Kahan<float> ap[DIM];
    am.init();
#pragma unroll
    for (int a = 0; a < DIM; ++a) ap[a].init();
    int64_t b = active ? row_ptr[ii] : 0, e = active ? row_ptr[ii + 1] : 0;
    for (int64_t p = b + lane; p < e; p += LANES) {
        int j = __ldg(&col[p]);
        float xhj[DIM], xlj[DIM], Vj, Bj[NS], vj[DIM], drj;
        load_geo32<DIM>(geo, j, xhj, xlj, Vj, Bj);
        load_q32<DIM>(q, j, vj, drj);
        float r[DIM], d2 = 0.0f;
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            float dh = xhi[a] - xhj[a];
            float dl = xli[a] - xlj[a];
            if ((K.periodic >> a) & 1u) {
                if (dh > K.half[a]) { dh -= K.Lh[a]; dl -= K.Ll[a]; }
                else if (dh < -K.half[a]) { dh += K.Lh[a]; dl += K.Ll[a]; }
            }
            r[a] = dh + dl;
            d2 = fmaf(r[a], r[a], d2);
        }
        float m = 0.0f, mo[DIM];
        euler_pair<DIM, MODE, float>(r, d2, Bi, Bj, vi, vj, dri, drj, Vj, K, m, mo);
        if (MODE & WANT_MASS) am.add(m);
        if (MODE & WANT_MOM) {
#pragma unroll
            for (int a = 0; a < DIM; ++a) ap[a].add(mo[a]);
        }
    }
    float rm = group_sum<LANES>(am.value());
    float rp[DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a) rp[a] = group_sum<LANES>(ap[a].value());
    if (!active || lane != 0) return;
    float rho_i = K.rho0 + dri;
    float vn[DIM];
    if (OUT == OUT_RATES) {
        if (MODE & WANT_MASS) rate_mass[i] = (double)rm;
        if (MODE & WANT_MOM)
            for (int a = 0; a < DIM; ++a) rate_mom[a * n + i] = (double)rp[a];
    } else if (OUT == OUT_MOM) {
#pragma unroll
        for (int a = 0; a < DIM; ++a) vn[a] = vi[a] + K.dt * rp[a] / rho_i;
        store_q32<DIM>(q_out, i, vn, dri);
    } else if (OUT == OUT_MASS) {
        float ddr = K.dt * rm;
        float dr1 = dri + ddr;
        float ratio = 1.0f - ddr / (K.rho0 + dr1);     // rho^n / rho^{n+1}
#pragma unroll
        for (int a = 0; a < DIM; ++a) vn[a] = vi[a] * ratio;
        store_q32<DIM>(q_out, i, vn, dr1);
    } else {
        float ddr = K.dt * rm;
        float dr1 = dri + ddr;
        float rho1 = K.rho0 + dr1;
        float ratio = 1.0f - ddr / rho1;
#pragma unroll
        for (int a = 0; a < DIM; ++a) vn[a] = vi[a] * ratio + K.dt * rp[a] / rho1;
        store_q32<DIM>(q_out, i, vn, dr1);
    }
}

// ---------------------------------------------------------------- pack / unpack
template <int DIM>
__global__ void k_pack_geo(const double* __restrict__ pos, const double* __restrict__ vol,
                           const double* __restrict__ B, int64_t n, float* __restrict__ geo) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float xh[3], xl[3];
    for (int a = 0; a < DIM; ++a) {
        double x = pos[a * n + i];
        xh[a] = (float)x;
        xl[a] = (float)(x - (double)xh[a]);
    }
    if (DIM == 2) {
        float* g = geo + 8 * i;
        g[0] = xh[0]; g[1] = xh[1]; g[2] = xl[0]; g[3] = xl[1];
        g[4] = (float)vol[i]; g[5] = (float)B[i]; g[6] = (float)B[n + i]; g[7] = (float)B[2 * n + i];
    } else {
        float* g = geo + 16 * i;
        g[0] = xh[0]; g[1] = xh[1]; g[2] = xh[2]; g[3] = (float)vol[i];
        g[4] = xl[0]; g[5] = xl[1]; g[6] = xl[2]; g[7] = (float)B[i];
        g[8] = (float)B[n + i]; g[9] = (float)B[2 * n + i]; g[10] = (float)B[3 * n + i]; g[11] = (float)B[4 * n + i];
        g[12] = (float)B[5 * n + i]; g[13] = 0.0f; g[14] = 0.0f; g[15] = 0.0f;
    }
}

template <int DIM>
__global__ void k_pack_q(const double* __restrict__ drho, const double* __restrict__ v, int64_t n,
                         float4* __restrict__ q) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float vv[DIM];
    for (int a = 0; a < DIM; ++a) vv[a] = (float)v[a * n + i];
    store_q32<DIM>(q, i, vv, (float)drho[i]);
}

template <int DIM>
__global__ void k_unpack_q(const float4* __restrict__ q, int64_t n, double* __restrict__ drho,
                           double* __restrict__ v) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float vv[DIM], dr;
    float4 a = q[i];
    if (DIM == 2) { vv[0] = a.x; vv[1] = a.y; dr = a.z; }
    else { vv[0] = a.x; vv[1] = a.y; vv[2] = a.z; dr = a.w; }
    drho[i] = dr;
    for (int c = 0; c < DIM; ++c) v[c * n + i] = vv[c];
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
    for (int a = 0; a < 3; ++a) {
        K.half[a] = (R)(0.5 * d.len[a]);
        K.Lh[a] = (R)d.len[a];
        K.Ll[a] = (R)(d.len[a] - (double)K.Lh[a]);
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

template <int DIM, int LANES>
void launch32(int out, const sph_eulerian_params* p, const sph_eulerian_state* st, const EulerK<float>& K,
              const float4* q, float4* q_out, double* rm, double* rp, cudaStream_t s) {
    int64_t n = p->dom.n;
    const int block = 256;
    dim3 g(grid_for(n * LANES, block)), b(block);
    const float4* geo = reinterpret_cast<const float4*>(st->geo);
#define L32(M, O) k_euler32<DIM, M, O, LANES><<<g, b, 0, s>>>(geo, st->row_ptr, st->col, n, K, q, q_out, rm, rp)
    if (out == OUT_RATES) L32(WANT_BOTH, OUT_RATES);
    else if (out == OUT_MOM) L32(WANT_MOM, OUT_MOM);
    else if (out == OUT_MASS) L32(WANT_MASS, OUT_MASS);
    else L32(WANT_BOTH, OUT_FUSED);
#undef L32
}

template <int DIM>
void dispatch32(int g_lanes, int out, const sph_eulerian_params* p, const sph_eulerian_state* st, const EulerK<float>& K,
                const float4* q, float4* q_out, double* rm, double* rp, cudaStream_t s) {
    switch (g_lanes) {
        case 1: launch32<DIM, 1>(out, p, st, K, q, q_out, rm, rp, s); break;
        case 2: launch32<DIM, 2>(out, p, st, K, q, q_out, rm, rp, s); break;
        case 8: launch32<DIM, 8>(out, p, st, K, q, q_out, rm, rp, s); break;
        default: launch32<DIM, 4>(out, p, st, K, q, q_out, rm, rp, s); break;
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
    if (!st->pos || !st->vol || !st->B || !st->drho || !st->v || !st->geo || !st->q) return SPH_ERR_ARG;
    cudaStream_t s = as_stream(stream);
    if (p->dom.dim == 2) {
        k_pack_geo<2><<<grid_for(n, 256), 256, 0, s>>>(st->pos, st->vol, st->B, n, st->geo);
        k_pack_q<2><<<grid_for(n, 256), 256, 0, s>>>(st->drho, st->v, n, reinterpret_cast<float4*>(st->q));
    } else {
        k_pack_geo<3><<<grid_for(n, 256), 256, 0, s>>>(st->pos, st->vol, st->B, n, st->geo);
        k_pack_q<3><<<grid_for(n, 256), 256, 0, s>>>(st->drho, st->v, n, reinterpret_cast<float4*>(st->q));
    }
    SPH_LAUNCH_CHECK(ctx);
    return SPH_OK;
}

extern "C" int sph_eulerian_unpack(sph_ctx* ctx, const sph_eulerian_params* p, const sph_eulerian_state* st,
                                   void* stream) {
    if (!ctx) return SPH_ERR_ARG;
    int r = check_params(p, st);
    if (r) return r;
    int64_t n = p->dom.n;
    if (n == 0) return SPH_OK;
    if (!st->drho || !st->v || !st->q) return SPH_ERR_ARG;
    cudaStream_t s = as_stream(stream);
    const float4* q = reinterpret_cast<const float4*>(st->q);
    if (p->dom.dim == 2) k_unpack_q<2><<<grid_for(n, 256), 256, 0, s>>>(q, n, st->drho, st->v);
    else k_unpack_q<3><<<grid_for(n, 256), 256, 0, s>>>(q, n, st->drho, st->v);
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
        if (!st->geo || !st->q) return SPH_ERR_ARG;
        EulerK<float> K = make_consts<float>(p);
        const float4* q = reinterpret_cast<const float4*>(st->q);
        if (p->dom.dim == 2) dispatch32<2>(ctx->lanes[SPH_PASS_EULERIAN], OUT_RATES, p, st, K, q, nullptr, drho_dt, dmom_dt, s);
        else dispatch32<3>(ctx->lanes[SPH_PASS_EULERIAN], OUT_RATES, p, st, K, q, nullptr, drho_dt, dmom_dt, s);
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
    if (!st->geo || !st->q || !st->q_tmp) return SPH_ERR_ARG;
    EulerK<float> K = make_consts<float>(p);
    float4* q0 = reinterpret_cast<float4*>(st->q);
    float4* q1 = reinterpret_cast<float4*>(st->q_tmp);
    int lanes = ctx->lanes[SPH_PASS_EULERIAN];
    for (int k = 0; k < nsteps; ++k) {
        if (p->integrator == SPH_TWO_PASS) {
            int t = sph_timer_begin(ctx, SPH_TIMER_EU_MOMENTUM, s);
            if (dim == 2) dispatch32<2>(lanes, OUT_MOM, p, st, K, q0, q1, nullptr, nullptr, s);
            else dispatch32<3>(lanes, OUT_MOM, p, st, K, q0, q1, nullptr, nullptr, s);
            sph_timer_end(ctx, t, s);
            t = sph_timer_begin(ctx, SPH_TIMER_EU_MASS, s);
            if (dim == 2) dispatch32<2>(lanes, OUT_MASS, p, st, K, q1, q0, nullptr, nullptr, s);
            else dispatch32<3>(lanes, OUT_MASS, p, st, K, q1, q0, nullptr, nullptr, s);
            sph_timer_end(ctx, t, s);
        } else {
            int t = sph_timer_begin(ctx, SPH_TIMER_EU_FUSED, s);
            if (dim == 2) dispatch32<2>(lanes, OUT_FUSED, p, st, K, q0, q1, nullptr, nullptr, s);
            else dispatch32<3>(lanes, OUT_FUSED, p, st, K, q0, q1, nullptr, nullptr, s);
            sph_timer_end(ctx, t, s);
            float4* tt = q0; q0 = q1; q1 = tt;
        }
    }
    SPH_LAUNCH_CHECK(ctx);
    if (q0 != reinterpret_cast<float4*>(st->q))
        SPH_CUDA(ctx, cudaMemcpyAsync(st->q, q0, n * sizeof(float4), cudaMemcpyDeviceToDevice, s));
    return SPH_OK;
}

// Autotuner of the float32 pair passes (lanes per particle in {1, 2, 4, 8}); the
// packed state q is saved before and restored after every trial.
extern "C" int sph_autotune_eulerian(sph_ctx* ctx, const sph_eulerian_params* p, const sph_eulerian_state* st,
                                     int trial_steps, int* lanes_host, double* ms_host, void* stream) {
    if (!ctx || trial_steps < 1) return SPH_ERR_ARG;
    int r = check_params(p, st);
    if (r) return r;
    if (p->precision != SPH_FP32_KAHAN || !st->geo || !st->q || !st->q_tmp) return SPH_ERR_ARG;
    int64_t n = p->dom.n;
    if (n == 0) return SPH_OK;
    cudaStream_t s = as_stream(stream);
    size_t bq = (size_t)n * 16;
    void* save = sph_scratch(ctx, S_MISC3, bq, &r);
    if (r) return r;
    SPH_CUDA(ctx, cudaMemcpyAsync(save, st->q, bq, cudaMemcpyDeviceToDevice, s));
    cudaEvent_t e0, e1;
    SPH_CUDA(ctx, cudaEventCreate(&e0));
    SPH_CUDA(ctx, cudaEventCreate(&e1));
    const int lanes_set[4] = {1, 2, 4, 8};
    int keep = ctx->lanes[SPH_PASS_EULERIAN];
    bool timing = ctx->timing;
    ctx->timing = false;
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
        SPH_CUDA(ctx, cudaMemcpyAsync(st->q, save, bq, cudaMemcpyDeviceToDevice, s));
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
