// a7-a9: total-Lagrangian SPH for solids (Sec. 3.2; Eqs. 28-31).
//
// A step is two pair passes over the fixed CSR lists of the reference
// configuration:
//   pass A (momentum, Eq. 30): a_i = (1/rho0) sum_j (M_i + M_j) grad0 W_ij V0_j,
//          v_i += dt a_i (v = 0 on clamped particles);
//   pass B (deformation rate, Eq. 31): dF_i/dt = (sum_j V0_j (v_j - v_i) (x) grad0 W_ij) B0_i,
//          F_i += dt dF_i/dt (F = I on clamped particles), x_i += dt v_i, and, fused
//          in the epilogue, the next step's stress factor M_i = P(F_i) B0_i^T.
// F is carried as H = F - I and the stress is written in H (Green strain
// E = (H + H^T + H^T H)/2, neo-Hookean S = C^-1 (2 G E + lambda ln J I) with
// ln J = log1p(det(I+H) - 1) expanded in H), which keeps float32 accurate for
// the small strains of a solid.
#include "common.cuh"

namespace {

template <typename R>
struct TLK {
    R coef, inv_h;       // Wendland gs coefficient and 1/h
    R inv_rho0, dt, lam, G;
    int law;
    R half[3], Lh[3], Ll[3];
    uint32_t periodic;
};

template <typename R> __device__ __forceinline__ R log1p_(R x);
template <> __device__ __forceinline__ double log1p_<double>(double x) { return log1p(x); }
template <> __device__ __forceinline__ float log1p_<float>(float x) { return log1pf(x); }

// M = P B0^T with P = (I + H) S(H); H, M row-major DIM x DIM, B0 symmetric (NS entries).
template <int DIM, typename R>
__device__ __forceinline__ void stress_factor(const R* H, const R* B0s, const TLK<R>& K, R* M) {
    R E[DIM][DIM], S[DIM][DIM], B0[DIM][DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a)
#pragma unroll
        for (int b = 0; b < DIM; ++b) {
            R hth = R(0);
#pragma unroll
            for (int k = 0; k < DIM; ++k) hth += H[k * DIM + a] * H[k * DIM + b];
            E[a][b] = R(0.5) * (H[a * DIM + b] + H[b * DIM + a] + hth);
        }
    if (DIM == 2) {
        B0[0][0] = B0s[0]; B0[0][1] = B0[1][0] = B0s[1]; B0[1][1] = B0s[2];
    } else {
        B0[0][0] = B0s[0]; B0[0][1] = B0[1][0] = B0s[1]; B0[0][2] = B0[2][0] = B0s[2];
        B0[1][1] = B0s[3]; B0[1][2] = B0[2][1] = B0s[4]; B0[2][2] = B0s[5];
    }
    if (K.law == SPH_SVK) {
        R tr = R(0);
#pragma unroll
        for (int a = 0; a < DIM; ++a) tr += E[a][a];
#pragma unroll
        for (int a = 0; a < DIM; ++a)
#pragma unroll
            for (int b = 0; b < DIM; ++b) S[a][b] = R(2) * K.G * E[a][b] + (a == b ? K.lam * tr : R(0));
    } else {
        // j1 = det(I + H) - 1 expanded in H
        R j1;
        if (DIM == 2) {
            j1 = H[0] + H[3] + (H[0] * H[3] - H[1] * H[2]);
        } else {
            R tr = H[0] + H[4] + H[8];
            R m2 = (H[0] * H[4] - H[1] * H[3]) + (H[0] * H[8] - H[2] * H[6]) + (H[4] * H[8] - H[5] * H[7]);
            R d3 = H[0] * (H[4] * H[8] - H[5] * H[7]) - H[1] * (H[3] * H[8] - H[5] * H[6]) +
                   H[2] * (H[3] * H[7] - H[4] * H[6]);
            j1 = tr + m2 + d3;
        }
        R lnJ = log1p_<R>(j1);
        // C = I + 2E, C^-1 by adjugate; det C = J^2
        R C[DIM][DIM], Ci[DIM][DIM];
#pragma unroll
        for (int a = 0; a < DIM; ++a)
#pragma unroll
            for (int b = 0; b < DIM; ++b) C[a][b] = (a == b ? R(1) : R(0)) + R(2) * E[a][b];
        if (DIM == 2) {
            R det = C[0][0] * C[1][1] - C[0][1] * C[1][0];
            R id = R(1) / det;
            Ci[0][0] = C[1][1] * id; Ci[1][1] = C[0][0] * id;
            Ci[0][1] = -C[0][1] * id; Ci[1][0] = -C[1][0] * id;
        } else {
            R c00 = C[1][1] * C[2][2] - C[1][2] * C[2][1];
            R c01 = C[0][2] * C[2][1] - C[0][1] * C[2][2];
            R c02 = C[0][1] * C[1][2] - C[0][2] * C[1][1];
            R c10 = C[1][2] * C[2][0] - C[1][0] * C[2][2];
            R c11 = C[0][0] * C[2][2] - C[0][2] * C[2][0];
            R c12 = C[0][2] * C[1][0] - C[0][0] * C[1][2];
            R c20 = C[1][0] * C[2][1] - C[1][1] * C[2][0];
            R c21 = C[0][1] * C[2][0] - C[0][0] * C[2][1];
            R c22 = C[0][0] * C[1][1] - C[0][1] * C[1][0];
            R det = C[0][0] * c00 + C[0][1] * c10 + C[0][2] * c20;
            R id = R(1) / det;
            Ci[0][0] = c00 * id; Ci[0][1] = c01 * id; Ci[0][2] = c02 * id;
            Ci[1][0] = c10 * id; Ci[1][1] = c11 * id; Ci[1][2] = c12 * id;
            Ci[2][0] = c20 * id; Ci[2][1] = c21 * id; Ci[2][2] = c22 * id;
        }
        // S = C^-1 (2 G E + lambda ln J I)
#pragma unroll
        for (int a = 0; a < DIM; ++a)
#pragma unroll
            for (int b = 0; b < DIM; ++b) {
                R acc = R(0);
#pragma unroll
                for (int k = 0; k < DIM; ++k) acc += Ci[a][k] * (R(2) * K.G * E[k][b] + (k == b ? K.lam * lnJ : R(0)));
                S[a][b] = acc;
            }
    }
    // P = (I + H) S, M = P B0
    R P[DIM][DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a)
#pragma unroll
        for (int b = 0; b < DIM; ++b) {
            R acc = S[a][b];
#pragma unroll
            for (int k = 0; k < DIM; ++k) acc += H[a * DIM + k] * S[k][b];
            P[a][b] = acc;
        }
#pragma unroll
    for (int a = 0; a < DIM; ++a)
#pragma unroll
        for (int b = 0; b < DIM; ++b) {
            R acc = R(0);
#pragma unroll
            for (int k = 0; k < DIM; ++k) acc += P[a][k] * B0[k][b];
            M[a * DIM + b] = acc;
        }
}

// dF/dt = L B0 with B0 symmetric
template <int DIM, typename R>
__device__ __forceinline__ void times_b0(const R* L, const R* B0s, R* out) {
    R B0[DIM][DIM];
    if (DIM == 2) {
        B0[0][0] = B0s[0]; B0[0][1] = B0[1][0] = B0s[1]; B0[1][1] = B0s[2];
    } else {
        B0[0][0] = B0s[0]; B0[0][1] = B0[1][0] = B0s[1]; B0[0][2] = B0[2][0] = B0s[2];
        B0[1][1] = B0s[3]; B0[1][2] = B0[2][1] = B0s[4]; B0[2][2] = B0s[5];
    }
#pragma unroll
    for (int a = 0; a < DIM; ++a)
#pragma unroll
        for (int b = 0; b < DIM; ++b) {
            R acc = R(0);
#pragma unroll
            for (int k = 0; k < DIM; ++k) acc += L[a * DIM + k] * B0[k][b];
            out[a * DIM + b] = acc;
        }
}

enum { OUT_RATES = 0, OUT_STEP = 1 };

// ---------------------------------------------------------------- float64 path
template <int DIM>
__global__ void k_tl_stress64(const double* __restrict__ H, const double* __restrict__ B0, int64_t n,
                              TLK<double> K, double* __restrict__ M) {
    constexpr int NS = DIM == 2 ? 3 : 6;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double h[DIM * DIM], b[NS], m[DIM * DIM];
    for (int k = 0; k < DIM * DIM; ++k) h[k] = H[k * n + i];
    for (int s = 0; s < NS; ++s) b[s] = B0[s * n + i];
    stress_factor<DIM, double>(h, b, K, m);
    for (int k = 0; k < DIM * DIM; ++k) M[k * n + i] = m[k];
}

template <int DIM>
__device__ __forceinline__ void pair_r64(const double* xi, const double* __restrict__ r0, int64_t n, int j,
                                         const TLK<double>& K, double* r, double& d2) {
    d2 = 0.0;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        double dx = xi[a] - r0[a * n + j];
        if ((K.periodic >> a) & 1u) {
            if (dx > K.half[a]) dx -= K.Lh[a];
            else if (dx < -K.half[a]) dx += K.Lh[a];
        }
        r[a] = dx;
        d2 += dx * dx;
    }
}

template <int DIM, int OUT>
__global__ void k_tl_mom64(const double* __restrict__ r0, const double* __restrict__ V0,
                           const uint8_t* __restrict__ fixed, const int64_t* __restrict__ row_ptr,
                           const int32_t* __restrict__ col, int64_t n, TLK<double> K,
                           const double* __restrict__ M, double* __restrict__ v, double* __restrict__ dvdt) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double xi[DIM], Mi[DIM * DIM], acc[DIM];
    for (int a = 0; a < DIM; ++a) { xi[a] = r0[a * n + i]; acc[a] = 0.0; }
    for (int k = 0; k < DIM * DIM; ++k) Mi[k] = M[k * n + i];
    for (int64_t p = row_ptr[i], e = row_ptr[i + 1]; p < e; ++p) {
        int j = col[p];
        double r[DIM], d2;
        pair_r64<DIM>(xi, r0, n, j, K, r, d2);
        double gs = wendland_gs<double>(sqrt(d2) * K.inv_h, K.coef) * V0[j];
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            double s = 0.0;
#pragma unroll
            for (int b = 0; b < DIM; ++b) s += (Mi[a * DIM + b] + M[(a * DIM + b) * n + j]) * (gs * r[b]);
            acc[a] += s;
        }
    }
    if (OUT == OUT_RATES) {
        for (int a = 0; a < DIM; ++a) dvdt[a * n + i] = acc[a] * K.inv_rho0;
    } else {
        bool fx = fixed && fixed[i];
        for (int a = 0; a < DIM; ++a) v[a * n + i] = fx ? 0.0 : v[a * n + i] + K.dt * (acc[a] * K.inv_rho0);
    }
}

template <int DIM, int OUT>
__global__ void k_tl_defo64(const double* __restrict__ r0, const double* __restrict__ V0,
                            const double* __restrict__ B0, const uint8_t* __restrict__ fixed,
                            const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col, int64_t n,
                            TLK<double> K, const double* __restrict__ v, double* __restrict__ H,
                            double* __restrict__ x, double* __restrict__ M, double* __restrict__ dFdt) {
    constexpr int NS = DIM == 2 ? 3 : 6;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double xi[DIM], vi[DIM], L[DIM * DIM], b0[NS];
    for (int a = 0; a < DIM; ++a) { xi[a] = r0[a * n + i]; vi[a] = v[a * n + i]; }
    for (int k = 0; k < DIM * DIM; ++k) L[k] = 0.0;
    for (int s = 0; s < NS; ++s) b0[s] = B0[s * n + i];
    for (int64_t p = row_ptr[i], e = row_ptr[i + 1]; p < e; ++p) {
        int j = col[p];
        double r[DIM], d2;
        pair_r64<DIM>(xi, r0, n, j, K, r, d2);
        double gs = wendland_gs<double>(sqrt(d2) * K.inv_h, K.coef);
        double w = V0[j];
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            double dv = w * (v[a * n + j] - vi[a]);
#pragma unroll
            for (int b = 0; b < DIM; ++b) L[a * DIM + b] += dv * (gs * r[b]);
        }
    }
    double Fd[DIM * DIM];
    times_b0<DIM, double>(L, b0, Fd);
    if (OUT == OUT_RATES) {
        for (int k = 0; k < DIM * DIM; ++k) dFdt[k * n + i] = Fd[k];
        return;
    }
    bool fx = fixed && fixed[i];
    double h[DIM * DIM], m[DIM * DIM];
    for (int k = 0; k < DIM * DIM; ++k) {
        h[k] = fx ? 0.0 : H[k * n + i] + K.dt * Fd[k];
        H[k * n + i] = h[k];
    }
    for (int a = 0; a < DIM; ++a) x[a * n + i] += K.dt * vi[a];
    stress_factor<DIM, double>(h, b0, K, m);
    for (int k = 0; k < DIM * DIM; ++k) M[k * n + i] = m[k];
}

// ---------------------------------------------------------------- float32 path
template <int DIM>
__device__ __forceinline__ void load_geo(const float4* __restrict__ geo, int64_t i, float* xh, float* xl, float& V,
                                         float& fx) {
    float4 a = __ldg(&geo[2 * i]);
    float4 b = __ldg(&geo[2 * i + 1]);
    if (DIM == 2) { xh[0] = a.x; xh[1] = a.y; xl[0] = a.z; xl[1] = a.w; V = b.x; fx = b.y; }
    else { xh[0] = a.x; xh[1] = a.y; xh[2] = a.z; V = a.w; xl[0] = b.x; xl[1] = b.y; xl[2] = b.z; fx = b.w; }
}

template <int DIM>
__device__ __forceinline__ void load_M(const float4* __restrict__ M, int64_t i, float* m) {
    if (DIM == 2) {
        float4 a = __ldg(&M[i]);
        m[0] = a.x; m[1] = a.y; m[2] = a.z; m[3] = a.w;
    } else {
        float4 a = __ldg(&M[3 * i]), b = __ldg(&M[3 * i + 1]), c = __ldg(&M[3 * i + 2]);
        m[0] = a.x; m[1] = a.y; m[2] = a.z;
        m[3] = b.x; m[4] = b.y; m[5] = b.z;
        m[6] = c.x; m[7] = c.y; m[8] = c.z;
    }
}

template <int DIM>
__device__ __forceinline__ void store_M(float4* M, int64_t i, const float* m) {
    if (DIM == 2) {
        M[i] = make_float4(m[0], m[1], m[2], m[3]);
    } else {
        M[3 * i] = make_float4(m[0], m[1], m[2], 0.0f);
        M[3 * i + 1] = make_float4(m[3], m[4], m[5], 0.0f);
        M[3 * i + 2] = make_float4(m[6], m[7], m[8], 0.0f);
    }
}

template <int DIM>
__device__ __forceinline__ void pair_r32(const float* xhi, const float* xli, const float* xhj, const float* xlj,
                                         const TLK<float>& K, float* r, float& d2) {
    d2 = 0.0f;
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
}

template <int DIM>
__global__ void k_tl_stress32(const float* __restrict__ H, const float* __restrict__ B0, int64_t n, TLK<float> K,
                              float4* __restrict__ M) {
    constexpr int NS = DIM == 2 ? 3 : 6;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float h[DIM * DIM], b[NS], m[DIM * DIM];
    for (int k = 0; k < DIM * DIM; ++k) h[k] = H[k * n + i];
    for (int s = 0; s < NS; ++s) b[s] = B0[s * n + i];
    stress_factor<DIM, float>(h, b, K, m);
    store_M<DIM>(M, i, m);
}

template <int DIM, int OUT, int LANES>
__global__ void __launch_bounds__(256) k_tl_mom32(const float4* __restrict__ geo, const int64_t* __restrict__ row_ptr,
                                                  const int32_t* __restrict__ col, int64_t n, TLK<float> K,
                                                  const float4* __restrict__ M, float4* __restrict__ vq,
                                                  double* __restrict__ dvdt) {
    int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t i = gt / LANES;
    int lane = (int)(gt % LANES);
    bool active = i < n;
    int64_t ii = active ? i : 0;
    float xhi[DIM], xli[DIM], Vi, fx, Mi[DIM * DIM];
    load_geo<DIM>(geo, ii, xhi, xli, Vi, fx);
    load_M<DIM>(M, ii, Mi);
    Kahan<float> acc[DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a) acc[a].init();
    int64_t b = active ? row_ptr[ii] : 0, e = active ? row_ptr[ii + 1] : 0;
    for (int64_t p = b + lane; p < e; p += LANES) {
        int j = __ldg(&col[p]);
        float xhj[DIM], xlj[DIM], Vj, fj, Mj[DIM * DIM];
        load_geo<DIM>(geo, j, xhj, xlj, Vj, fj);
        load_M<DIM>(M, j, Mj);
        float r[DIM], d2;
        pair_r32<DIM>(xhi, xli, xhj, xlj, K, r, d2);
        float gs = wendland_gs<float>(sqrtf(d2) * K.inv_h, K.coef) * Vj;
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            float s = 0.0f;
#pragma unroll
            for (int c = 0; c < DIM; ++c) s = fmaf(Mi[a * DIM + c] + Mj[a * DIM + c], gs * r[c], s);
            acc[a].add(s);
        }
    }
    float tot[DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a) tot[a] = group_sum<LANES>(acc[a].value());
    if (!active || lane != 0) return;
    if (OUT == OUT_RATES) {
        for (int a = 0; a < DIM; ++a) dvdt[a * n + i] = (double)(tot[a] * K.inv_rho0);
        return;
    }
    float4 vv = vq[i];
    float vn[3] = {vv.x, vv.y, vv.z};
#pragma unroll
    for (int a = 0; a < DIM; ++a) vn[a] = fx != 0.0f ? 0.0f : vn[a] + K.dt * (tot[a] * K.inv_rho0);
    vq[i] = make_float4(vn[0], vn[1], DIM == 3 ? vn[2] : 0.0f, 0.0f);
}

template <int DIM, int OUT, int LANES>
__global__ void __launch_bounds__(256) k_tl_defo32(const float4* __restrict__ geo, const int64_t* __restrict__ row_ptr,
                                                   const int32_t* __restrict__ col, int64_t n, TLK<float> K,
                                                   const float4* __restrict__ vq, const float* __restrict__ B0,
                                                   float* __restrict__ H, float* __restrict__ u,
                                                   float4* __restrict__ M, double* __restrict__ dFdt) {
    constexpr int NS = DIM == 2 ? 3 : 6;
    int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t i = gt / LANES;
    int lane = (int)(gt % LANES);
    bool active = i < n;
    int64_t ii = active ? i : 0;
    float xhi[DIM], xli[DIM], Vi, fx, vi[DIM];
    load_geo<DIM>(geo, ii, xhi, xli, Vi, fx);
    float4 vv = __ldg(&vq[ii]);
    vi[0] = vv.x; vi[1] = vv.y;
    if (DIM == 3) vi[DIM - 1] = vv.z;
    Kahan<float> L[DIM * DIM];
#pragma unroll
    for (int k = 0; k < DIM * DIM; ++k) L[k].init();
    int64_t b = active ? row_ptr[ii] : 0, e = active ? row_ptr[ii + 1] : 0;
    for (int64_t p = b + lane; p < e; p += LANES) {
        int j = __ldg(&col[p]);
        float xhj[DIM], xlj[DIM], Vj, fj;
        load_geo<DIM>(geo, j, xhj, xlj, Vj, fj);
        float4 vjv = __ldg(&vq[j]);
        float vj[3] = {vjv.x, vjv.y, vjv.z};
        float r[DIM], d2;
        pair_r32<DIM>(xhi, xli, xhj, xlj, K, r, d2);
        float gs = wendland_gs<float>(sqrtf(d2) * K.inv_h, K.coef);
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            float dv = Vj * (vj[a] - vi[a]);
#pragma unroll
            for (int c = 0; c < DIM; ++c) L[a * DIM + c].add(dv * (gs * r[c]));
        }
    }
    float Lt[DIM * DIM];
#pragma unroll
    for (int k = 0; k < DIM * DIM; ++k) Lt[k] = group_sum<LANES>(L[k].value());
    if (!active || lane != 0) return;
    float b0[NS], Fd[DIM * DIM];
#pragma unroll
    for (int s = 0; s < NS; ++s) b0[s] = B0[s * n + i];
    times_b0<DIM, float>(Lt, b0, Fd);
    if (OUT == OUT_RATES) {
        for (int k = 0; k < DIM * DIM; ++k) dFdt[k * n + i] = (double)Fd[k];
        return;
    }
    float h[DIM * DIM], m[DIM * DIM];
#pragma unroll
    for (int k = 0; k < DIM * DIM; ++k) {
        h[k] = fx != 0.0f ? 0.0f : H[k * n + i] + K.dt * Fd[k];
        H[k * n + i] = h[k];
    }
#pragma unroll
    for (int a = 0; a < DIM; ++a) u[a * n + i] += K.dt * vi[a];
    stress_factor<DIM, float>(h, b0, K, m);
    store_M<DIM>(M, i, m);
}

// ---------------------------------------------------------------- pack / unpack
template <int DIM>
__global__ void k_tl_pack(const double* __restrict__ r0, const double* __restrict__ V0,
                          const double* __restrict__ B0, const uint8_t* __restrict__ fixed,
                          const double* __restrict__ x, const double* __restrict__ v,
                          const double* __restrict__ H, int64_t n, float* __restrict__ geo,
                          float4* __restrict__ vq, float* __restrict__ H32, float* __restrict__ u32,
                          float* __restrict__ B32) {
    constexpr int NS = DIM == 2 ? 3 : 6;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float xh[3] = {0, 0, 0}, xl[3] = {0, 0, 0};
    for (int a = 0; a < DIM; ++a) {
        double xv = r0[a * n + i];
        xh[a] = (float)xv;
        xl[a] = (float)(xv - (double)xh[a]);
    }
    float fx = (fixed && fixed[i]) ? 1.0f : 0.0f;
    float* g = geo + 8 * i;
    if (DIM == 2) {
        g[0] = xh[0]; g[1] = xh[1]; g[2] = xl[0]; g[3] = xl[1];
        g[4] = (float)V0[i]; g[5] = fx; g[6] = 0.0f; g[7] = 0.0f;
    } else {
        g[0] = xh[0]; g[1] = xh[1]; g[2] = xh[2]; g[3] = (float)V0[i];
        g[4] = xl[0]; g[5] = xl[1]; g[6] = xl[2]; g[7] = fx;
    }
    float vv[3] = {0, 0, 0};
    for (int a = 0; a < DIM; ++a) vv[a] = (float)v[a * n + i];
    vq[i] = make_float4(vv[0], vv[1], vv[2], 0.0f);
    for (int k = 0; k < DIM * DIM; ++k) H32[k * n + i] = (float)H[k * n + i];
    for (int a = 0; a < DIM; ++a) u32[a * n + i] = (float)(x[a * n + i] - r0[a * n + i]);
    for (int s = 0; s < NS; ++s) B32[s * n + i] = (float)B0[s * n + i];
}

template <int DIM>
__global__ void k_tl_unpack(const double* __restrict__ r0, const float4* __restrict__ vq,
                            const float* __restrict__ H32, const float* __restrict__ u32, int64_t n,
                            double* __restrict__ x, double* __restrict__ v, double* __restrict__ H) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float4 vv = vq[i];
    float vc[3] = {vv.x, vv.y, vv.z};
    for (int a = 0; a < DIM; ++a) {
        v[a * n + i] = vc[a];
        x[a * n + i] = r0[a * n + i] + (double)u32[a * n + i];
    }
    for (int k = 0; k < DIM * DIM; ++k) H[k * n + i] = H32[k * n + i];
}

template <typename R>
TLK<R> make_tl_consts(const sph_tlsph_params* p) {
    TLK<R> K;
    const sph_domain& d = p->dom;
    double h = d.h;
    double hd2 = d.dim == 2 ? h * h * h * h : h * h * h * h * h;
    K.coef = (R)(-5.0 * wendland_alpha(d.dim) / hd2);
    K.inv_h = (R)(1.0 / h);
    K.inv_rho0 = (R)(1.0 / p->rho0);
    K.dt = (R)p->dt;
    K.lam = (R)p->lambda;
    K.G = (R)p->G;
    K.law = p->law;
    K.periodic = d.periodic_mask;
    for (int a = 0; a < 3; ++a) {
        K.half[a] = (R)(0.5 * d.len[a]);
        K.Lh[a] = (R)d.len[a];
        K.Ll[a] = (R)(d.len[a] - (double)K.Lh[a]);
    }
    return K;
}

int check_tl(const sph_tlsph_params* p, const sph_tlsph_state* st) {
    if (!p || !st) return SPH_ERR_ARG;
    int s = sph_check_domain(&p->dom);
    if (s) return s;
    if (p->precision != SPH_FP64 && p->precision != SPH_FP32_KAHAN) return SPH_ERR_ARG;
    if (p->law != SPH_SVK && p->law != SPH_NEO_HOOKEAN) return SPH_ERR_ARG;
    if (!(p->rho0 > 0.0)) return SPH_ERR_ARG;
    if (p->dom.n > 0 && (!st->row_ptr || !st->col || !st->r0 || !st->V0 || !st->B0)) return SPH_ERR_ARG;
    return SPH_OK;
}

template <int DIM, int LANES>
void tl32_passes(int which, int out, int64_t n, const sph_tlsph_state* st, const TLK<float>& K, double* r1, double* r2,
                 cudaStream_t s) {
    const int block = 256;
    dim3 g(grid_for(n * LANES, block)), b(block);
    const float4* geo = reinterpret_cast<const float4*>(st->geo);
    float4* M = reinterpret_cast<float4*>(st->M32);
    float4* vq = reinterpret_cast<float4*>(st->vq);
    if (which == 0) {
        if (out == OUT_RATES) k_tl_mom32<DIM, OUT_RATES, LANES><<<g, b, 0, s>>>(geo, st->row_ptr, st->col, n, K, M, vq, r1);
        else k_tl_mom32<DIM, OUT_STEP, LANES><<<g, b, 0, s>>>(geo, st->row_ptr, st->col, n, K, M, vq, nullptr);
    } else {
        if (out == OUT_RATES)
            k_tl_defo32<DIM, OUT_RATES, LANES><<<g, b, 0, s>>>(geo, st->row_ptr, st->col, n, K, vq, st->B32, st->H32,
                                                              st->u32, M, r2);
        else
            k_tl_defo32<DIM, OUT_STEP, LANES><<<g, b, 0, s>>>(geo, st->row_ptr, st->col, n, K, vq, st->B32, st->H32,
                                                             st->u32, M, nullptr);
    }
}

template <int DIM>
void tl32(int lanes, int which, int out, int64_t n, const sph_tlsph_state* st, const TLK<float>& K, double* r1,
          double* r2, cudaStream_t s) {
    switch (lanes) {
        case 1: tl32_passes<DIM, 1>(which, out, n, st, K, r1, r2, s); break;
        case 2: tl32_passes<DIM, 2>(which, out, n, st, K, r1, r2, s); break;
        case 8: tl32_passes<DIM, 8>(which, out, n, st, K, r1, r2, s); break;
        default: tl32_passes<DIM, 4>(which, out, n, st, K, r1, r2, s); break;
    }
}

bool fp32_ready(const sph_tlsph_state* st) {
    return st->geo && st->vq && st->H32 && st->u32 && st->M32 && st->B32;
}
bool fp64_ready(const sph_tlsph_state* st) { return st->x && st->v && st->H && st->M; }

}  // namespace

extern "C" int sph_tlsph_pack(sph_ctx* ctx, const sph_tlsph_params* p, const sph_tlsph_state* st, void* stream) {
    if (!ctx) return SPH_ERR_ARG;
    int r = check_tl(p, st);
    if (r) return r;
    int64_t n = p->dom.n;
    if (n == 0) return SPH_OK;
    if (!fp32_ready(st) || !st->x || !st->v || !st->H) return SPH_ERR_ARG;
    cudaStream_t s = as_stream(stream);
    float4* vq = reinterpret_cast<float4*>(st->vq);
    if (p->dom.dim == 2)
        k_tl_pack<2><<<grid_for(n, 256), 256, 0, s>>>(st->r0, st->V0, st->B0, st->fixed, st->x, st->v, st->H, n, st->geo,
                                                      vq, st->H32, st->u32, st->B32);
    else
        k_tl_pack<3><<<grid_for(n, 256), 256, 0, s>>>(st->r0, st->V0, st->B0, st->fixed, st->x, st->v, st->H, n, st->geo,
                                                      vq, st->H32, st->u32, st->B32);
    SPH_LAUNCH_CHECK(ctx);
    return SPH_OK;
}

extern "C" int sph_tlsph_unpack(sph_ctx* ctx, const sph_tlsph_params* p, const sph_tlsph_state* st, void* stream) {
    if (!ctx) return SPH_ERR_ARG;
    int r = check_tl(p, st);
    if (r) return r;
    int64_t n = p->dom.n;
    if (n == 0) return SPH_OK;
    if (!st->vq || !st->H32 || !st->u32 || !st->x || !st->v || !st->H) return SPH_ERR_ARG;
    cudaStream_t s = as_stream(stream);
    const float4* vq = reinterpret_cast<const float4*>(st->vq);
    if (p->dom.dim == 2)
        k_tl_unpack<2><<<grid_for(n, 256), 256, 0, s>>>(st->r0, vq, st->H32, st->u32, n, st->x, st->v, st->H);
    else
        k_tl_unpack<3><<<grid_for(n, 256), 256, 0, s>>>(st->r0, vq, st->H32, st->u32, n, st->x, st->v, st->H);
    SPH_LAUNCH_CHECK(ctx);
    return SPH_OK;
}

extern "C" int sph_tlsph_rates(sph_ctx* ctx, const sph_tlsph_params* p, const sph_tlsph_state* st, double* dvdt,
                               double* dFdt, void* stream) {
    if (!ctx) return SPH_ERR_ARG;
    int r = check_tl(p, st);
    if (r) return r;
    int64_t n = p->dom.n;
    if (n == 0) return SPH_OK;
    if (!dvdt || !dFdt) return SPH_ERR_ARG;
    cudaStream_t s = as_stream(stream);
    int dim = p->dom.dim;
    if (p->precision == SPH_FP64) {
        if (!fp64_ready(st)) return SPH_ERR_ARG;
        TLK<double> K = make_tl_consts<double>(p);
        dim3 g(grid_for(n, 128)), b(128);
        if (dim == 2) {
            k_tl_stress64<2><<<g, b, 0, s>>>(st->H, st->B0, n, K, st->M);
            k_tl_mom64<2, OUT_RATES><<<g, b, 0, s>>>(st->r0, st->V0, st->fixed, st->row_ptr, st->col, n, K, st->M, nullptr, dvdt);
            k_tl_defo64<2, OUT_RATES><<<g, b, 0, s>>>(st->r0, st->V0, st->B0, st->fixed, st->row_ptr, st->col, n, K, st->v,
                                                      nullptr, nullptr, nullptr, dFdt);
        } else {
            k_tl_stress64<3><<<g, b, 0, s>>>(st->H, st->B0, n, K, st->M);
            k_tl_mom64<3, OUT_RATES><<<g, b, 0, s>>>(st->r0, st->V0, st->fixed, st->row_ptr, st->col, n, K, st->M, nullptr, dvdt);
            k_tl_defo64<3, OUT_RATES><<<g, b, 0, s>>>(st->r0, st->V0, st->B0, st->fixed, st->row_ptr, st->col, n, K, st->v,
                                                      nullptr, nullptr, nullptr, dFdt);
        }
    } else {
        if (!fp32_ready(st)) return SPH_ERR_ARG;
        TLK<float> K = make_tl_consts<float>(p);
        int lanes = ctx->lanes[SPH_PASS_TLSPH];
        float4* M = reinterpret_cast<float4*>(st->M32);
        if (dim == 2) {
            k_tl_stress32<2><<<grid_for(n, 128), 128, 0, s>>>(st->H32, st->B32, n, K, M);
            tl32<2>(lanes, 0, OUT_RATES, n, st, K, dvdt, dFdt, s);
            tl32<2>(lanes, 1, OUT_RATES, n, st, K, dvdt, dFdt, s);
        } else {
            k_tl_stress32<3><<<grid_for(n, 128), 128, 0, s>>>(st->H32, st->B32, n, K, M);
            tl32<3>(lanes, 0, OUT_RATES, n, st, K, dvdt, dFdt, s);
            tl32<3>(lanes, 1, OUT_RATES, n, st, K, dvdt, dFdt, s);
        }
    }
    SPH_LAUNCH_CHECK(ctx);
    return SPH_OK;
}

extern "C" int sph_tlsph_step(sph_ctx* ctx, const sph_tlsph_params* p, const sph_tlsph_state* st, int nsteps,
                              void* stream) {
    if (!ctx || nsteps < 0) return SPH_ERR_ARG;
    int r = check_tl(p, st);
    if (r) return r;
    int64_t n = p->dom.n;
    if (n == 0 || nsteps == 0) return SPH_OK;
    cudaStream_t s = as_stream(stream);
    int dim = p->dom.dim;
    if (p->precision == SPH_FP64) {
        if (!fp64_ready(st)) return SPH_ERR_ARG;
        TLK<double> K = make_tl_consts<double>(p);
        dim3 g(grid_for(n, 128)), b(128);
        int t = sph_timer_begin(ctx, SPH_TIMER_TL_STRESS, s);
        if (dim == 2) k_tl_stress64<2><<<g, b, 0, s>>>(st->H, st->B0, n, K, st->M);
        else k_tl_stress64<3><<<g, b, 0, s>>>(st->H, st->B0, n, K, st->M);
        sph_timer_end(ctx, t, s);
        for (int k = 0; k < nsteps; ++k) {
            t = sph_timer_begin(ctx, SPH_TIMER_TL_MOMENTUM, s);
            if (dim == 2)
                k_tl_mom64<2, OUT_STEP><<<g, b, 0, s>>>(st->r0, st->V0, st->fixed, st->row_ptr, st->col, n, K, st->M, st->v, nullptr);
            else
                k_tl_mom64<3, OUT_STEP><<<g, b, 0, s>>>(st->r0, st->V0, st->fixed, st->row_ptr, st->col, n, K, st->M, st->v, nullptr);
            sph_timer_end(ctx, t, s);
            t = sph_timer_begin(ctx, SPH_TIMER_TL_DEFORM, s);
            if (dim == 2)
                k_tl_defo64<2, OUT_STEP><<<g, b, 0, s>>>(st->r0, st->V0, st->B0, st->fixed, st->row_ptr, st->col, n, K, st->v,
                                                         st->H, st->x, st->M, nullptr);
            else
                k_tl_defo64<3, OUT_STEP><<<g, b, 0, s>>>(st->r0, st->V0, st->B0, st->fixed, st->row_ptr, st->col, n, K, st->v,
                                                         st->H, st->x, st->M, nullptr);
            sph_timer_end(ctx, t, s);
        }
        SPH_LAUNCH_CHECK(ctx);
        return SPH_OK;
    }
    if (!fp32_ready(st)) return SPH_ERR_ARG;
    TLK<float> K = make_tl_consts<float>(p);
    int lanes = ctx->lanes[SPH_PASS_TLSPH];
    float4* M = reinterpret_cast<float4*>(st->M32);
    int t = sph_timer_begin(ctx, SPH_TIMER_TL_STRESS, s);
    if (dim == 2) k_tl_stress32<2><<<grid_for(n, 128), 128, 0, s>>>(st->H32, st->B32, n, K, M);
    else k_tl_stress32<3><<<grid_for(n, 128), 128, 0, s>>>(st->H32, st->B32, n, K, M);
    sph_timer_end(ctx, t, s);
    for (int k = 0; k < nsteps; ++k) {
        t = sph_timer_begin(ctx, SPH_TIMER_TL_MOMENTUM, s);
        if (dim == 2) tl32<2>(lanes, 0, OUT_STEP, n, st, K, nullptr, nullptr, s);
        else tl32<3>(lanes, 0, OUT_STEP, n, st, K, nullptr, nullptr, s);
        sph_timer_end(ctx, t, s);
        t = sph_timer_begin(ctx, SPH_TIMER_TL_DEFORM, s);
        if (dim == 2) tl32<2>(lanes, 1, OUT_STEP, n, st, K, nullptr, nullptr, s);
        else tl32<3>(lanes, 1, OUT_STEP, n, st, K, nullptr, nullptr, s);
        sph_timer_end(ctx, t, s);
    }
    SPH_LAUNCH_CHECK(ctx);
    return SPH_OK;
}
