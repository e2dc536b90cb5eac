// Per-pair physics and packed-record helpers of the Eulerian WCSPH passes, shared by the
// single-case kernels (eulerian.cu) and the batched persistent kernel (batched.cu).
#pragma once
#include "common.cuh"

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
template <int DIM> struct Rec32;
template <> struct Rec32<2> { static constexpr int words = 2; };
template <> struct Rec32<3> { static constexpr int words = 4; };

template <int DIM>
__device__ __forceinline__ void load_geo32(const float4* __restrict__ geo, int64_t i, float* xh, float* xl,
                                           float& V, float* Bs) {
    if (DIM == 2) {
        float4 a = __ldg(&geo[2 * i]);
        float4 b = __ldg(&geo[2 * i + 1]);
        xh[0] = a.x; xh[1] = a.y; xl[0] = a.z; xl[1] = a.w;
        V = b.x; Bs[0] = b.y; Bs[1] = b.z; Bs[2] = b.w;
    } else {
        float4 a = __ldg(&geo[4 * i]);
        float4 b = __ldg(&geo[4 * i + 1]);
        float4 c = __ldg(&geo[4 * i + 2]);
        float d = __ldg(reinterpret_cast<const float*>(&geo[4 * i + 3]));
        xh[0] = a.x; xh[1] = a.y; xh[2] = a.z; V = a.w;
        xl[0] = b.x; xl[1] = b.y; xl[2] = b.z; Bs[0] = b.w;
        Bs[1] = c.x; Bs[2] = c.y; Bs[3] = c.z; Bs[4] = c.w; Bs[5] = d;
    }
}

template <int DIM>
__device__ __forceinline__ void load_q32(const float4* __restrict__ q, int64_t i, float* v, float& drho) {
    float4 a = __ldg(&q[i]);
    if (DIM == 2) { v[0] = a.x; v[1] = a.y; drho = a.z; }
    else { v[0] = a.x; v[1] = a.y; v[2] = a.z; drho = a.w; }
}

template <int DIM>
__device__ __forceinline__ void store_q32(float4* q, int64_t i, const float* v, float drho) {
    float4 a;
    if (DIM == 2) { a.x = v[0]; a.y = v[1]; a.z = drho; a.w = 0.0f; }
    else { a.x = v[0]; a.y = v[1]; a.z = v[2]; a.w = drho; }
    q[i] = a;
}


}  // namespace euler
